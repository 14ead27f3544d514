// The per-C-block body of the FP64 numeric phase, shared by every kernel
// that sums FP64 block products on the DMMA pipe (the library's single and
// batched forms and the allocation-free entry point), so that there is one
// copy of its copy ring, bounds check, timeout unwind and epilogue.
//
// One CTA of 128 threads sums the block products seg[c] .. seg[c+1]-1 of C
// block c in ascending list order: each (A_IK, B_KJ) pair is staged into shared memory
// by two 1-D bulk copies completing on an mbarrier, a kFp64Stages-deep ring
// overlaps the next pair's copies with the current pair's DMMAs, and the sum
// stays in registers until one store (Sec. 4.1, Fig. 3: the leaf multiply as
// a sum of block products, here with one owner per C block and no atomics).
#pragma once

#include "bsm_ptx.cuh"

namespace {

constexpr int kFp64Stages = 2;  // bulk-copy ring depth

__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// Sums the products seg[c] .. seg[c+1]-1 into C block c (all 128 threads of
// the CTA).  use0 / use1 count the completed phases of the two stage barriers
// across calls.  Returns false (after recording the error) on a bad index or a
// timed-out wait; every thread returns the same value.
// Two forms of the arithmetic, bit-compatible with nothing but themselves:
// MODE 0 sums on the FP64 tensor pipe (mma.sync m8n8k4, 2 x 2 warps of 8 x 8
// tiles); MODE >= 1 with scalar DFMA, every output summed one k at a time in
// ascending order (a plain dot product of fused multiply-adds), each thread a
// tile of TR x TC outputs: TC = BS/8 (MODE 1), BS/16 (MODE 2) or BS/4
// (MODE 3; at most BS^2/128, one row per thread) consecutive columns of
// TR = BS^2 / (128 TC) rows 128 TC / BS apart.  The DFMA tiles give identical
// results (same order per output).
template <int BS, int MODE>
struct DfmaTile {
  static constexpr int TC = MODE == 2 ? BS / 16
                                      : (MODE == 3 ? (BS / 4 < BS * BS / 128 ? BS / 4 : BS * BS / 128)
                                                   : BS / 8);
  static constexpr int TPR = BS / TC;       // threads per row
  static constexpr int RS = 128 / TPR;      // row stride between a thread's rows
  static constexpr int TR = BS / RS;
  static_assert(TR >= 1 && TR * RS == BS && TC * TPR == BS, "thread tile");
};

template <int BS, int MODE>
__device__ bool cblock_fp64(const int32_t *__restrict__ seg, const int32_t *__restrict__ ta,
                            const int32_t *__restrict__ tb, int64_t c, int64_t na, int64_t nb,
                            const double *__restrict__ Av, const double *__restrict__ Bv,
                            double *__restrict__ Cv, int32_t *__restrict__ nzflag,
                            unsigned *__restrict__ err, double *smem, uint64_t *full,
                            uint32_t &use0, uint32_t &use1) {
  constexpr int BB = BS * BS;
  constexpr int WT = BS / 2;   // warp tile side (2 x 2 warps)
  constexpr int TW = WT / 8;   // 8x8 DMMA tiles per warp tile side
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wr = warp >> 1, wc = warp & 1;
  const int32_t k0 = seg[c], nk = seg[c + 1] - k0;
  // every block index is checked before any copy is issued
  bool bad = nk < 0;
  for (int j = tid; j < nk; j += blockDim.x)
    bad |= ta[k0 + j] < 0 || ta[k0 + j] >= na || tb[k0 + j] < 0 || tb[k0 + j] >= nb;
  if (__syncthreads_or(bad)) {
    if (tid == 0) set_err(err, DERR_BOUNDS);
    return false;
  }
  auto issue = [&](int j) {
    int s = j % kFp64Stages;
    double *sa = smem + (size_t)s * 2 * BB;
    mbar_expect_tx(&full[s], 2u * BB * 8u);
    bulk_g2s(sa, Av + (int64_t)ta[k0 + j] * BB, BB * 8u, &full[s]);
    bulk_g2s(sa + BB, Bv + (int64_t)tb[k0 + j] * BB, BB * 8u, &full[s]);
  };
  if (tid == 0)
    for (int j = 0; j < kFp64Stages && j < nk; j++) issue(j);

  double acc[TW][TW][2];
#pragma unroll
  for (int i = 0; i < TW; i++)
#pragma unroll
    for (int j = 0; j < TW; j++) acc[i][j][0] = acc[i][j][1] = 0.0;
  // DFMA form: rows i * RS + tid / TPR, columns (tid % TPR) * TC + x
  using DT = DfmaTile<BS, MODE>;
  constexpr int TR = DT::TR, TC = DT::TC, RS = DT::RS, TPR = DT::TPR;
  double fac[TR][TC];
#pragma unroll
  for (int i = 0; i < TR; i++)
#pragma unroll
    for (int x = 0; x < TC; x++) fac[i][x] = 0.0;
  const int frow = tid / TPR, fcol = (tid % TPR) * TC;

  const int ar = lane >> 2, ak = lane & 3;
  bool ok = true;
  int jfail = 0;
  for (int j = 0; j < nk; j++) {
    const int s = j % kFp64Stages;
    const uint32_t par = (s == 0 ? use0 : use1) & 1u;
    if (!mbar_wait(&full[s], par)) ok = false;
    // every thread takes the same path: a failed wait aborts the whole CTA
    if (__syncthreads_or(!ok)) {
      ok = false;
      jfail = j;
      break;
    }
    if (s == 0)
      use0++;
    else
      use1++;
    const double *sa = smem + (size_t)s * 2 * BB;
    const double *sb = sa + BB;
    if constexpr (MODE >= 1) {
#pragma unroll 4
      for (int kk = 0; kk < BS; kk++) {
        double a[TR], b[TC];
#pragma unroll
        for (int i = 0; i < TR; i++) a[i] = sa[(i * RS + frow) * BS + kk];
        if constexpr (TC % 2 == 0) {
#pragma unroll
          for (int x = 0; x < TC; x += 2) {
            const double2 v = *reinterpret_cast<const double2 *>(sb + kk * BS + fcol + x);
            b[x] = v.x;
            b[x + 1] = v.y;
          }
        } else {
#pragma unroll
          for (int x = 0; x < TC; x++) b[x] = sb[kk * BS + fcol + x];
        }
#pragma unroll
        for (int i = 0; i < TR; i++)
#pragma unroll
          for (int x = 0; x < TC; x++) fac[i][x] = fma(a[i], b[x], fac[i][x]);
      }
    } else {
#pragma unroll 2
    for (int kk = 0; kk < BS; kk += 4) {
      double a[TW], b[TW];
#pragma unroll
      for (int i = 0; i < TW; i++) a[i] = sa[(wr * WT + i * 8 + ar) * BS + kk + ak];
#pragma unroll
      for (int i = 0; i < TW; i++) b[i] = sb[(kk + ak) * BS + wc * WT + i * 8 + ar];
#pragma unroll
      for (int i = 0; i < TW; i++)
#pragma unroll
        for (int q = 0; q < TW; q++) dmma_8x8x4(acc[i][q], a[i], b[q]);
    }
    }
    __syncthreads();  // stage s fully consumed
    if (tid == 0 && j + kFp64Stages < nk) issue(j + kFp64Stages);
  }
  if (!ok) {
    if (tid == 0) {
      set_err(err, DERR_TIMEOUT);
      // let copies still in flight land before shared memory is reused
      for (int j = jfail; j < jfail + kFp64Stages && j < nk; j++) {
        const int s = j % kFp64Stages;
        mbar_wait(&full[s], (s == 0 ? use0 : use1) & 1u);
      }
    }
    return false;
  }
  bool any = false;
  double *cb = Cv + c * BB;
  if constexpr (MODE >= 1) {
#pragma unroll
    for (int i = 0; i < TR; i++) {
      if constexpr (TC % 2 == 0) {
#pragma unroll
        for (int x = 0; x < TC; x += 2) {
          any |= nonzero_f64(fac[i][x]) | nonzero_f64(fac[i][x + 1]);
          *reinterpret_cast<double2 *>(cb + (i * RS + frow) * BS + fcol + x) =
              make_double2(fac[i][x], fac[i][x + 1]);
        }
      } else {
#pragma unroll
        for (int x = 0; x < TC; x++) {
          any |= nonzero_f64(fac[i][x]);
          cb[(i * RS + frow) * BS + fcol + x] = fac[i][x];
        }
      }
    }
  } else {
#pragma unroll
  for (int i = 0; i < TW; i++)
#pragma unroll
    for (int q = 0; q < TW; q++) {
      any |= nonzero_f64(acc[i][q][0]) | nonzero_f64(acc[i][q][1]);
      int row = wr * WT + i * 8 + ar, col = wc * WT + q * 8 + 2 * ak;
      *reinterpret_cast<double2 *>(cb + row * BS + col) = make_double2(acc[i][q][0], acc[i][q][1]);
    }
  }
  int nzb = __syncthreads_or(any);
  if (tid == 0) nzflag[c] = nzb;
  return true;
}


}  // namespace
