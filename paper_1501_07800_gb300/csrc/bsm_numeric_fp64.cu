// FP64 numeric phase: C_IJ = sum_K A_IK B_KJ on the FP64 tensor pipe.
//
// This is the leaf multiply of Sec. 4.1 (a sum of outer products, Fig. 3) with
// the batching turned around: instead of one batched GEMM per outer product,
// whose products must not share an output block, each C block is owned by one
// CTA that walks the block's (A_IK, B_KJ) list in ascending K and keeps the sum
// in registers -- no two writers per C block, no atomics, one store.
//
// Leaf blocks are contiguous bs*bs*8-byte records, so each is staged into
// shared memory by one 1-D bulk copy (cp.async.bulk) completing on an
// mbarrier; a two-stage ring overlaps the next pair's copy with the current
// pair's DMMA (mma.sync m8n8k4 f64).  tcgen05 has no f64 kind, and on GB300 the
// FP64 rate of DMMA and DFMA is the same ~1 TFLOP/s, far below what the copies
// can feed, so the kernel only has to keep the FP64 pipe busy.  The epilogue
// also raises the C block's nonzero flag (exact-zero detection).
//
// Two launch forms share the per-C-block body: one CTA per C block of a single
// product, and a persistent form that walks a global work list of
// (product, C block) items of many independent products (batched products),
// claiming items from an atomic counter in the list's order.
#include "bsm_batch.cuh"
#include "bsm_ptx.cuh"

namespace {

constexpr int kStages = 2;

__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// Sums the products seg[c] .. seg[c+1]-1 into C block c (all 128 threads of
// the CTA).  use0 / use1 count the completed phases of the two stage barriers
// across calls.  Returns false (after recording the error) on a bad index or a
// timed-out wait; every thread returns the same value.
template <int BS>
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
    int s = j % kStages;
    double *sa = smem + (size_t)s * 2 * BB;
    mbar_expect_tx(&full[s], 2u * BB * 8u);
    bulk_g2s(sa, Av + (int64_t)ta[k0 + j] * BB, BB * 8u, &full[s]);
    bulk_g2s(sa + BB, Bv + (int64_t)tb[k0 + j] * BB, BB * 8u, &full[s]);
  };
  if (tid == 0)
    for (int j = 0; j < kStages && j < nk; j++) issue(j);

  double acc[TW][TW][2];
#pragma unroll
  for (int i = 0; i < TW; i++)
#pragma unroll
    for (int j = 0; j < TW; j++) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int ar = lane >> 2, ak = lane & 3;
  bool ok = true;
  int jfail = 0;
  for (int j = 0; j < nk; j++) {
    const int s = j % kStages;
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
    __syncthreads();  // stage s fully consumed
    if (tid == 0 && j + kStages < nk) issue(j + kStages);
  }
  if (!ok) {
    if (tid == 0) {
      set_err(err, DERR_TIMEOUT);
      // let copies still in flight land before shared memory is reused
      for (int j = jfail; j < jfail + kStages && j < nk; j++) {
        const int s = j % kStages;
        mbar_wait(&full[s], (s == 0 ? use0 : use1) & 1u);
      }
    }
    return false;
  }
  bool any = false;
  double *cb = Cv + c * BB;
#pragma unroll
  for (int i = 0; i < TW; i++)
#pragma unroll
    for (int q = 0; q < TW; q++) {
      any |= nonzero_f64(acc[i][q][0]) | nonzero_f64(acc[i][q][1]);
      int row = wr * WT + i * 8 + ar, col = wc * WT + q * 8 + 2 * ak;
      *reinterpret_cast<double2 *>(cb + row * BS + col) = make_double2(acc[i][q][0], acc[i][q][1]);
    }
  int nzb = __syncthreads_or(any);
  if (tid == 0) nzflag[c] = nzb;
  return true;
}

template <int BS>
__global__ void __launch_bounds__(128) k_numeric_fp64(
    const int32_t *__restrict__ seg, const int32_t *__restrict__ ta, const int32_t *__restrict__ tb,
    int64_t nc, int64_t na, int64_t nb, const double *__restrict__ Av,
    const double *__restrict__ Bv, double *__restrict__ Cv, int32_t *__restrict__ nzflag,
    unsigned *__restrict__ err) {
  extern __shared__ __align__(128) double smem[];  // [kStages][2][BS*BS]
  __shared__ __align__(8) uint64_t full[kStages];
  const int64_t c = blockIdx.x;
  if (c >= nc) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t use0 = 0, use1 = 0;
  cblock_fp64<BS>(seg, ta, tb, c, na, nb, Av, Bv, Cv, nzflag, err, smem, full, use0, use1);
}

// Persistent form over a global work list of (product, C block) items.
template <int BS>
__global__ void __launch_bounds__(128) k_numeric_fp64_batched(const ProdDesc *__restrict__ prods,
                                                              const uint64_t *__restrict__ items,
                                                              int64_t nitems,
                                                              unsigned long long *counter,
                                                              unsigned *__restrict__ err) {
  extern __shared__ __align__(128) double smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ unsigned long long next_item;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t use0 = 0, use1 = 0;
  for (;;) {
    if (threadIdx.x == 0) next_item = atomicAdd(counter, 1ull);
    __syncthreads();
    const unsigned long long w = next_item;
    __syncthreads();
    if ((int64_t)w >= nitems) break;
    const uint64_t it = items[w];
    const ProdDesc &p = prods[item_product(it)];
    if (!cblock_fp64<BS>(p.seg, p.ta, p.tb, item_cblock(it), p.na, p.nb, p.av, p.bv, p.cv, p.nz,
                         err, smem, full, use0, use1))
      break;
  }
}

template <int BS>
bsm_status launch(const SymbolicResult &sym, bsm_matrix A, bsm_matrix B, double *Cv, int32_t *nz,
                  unsigned *err, cudaStream_t s) {
  size_t smem = (size_t)kStages * 2 * BS * BS * sizeof(double);
  static std::atomic<uint64_t> attr{0};
  BSM_TRY(once_per_device(attr, [&] {
    return cuda_status(cudaFuncSetAttribute(
        k_numeric_fp64<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }));
  // one CTA per C block (nc < 2^31 is checked by the caller)
  count_launch();
  k_numeric_fp64<BS><<<(unsigned)sym.nc, 128, smem, s>>>(sym.seg, sym.ta, sym.tb, sym.nc, A->nblk,
                                                         B->nblk, A->vals, B->vals, Cv, nz, err);
  return cuda_status(cudaGetLastError());
}

template <int BS>
bsm_status launch_batched(const ProdDesc *prods, const uint64_t *items, int64_t nitems,
                          unsigned long long *counter, unsigned *err, int ctas_per_sm,
                          cudaStream_t s) {
  size_t smem = (size_t)kStages * 2 * BS * BS * sizeof(double);
  static std::atomic<uint64_t> attr{0};
  BSM_TRY(once_per_device(attr, [&] {
    return cuda_status(cudaFuncSetAttribute(
        k_numeric_fp64_batched<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }));
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  BSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_numeric_fp64_batched<BS>, 128,
                                                         smem));
  if (occ < 1) occ = 1;
  if (ctas_per_sm <= 0 || ctas_per_sm > occ) ctas_per_sm = occ;
  int64_t grid = (int64_t)sms * ctas_per_sm;
  if (grid > nitems) grid = nitems;
  if (grid < 1) return BSM_OK;
  count_launch();
  k_numeric_fp64_batched<BS><<<(unsigned)grid, 128, smem, s>>>(prods, items, nitems, counter, err);
  return cuda_status(cudaGetLastError());
}

}  // namespace

bsm_status numeric_fp64(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, double *cvals,
                        int32_t *nzflag, unsigned *errword, cudaStream_t s) {
  if (sym.nc == 0) return BSM_OK;
  if (sym.nc > 0x7FFFFFFF) return BSM_ERR_UNSUPPORTED;
  switch (A->bs) {
    case 16: return launch<16>(sym, A, B, cvals, nzflag, errword, s);
    case 32: return launch<32>(sym, A, B, cvals, nzflag, errword, s);
    case 64: return launch<64>(sym, A, B, cvals, nzflag, errword, s);
  }
  return BSM_ERR_BLOCKSIZE;
}

bsm_status numeric_fp64_batched(int bs, const ProdDesc *prods, const uint64_t *items,
                                int64_t nitems, unsigned long long *counter, unsigned *errword,
                                int ctas_per_sm, cudaStream_t s) {
  if (nitems == 0) return BSM_OK;
  switch (bs) {
    case 16: return launch_batched<16>(prods, items, nitems, counter, errword, ctas_per_sm, s);
    case 32: return launch_batched<32>(prods, items, nitems, counter, errword, ctas_per_sm, s);
    case 64: return launch_batched<64>(prods, items, nitems, counter, errword, ctas_per_sm, s);
  }
  return BSM_ERR_BLOCKSIZE;
}
