// Split-precision numeric phase: FP64 block products on BF16 tensor cores.
//
// Each FP64 entry is written exactly as a sum of s BF16-representable digits
// (an error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59 (2012)), scaled per matrix row of A and per matrix
// column of B by a power of two:
//   A[r,k] = 2^E_r * sum_i a_i[r,k] 2^(-7(i+1)),   |a_0| <= 128, |a_i>0| <= 64
//   B[k,c] = 2^F_c * sum_j b_j[k,c] 2^(-7(j+1))   (up to 2^(-7s-1) truncation)
// with integer digits (base 2^7, balanced).  The product keeps the digit pairs
// on the diagonals d = i + j < s:
//   C[r,c] ~= 2^(E_r + F_c - 7(s+1)) * sum_d D_d[r,c] 2^(7(s-1-d)),
//   D_d = sum_k sum_{i+j=d} a_i[r,k] b_j[k,c].
// Every D_d is a sum of integer products, so it is exact in the FP32 tensor
// accumulator as long as it stays below 2^22 in magnitude (and below 2^24 for
// every partial sum); the k-products of a C block are therefore accumulated in
// groups ("flushes") of at most `flushk` leaf blocks, each flush moved out of
// TMEM into 32-bit integer registers.  After the last flush the diagonals are
// combined in 128-bit integer arithmetic and rounded once to FP64.  No FP64
// arithmetic is done per k-product: on GB300 the FP64 pipe is ~1 TFLOP/s,
// three orders of magnitude below the BF16 tensor rate.
//
// Tensor-core mapping (tcgen05.mma kind::f16, M = 128, N = bs, K = 16):
//   rows of the 128-row A operand = (lane block L, row r) with L = 0..128/bs-1,
//   lane block L of group g holding diagonal d = g*128/bs + L;
//   B operand = the B digit slices concatenated along K (K-block t = slice t);
//   A operand K-block t of lane block L = A slice d - t (zero if d < t).
// The slices of one A block sit contiguously in shared memory behind
// 128/bs - 1 zero slices, so the Toeplitz arrangement of the A operand is just
// a descriptor start address per K-block: lane block L reads slice
// (g*128/bs + L - t) because consecutive lane blocks are one slice apart.
// D_d then lands in TMEM lane block L of group g's accumulator.
//
// Roles (192 threads, one CTA per SM, persistent over C blocks):
//   warp 4 lane 0: producer -- 1-D bulk copies of the A and B slices of each
//                  k-product into a ring of stages (mbarrier complete_tx);
//   warp 5 lane 0: issues the MMAs of each k-product, commits the stage back
//                  to the producer and each finished flush to the epilogue;
//   warps 0-3:     epilogue -- drain TMEM (double-buffered) into integer
//                  accumulators, combine and round, store C, raise the
//                  nonzero flag.
#include <climits>

#include "bsm_ptx.cuh"

namespace {

constexpr int kBeta = 7;       // digit width in bits
constexpr int kMaxSlices = 8;  // 56-bit fixed point at most
constexpr uint32_t kMagic = 0x4B400000u;  // bits of 1.5 * 2^23
constexpr float kMagicF = 12582912.0f;

template <int BS>
struct Cfg {
  static constexpr int DPG = 128 / BS;                       // diagonals per group
  static constexpr int SLICE = BS * BS * 2;                  // bytes of one BF16 slice
  static constexpr int GMAX = (kMaxSlices + DPG - 1) / DPG;  // groups at most
  static constexpr int ASLOTS = (DPG - 1) + GMAX * DPG;      // zero pad + slices + pad
  static constexpr int BSLOTS = kMaxSlices;
  static constexpr int STAGE = (ASLOTS + BSLOTS) * SLICE;
  static constexpr int NST = BS == 32 ? 4 : 8;               // ring depth
  static constexpr int CROW = BS + 4;                        // padded int32 row (combine)
  static constexpr int COMB = kMaxSlices * BS * CROW * 4;    // combine buffer bytes
  static constexpr int SMEM = NST * STAGE + COMB + 1024;
  static constexpr uint32_t SBO = BS * 16;                   // 8-row group stride
  static constexpr uint32_t LBO = 128;                       // K core-matrix stride
};

// ------------------------------------------------------------ slicing
__device__ __forceinline__ int exp_bound(double x) {
  // smallest E with |x| < 2^E (x != 0); 1025 flags Inf/NaN
  uint64_t b = (uint64_t)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF);
  if ((b << 1) == 0) return INT_MIN;
  if (e == 0x7FF) return 1025;
  return e == 0 ? -1022 : e - 1022;
}

// Row exponents of A: one warp per block; lanes stride the columns.
__global__ void k_row_exp(const double *__restrict__ vals, const uint64_t *__restrict__ keys,
                          int64_t n, int bs, int *__restrict__ rowexp, unsigned *__restrict__ err) {
  int64_t t = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (t >= n) return;
  int64_t I = morton_compact(keys[t] >> 1);
  const double *b = vals + t * (int64_t)bs * bs;
  for (int r = 0; r < bs; r++) {
    int m = INT_MIN;
    for (int c = lane; c < bs; c += 32) m = max(m, exp_bound(b[r * bs + c]));
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0 && m != INT_MIN) {
      if (m == 1025) set_err(err, DERR_BOUNDS);
      atomicMax(rowexp + I * bs + r, m);
    }
  }
}

// Column exponents of B: one thread per (block, column).
__global__ void k_col_exp(const double *__restrict__ vals, const uint64_t *__restrict__ keys,
                          int64_t n, int bs, int *__restrict__ colexp, unsigned *__restrict__ err) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * bs) return;
  int64_t t = g / bs;
  int c = (int)(g % bs);
  int64_t J = morton_compact(keys[t]);
  const double *b = vals + t * (int64_t)bs * bs;
  int m = INT_MIN;
  for (int r = 0; r < bs; r++) m = max(m, exp_bound(b[r * bs + c]));
  if (m == 1025) set_err(err, DERR_BOUNDS);
  if (m != INT_MIN) atomicMax(colexp + J * bs + c, m);
}

// Balanced base-2^7 digits of round(x * 2^(7s - E)), most significant first.
__device__ __forceinline__ void digits(double x, int E, int s, int (&d)[kMaxSlices]) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF);
  uint64_t m = b & ((1ull << 52) - 1);
  if (e == 0)
    e = 1;
  else
    m |= 1ull << 52;
  int64_t X = 0;
  if (m != 0 && E != INT_MIN) {
    int sh = e - 1075 - E + kBeta * s;  // x = m 2^(e-1075), |x| < 2^E
    if (sh >= 0) {
      X = (int64_t)(m << sh);  // < 2^(7s) <= 2^56
    } else if (sh > -64) {
      uint64_t q = m >> (-sh);
      uint64_t half = (m >> (-sh - 1)) & 1ull;  // round half away from zero
      X = (int64_t)(q + half);
    }
    if (b >> 63) X = -X;
  }
  for (int i = s - 1; i >= 1; i--) {
    int64_t dig = ((X + (1 << (kBeta - 1))) & ((1 << kBeta) - 1)) - (1 << (kBeta - 1));
    d[i] = (int)dig;
    X = (X - dig) >> kBeta;
  }
  d[0] = (int)X;
}

__device__ __forceinline__ uint16_t small_int_to_bf16(int v) {
  // |v| <= 128: the float is exact (magic-number conversion, |v| < 2^22) and
  // has at most 8 significant bits, so its upper 16 bits are the BF16 value
  float f = __int_as_float((int)kMagic + v) - kMagicF;
  return (uint16_t)(__float_as_uint(f) >> 16);
}

// Writes the s slices of every block in the MMA operand layout (K-major,
// 8x8 BF16 core matrices of 128 bytes, K core matrices 128 B apart, 8-row
// groups BS*16 B apart).  TRANS = 0: A block, operand rows = block rows,
// K = block columns, row scales.  TRANS = 1: B block, operand rows = block
// columns, K = block rows, column scales.
template <int BS, int TRANS>
__global__ void k_slice(const double *__restrict__ vals, const uint64_t *__restrict__ keys,
                        int64_t n, const int *__restrict__ exps, int s,
                        uint16_t *__restrict__ out) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * BS * BS) return;
  int64_t t = g / (BS * BS);
  int e = (int)(g % (BS * BS));
  int r = e / BS, c = e % BS;  // block row, block column
  double x = vals[g];
  int mrow, kcol;
  int E;
  if (TRANS == 0) {
    mrow = r;
    kcol = c;
    E = exps[(int64_t)morton_compact(keys[t] >> 1) * BS + r];
  } else {
    mrow = c;
    kcol = r;
    E = exps[(int64_t)morton_compact(keys[t]) * BS + c];
  }
  int d[kMaxSlices];
  digits(x, E, s, d);
  uint32_t off = (mrow >> 3) * (BS * 16) + (kcol >> 3) * 128 + (mrow & 7) * 16 + (kcol & 7) * 2;
  uint16_t *base = out + t * (int64_t)s * BS * BS;
  for (int i = 0; i < s; i++) base[(int64_t)i * BS * BS + off / 2] = small_int_to_bf16(d[i]);
}

__global__ void k_max_seg(const int32_t *__restrict__ seg, int64_t nc, int *__restrict__ out) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int v = 0;
  if (c < nc) v = seg[c + 1] - seg[c];
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// ----------------------------------------------------- int128 -> FP64
// Correctly rounded (to nearest, ties to even) v * 2^X.
__device__ __forceinline__ double fixed_to_double(__int128 v, int X) {
  if (v == 0) return 0.0;
  bool neg = v < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
  int top = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  uint64_t mant;
  if (top <= 52) {
    mant = lo << (52 - top);
  } else {
    int sh = top - 52;
    unsigned __int128 q = u >> sh;
    mant = (uint64_t)q;
    unsigned __int128 rem = u - (q << sh);
    unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      mant++;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        top++;
      }
    }
  }
  int be = top + X + 1023;  // biased exponent of the result
  double r;
  if (be >= 1 && be <= 2046)
    r = __longlong_as_double((long long)(((uint64_t)be << 52) | (mant & ((1ull << 52) - 1))));
  else
    r = scalbn((double)mant, top - 52 + X);  // overflow / subnormal range
  return neg ? -r : r;
}

// -------------------------------------------------------- the MMA kernel
struct SplitArgs {
  const int32_t *seg, *ta, *tb;
  const uint64_t *ckeys;
  int64_t nc, na, nb;
  const uint16_t *asl, *bsl;
  const int *rowexp, *colexp;
  int s, flushk;
  double *cv;
  int32_t *nz;
  unsigned *err;
};

template <int BS, int G>
__global__ void __launch_bounds__(192, 1) k_numeric_split(SplitArgs P) {
  using C = Cfg<BS>;
  constexpr int DPG = C::DPG;
  constexpr uint32_t IDESC = idesc_bf16_f32(128, BS);
  constexpr int NCOLS = 2 * G * BS < 32 ? 32 : (2 * G * BS <= 64 ? 64 : (2 * G * BS <= 128 ? 128 : 256));
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[C::NST], empty[C::NST], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int warp_any[4];
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = P.s;
  uint8_t *stages = smem;
  int32_t *comb = reinterpret_cast<int32_t *>(smem + C::NST * C::STAGE);

  // zero the slice ring once: the pad slots stay zero (copies fill only the
  // s slice slots of each stage)
  for (int i = tid; i < C::NST * C::STAGE / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(stages)[i] = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (tid == 0) {
    for (int i = 0; i < C::NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (warp == 4) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      const uint32_t bytes = (uint32_t)s * C::SLICE;
      bool pend[C::NST] = {};
      uint32_t ppar[C::NST] = {};
      for (int64_t c = blockIdx.x; c < P.nc && !abort_flag; c += gridDim.x) {
        int32_t k0 = P.seg[c], nk = P.seg[c + 1] - k0;
        for (int j = 0; j < nk; j++, it++) {
          int st = it % C::NST;
          if (!mbar_wait(&empty[st], ((it / C::NST) & 1u) ^ 1u)) {
            set_err(P.err, DERR_TIMEOUT);
            abort_flag = 1;
            break;
          }
          int32_t a = P.ta[k0 + j], b = P.tb[k0 + j];
          uint8_t *sa = stages + (size_t)st * C::STAGE;
          uint8_t *sb = sa + C::ASLOTS * C::SLICE;
          pend[st] = true;
          ppar[st] = (it / C::NST) & 1u;
          if (a < 0 || a >= P.na || b < 0 || b >= P.nb) {
            set_err(P.err, DERR_BOUNDS);  // complete the stage without data
            mbar_arrive(&full[st]);
            continue;
          }
          mbar_expect_tx(&full[st], 2 * bytes);
          bulk_g2s(sa + (DPG - 1) * C::SLICE, P.asl + (int64_t)a * s * BS * BS, bytes, &full[st]);
          bulk_g2s(sb, P.bsl + (int64_t)b * s * BS * BS, bytes, &full[st]);
        }
      }
      // copies still in flight must land before the CTA exits
      for (int st = 0; st < C::NST; st++)
        if (pend[st]) mbar_wait(&full[st], ppar[st]);
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, fc = 0;
      const uint32_t sbase = smem_u32(stages);
      for (int64_t c = blockIdx.x; c < P.nc && !abort_flag; c += gridDim.x) {
        int32_t k0 = P.seg[c], nk = P.seg[c + 1] - k0;
        int nfl = (nk + P.flushk - 1) / P.flushk;
        for (int f = 0; f < nfl && !abort_flag; f++, fc++) {
          int b = fc & 1;
          if (!mbar_wait(&tempty[b], ((fc >> 1) & 1u) ^ 1u)) {
            set_err(P.err, DERR_TIMEOUT);
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          int jend = min(nk, (f + 1) * P.flushk);
          for (int j = f * P.flushk; j < jend; j++, it++) {
            int st = it % C::NST;
            if (!mbar_wait(&full[st], (it / C::NST) & 1u)) {
              set_err(P.err, DERR_TIMEOUT);
              abort_flag = 1;
              break;
            }
            tc_fence_after();
            uint32_t sa = sbase + st * C::STAGE;
            uint32_t sb = sa + C::ASLOTS * C::SLICE;
#pragma unroll
            for (int g = 0; g < G; g++) {
              uint32_t dt = tbase + (uint32_t)((b * G + g) * BS);
              int nt = min(s, (g + 1) * DPG);  // K-blocks: slices t = 0 .. nt-1
              for (int t = 0; t < nt; t++)
#pragma unroll
                for (int h = 0; h < BS / 16; h++) {
                  uint32_t aaddr = sa + (uint32_t)((DPG - 1 + g * DPG - t) * C::SLICE + h * 256);
                  uint32_t baddr = sb + (uint32_t)(t * C::SLICE + h * 256);
                  uint32_t acc = (j > f * P.flushk || t > 0 || h > 0) ? 1u : 0u;
                  tc_mma_bf16(dt, smem_desc(aaddr, C::LBO, C::SBO), smem_desc(baddr, C::LBO, C::SBO),
                              IDESC, acc);
                }
            }
            tc_commit(&empty[st]);  // stage reusable once these MMAs are done
          }
          tc_commit(&tfull[b]);  // flush ready for the epilogue
        }
      }
      // no MMA may still be running when TMEM is released
      tc_commit(&done);
      if (!mbar_wait(&done, 0)) set_err(P.err, DERR_TIMEOUT);
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int row = warp * 32 + lane;  // TMEM lane = operand row
    const int L = row / BS, r = row % BS;
    const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
    uint32_t fc = 0;
    for (int64_t c = blockIdx.x; c < P.nc; c += gridDim.x) {
      int32_t k0 = P.seg[c], nk = P.seg[c + 1] - k0;
      int nfl = (nk + P.flushk - 1) / P.flushk;
      uint32_t acc[G][BS];
#pragma unroll
      for (int g = 0; g < G; g++)
#pragma unroll
        for (int q = 0; q < BS; q++) acc[g][q] = 0;
      // every decision below is uniform across the warp (tcgen05.ld is
      // .sync.aligned) and, at the barriers, across the 128 epilogue threads
      bool ok = __all_sync(0xffffffffu, abort_flag == 0);
      for (int f = 0; f < nfl && ok; f++, fc++) {
        int b = fc & 1;
        bool w = mbar_wait(&tfull[b], (fc >> 1) & 1u);
        if (!__all_sync(0xffffffffu, w)) {
          set_err(P.err, DERR_TIMEOUT);
          abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < G; g++) {
          uint32_t v[BS];
          if constexpr (BS == 32)
            tmem_ld32(tbase + lane_addr + (uint32_t)((b * G + g) * BS), v);
          else
            tmem_ld16(tbase + lane_addr + (uint32_t)((b * G + g) * BS), v);
          tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < BS; q++) acc[g][q] += __float_as_uint(__uint_as_float(v[q]) + kMagicF);
        }
        tc_fence_before();
        mbar_arrive(&tempty[b]);
      }
      // all 128 epilogue threads agree on whether to continue
      if (named_bar_or(1, 128, !ok || abort_flag != 0)) break;
      // diagonals -> shared memory, [d][r][c] with padded rows
#pragma unroll
      for (int g = 0; g < G; g++) {
        int d = g * DPG + L;
        if (d < s) {
          int32_t *dst = comb + (d * BS + r) * C::CROW;
#pragma unroll
          for (int q = 0; q < BS; q += 4)
            *reinterpret_cast<int4 *>(dst + q) =
                make_int4((int32_t)(acc[g][q] - (uint32_t)nfl * kMagic),
                          (int32_t)(acc[g][q + 1] - (uint32_t)nfl * kMagic),
                          (int32_t)(acc[g][q + 2] - (uint32_t)nfl * kMagic),
                          (int32_t)(acc[g][q + 3] - (uint32_t)nfl * kMagic));
        }
      }
      named_bar(1, 128);
      uint64_t key = P.ckeys[c];
      int64_t I = morton_compact(key >> 1), J = morton_compact(key);
      double *cb = P.cv + c * (int64_t)BS * BS;
      bool any = false;
      for (int e = tid; e < BS * BS; e += 128) {
        int rr = e / BS, cc = e % BS;
        __int128 V = 0;
        for (int d = 0; d < s; d++)
          V += (__int128)comb[(d * BS + rr) * C::CROW + cc] << (kBeta * (s - 1 - d));
        double out = 0.0;
        if (V != 0) {
          int X = P.rowexp[I * BS + rr] + P.colexp[J * BS + cc] - kBeta * (s + 1);
          out = fixed_to_double(V, X);
          any = true;
        }
        cb[e] = out;
      }
      any = __any_sync(0xffffffffu, any);
      if (lane == 0) warp_any[warp] = any;
      named_bar(1, 128);
      if (tid == 0) P.nz[c] = warp_any[0] | warp_any[1] | warp_any[2] | warp_any[3];
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, NCOLS);
  }
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int BS, int G>
bsm_status launch_split(const SplitArgs &a, cudaStream_t s) {
  using C = Cfg<BS>;
  static bool attr = false;
  if (!attr) {
    BSM_CUDA(cudaFuncSetAttribute(k_numeric_split<BS, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM));
    attr = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = a.nc < sms ? a.nc : sms;
  count_launch();
  k_numeric_split<BS, G><<<(unsigned)grid, 192, C::SMEM, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace

// Largest group of k-products whose diagonal sums stay exact (< 2^22) in the
// FP32 accumulator: d = 0 sums terms up to 2^14; d >= 1 at most (d + 3) 2^12
// per inner element.
static int flush_group(int bs, int s) {
  int maxel = (1 << 22) >> (2 * kBeta);                  // d = 0
  int m2 = ((1 << 22) >> (2 * kBeta - 2)) / (s + 2);     // d = s - 1
  if (m2 < maxel) maxel = m2;
  int g = maxel / bs;
  return g < 1 ? 1 : g;
}

bsm_status numeric_split(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, int slices,
                         double *cvals, int32_t *nzflag, unsigned *errword, cudaStream_t s) {
  int bs = A->bs;
  if (bs != 16 && bs != 32) return BSM_ERR_UNSUPPORTED;
  if (slices < 1 || slices > kMaxSlices) return BSM_ERR_INVALID_ARG;
  if (sym.nc == 0) return BSM_OK;
  int flushk = flush_group(bs, slices);
  // the 32-bit diagonal accumulators hold at most 511 flushes of < 2^22
  int *dmax = nullptr, *rowexp = nullptr, *colexp = nullptr;
  uint16_t *asl = nullptr, *bsl = nullptr;
  bsm_status st = BSM_OK;
  auto cleanup = [&]() {
    dev_free(dmax, s);
    dev_free(rowexp, s);
    dev_free(colexp, s);
    dev_free(asl, s);
    dev_free(bsl, s);
  };
  if ((st = dev_alloc((void **)&dmax, 4, s)) ||
      (st = dev_alloc((void **)&rowexp, 4 * A->mb * bs, s)) ||
      (st = dev_alloc((void **)&colexp, 4 * B->nb * bs, s)) ||
      (st = dev_alloc((void **)&asl, (size_t)2 * slices * bs * bs * A->nblk, s)) ||
      (st = dev_alloc((void **)&bsl, (size_t)2 * slices * bs * bs * B->nblk, s))) {
    cleanup();
    return st;
  }
  cudaMemsetAsync(dmax, 0, 4, s);
  cudaMemsetAsync(rowexp, 0x80, 4 * A->mb * bs, s);  // 0x80808080: below any exponent
  cudaMemsetAsync(colexp, 0x80, 4 * B->nb * bs, s);
  count_launch(5);
  k_max_seg<<<grid_for(sym.nc, 256), 256, 0, s>>>(sym.seg, sym.nc, dmax);
  k_row_exp<<<grid_for(A->nblk, 8), 256, 0, s>>>(A->vals, A->keys, A->nblk, bs, rowexp, errword);
  k_col_exp<<<grid_for(B->nblk * bs, 256), 256, 0, s>>>(B->vals, B->keys, B->nblk, bs, colexp,
                                                       errword);
  if (bs == 16) {
    k_slice<16, 0><<<grid_for(A->nblk * 256, 256), 256, 0, s>>>(A->vals, A->keys, A->nblk, rowexp,
                                                                slices, asl);
    k_slice<16, 1><<<grid_for(B->nblk * 256, 256), 256, 0, s>>>(B->vals, B->keys, B->nblk, colexp,
                                                                slices, bsl);
  } else {
    k_slice<32, 0><<<grid_for(A->nblk * 1024, 256), 256, 0, s>>>(A->vals, A->keys, A->nblk,
                                                                 rowexp, slices, asl);
    k_slice<32, 1><<<grid_for(B->nblk * 1024, 256), 256, 0, s>>>(B->vals, B->keys, B->nblk,
                                                                 colexp, slices, bsl);
  }
  int *h = (int *)host_scratch().get(16);
  if (!h) {
    cleanup();
    return BSM_ERR_OOM;
  }
  cudaMemcpyAsync(h, dmax, 4, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_status(e);
  }
  int nflmax = (h[0] + flushk - 1) / flushk;
  if (nflmax > 511) {
    cleanup();
    return BSM_ERR_UNSUPPORTED;  // a C block with too many products for 32-bit diagonals
  }
  SplitArgs a;
  a.seg = sym.seg;
  a.ta = sym.ta;
  a.tb = sym.tb;
  a.ckeys = sym.ckeys;
  a.nc = sym.nc;
  a.na = A->nblk;
  a.nb = B->nblk;
  a.asl = asl;
  a.bsl = bsl;
  a.rowexp = rowexp;
  a.colexp = colexp;
  a.s = slices;
  a.flushk = flushk;
  a.cv = cvals;
  a.nz = nzflag;
  a.err = errword;
  if (bs == 16)
    st = launch_split<16, 1>(a, s);
  else if (slices <= 4)
    st = launch_split<32, 1>(a, s);
  else
    st = launch_split<32, 2>(a, s);
  cleanup();  // stream-ordered: freed after the kernel
  return st;
}
