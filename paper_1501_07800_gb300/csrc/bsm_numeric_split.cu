// Split-precision numeric phase: FP64 block products on BF16 or FP8 (E4M3)
// tensor cores.  Written below for the BF16 form (digit base 2^7); the E4M3
// form is the same with base 2^4 (|a_0| <= 16, |a_i>0| <= 8), kind::f8f6f4
// MMAs with K = 32 per instruction, and 32-wide blocks only.
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
// TMEM into 32-bit integer sums (folded into 64-bit pairs every 511 flushes
// for very long product lists).  After the last flush the diagonals are
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
// Items: one C block, or (long product lists) a pair of sibling C blocks
// (I, 2y), (I, 2y+1) whose merged product list runs as 128 x 2bs MMAs: the B
// slices of the two sibling B blocks sit side by side (a pair slot), so each
// A tile feeds both C blocks; at bs 16 up to four consecutive C blocks of
// short lists (grouped items), each list into accumulator columns of its own.
//
// Roles (640 threads, or 576 with one team; one CTA per SM, persistent): two
// independent pipelines (one with a single team), each
//   a producer warp (16, 17) -- all lanes prefetch work descriptors and block
//                  indices; lane 0 issues the 1-D bulk copies of the A and B
//                  slices of each k-product into the pipeline's stages
//                  (mbarrier complete_tx) and hands per-item descriptors to
//                  the other roles through the pipeline's descriptor ring;
//   an MMA warp (18, 19), lane 0: issues the MMAs of each k-product, commits
//                  the stage back to the producer and each finished flush to
//                  the epilogue;
//   an epilogue team of eight warps (0-7, 8-15) with its own TMEM
//                  accumulator buffers -- drain TMEM (two warps per lane
//                  quadrant) into exact integer diagonal sums in shared
//                  memory, combine and round, store C, mark the nonzero C
//                  blocks.
#include <climits>
#include <cstddef>
#include <cstring>
#include <vector>

#include <cuda_fp8.h>

#include "bsm_batch.cuh"
#include "bsm_ptx.cuh"
#include "bsm_split_round.cuh"

namespace {

// Digit formats.  F = 0: BF16 operands, base-2^7 digits (|a_0| <= 128, the
// others <= 64, exact in BF16's 8-bit significand), MMA kind::f16, K = 16 per
// instruction.  F = 1: FP8 E4M3 operands, base-2^4 digits (|a_0| <= 16, the
// others <= 8, exact in E4M3), MMA kind::f8f6f4, K = 32 per instruction.
// TSPLIT: the combination keeps the digit terms with shift < TSPLIT in `lo`
// and the rest in `hi` (value = hi 2^TSPLIT + lo), chosen so that neither
// part can overflow 64 bits.
template <int F>
struct Fmt;
template <>
struct Fmt<0> {
  static constexpr int BETA = 7, EB = 2, KPI = 16, TSPLIT = 35, MAXS = 8;
};
template <>
struct Fmt<1> {
  static constexpr int BETA = 4, EB = 1, KPI = 32, TSPLIT = 32, MAXS = 12;
};
constexpr uint32_t kMagic = 0x4B400000u;  // bits of 1.5 * 2^23
constexpr float kMagicF = 12582912.0f;

// NP: C blocks per work item.  1: one C block (N = bs per MMA), two epilogue
// teams.  2: a pair of sibling C blocks (I, 2y), (I, 2y+1) sharing every A
// tile (N = 2 bs per MMA, half the A-operand traffic per output), one team.
// NQ (with NP = 1): up to NQ C blocks of short product lists per work item,
// each list multiplied into its own TMEM columns, drained and combined in one
// epilogue pass (grouped items: the per-item work of every role shared by NQ
// C blocks of 16 x 16).
template <int BS, int S, int F, int NP = 1, int NQ = 1>
struct Cfg {
  static constexpr int DPG = 128 / BS;                       // diagonals per group
  static constexpr int G = (S + DPG - 1) / DPG;              // diagonal groups
  static constexpr int SLICE = BS * BS * Fmt<F>::EB;         // bytes of one slice
  static constexpr int ASLOTS = (DPG - 1) + G * DPG;         // zero pad + slices + pad
  static constexpr int BSLOTS = NP * S;                      // B slices (a pair interleaved)
  static constexpr int STAGE = (ASLOTS + BSLOTS) * SLICE;
  static constexpr int NW = NP * BS * NQ;                    // output columns of an item
  static constexpr int CROW = NW + 4;                        // padded int32 row (combine)
  static constexpr int COMB = S * BS * CROW * 4;             // combine buffer bytes (per team)
  // ring depth: up to 4 (bs 32) / 8 (bs 16) stages within 227 KiB of shared
  // memory, 8 KiB of it left for the static barriers and descriptor rings (16
  // stages at bs 16 measured slower than 8), split evenly between the
  // pipelines
  static constexpr int NSTMAX = BS == 32 ? (F ? 6 : 4) : 8;
  static constexpr int stages_for(int teams) {
    return (227 * 1024 - 8 * 1024 - teams * COMB) / STAGE < NSTMAX
               ? (227 * 1024 - 8 * 1024 - teams * COMB) / STAGE
               : NSTMAX;
  }
  // epilogue teams = pipelines: one for pairs (a team of sixteen warps), and
  // where two would leave a pipeline fewer than two stages (BF16 x 8 at bs 32)
  static constexpr int NTEAM = (NP == 2 || stages_for(2) < 4) ? 1 : 2;
  static constexpr int NST = stages_for(NTEAM) / NTEAM * NTEAM;
  static constexpr int SMEM = NST * STAGE + NTEAM * COMB;
  static_assert(NST >= 2 * NTEAM, "shared memory too small for two stages per pipeline");
  static constexpr uint32_t SBO = BS * 8 * Fmt<F>::EB;       // 8-row group stride
  static constexpr uint32_t LBO = 128;                       // K core-matrix stride
};

// Order of the B slices in the operand.  Slice j = t + DPG k (t < DPG) sits
// at position b_off(t) + k: the slices sharing a residue t are adjacent, so
// one MMA with the Toeplitz A tile of group g and offset t (rows L carry
// a_(g DPG + L - t)) multiplies it by [b_t | b_(t+DPG) | ...] at once and adds
// into the accumulators of groups g, g+1, ... (column block k lands in group
// g + k, whose diagonal g DPG + k DPG + L is exactly (g DPG + L - t) + (t + k
// DPG)).  b_count(t): slices with residue t.
__host__ __device__ constexpr int b_count(int S, int DPG, int t) {
  return t < S ? (S - t + DPG - 1) / DPG : 0;
}
__host__ __device__ constexpr int b_off(int S, int DPG, int t) {
  int o = 0;
  for (int u = 0; u < t; u++) o += b_count(S, DPG, u);
  return o;
}
__host__ __device__ constexpr int b_pos(int S, int DPG, int j) {
  return b_off(S, DPG, j % DPG) + j / DPG;
}

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

// Balanced base-2^B digits of round(x * 2^(B S - E)), most significant first.
template <int S, int B>
__device__ __forceinline__ void digits(double x, int E, int (&d)[S]) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF);
  uint64_t m = b & ((1ull << 52) - 1);
  if (e == 0)
    e = 1;
  else
    m |= 1ull << 52;
  int64_t X = 0;
  if (m != 0) {
    int sh = e - 1075 - E + B * S;  // x = m 2^(e-1075), |x| < 2^E
    if (sh >= 0) {
      X = (int64_t)(m << sh);  // < 2^(B S) <= 2^56
    } else if (sh > -64) {
      uint64_t q = m >> (-sh);
      uint64_t half = (m >> (-sh - 1)) & 1ull;  // round half away from zero
      X = (int64_t)(q + half);
    }
    if (b >> 63) X = -X;
  }
#pragma unroll
  for (int i = S - 1; i >= 1; i--) {
    int64_t dig = ((X + (1 << (B - 1))) & ((1 << B) - 1)) - (1 << (B - 1));
    d[i] = (int)dig;
    X = (X - dig) >> B;
  }
  d[0] = (int)X;
}

__device__ __forceinline__ uint32_t small_int_to_bf16(int v) {
  // |v| <= 128: the float is exact (magic-number conversion, |v| < 2^22) and
  // has at most 8 significant bits, so its upper 16 bits are the BF16 value
  float f = __int_as_float((int)kMagic + v) - kMagicF;
  return __float_as_uint(f) >> 16;
}

__device__ __forceinline__ uint32_t small_int_to_e4m3(int v) {
  // |v| <= 16 has at most 4 significant bits and an exponent within E4M3's
  // range: the conversion is exact
  return (uint32_t)__nv_cvt_float_to_fp8((float)v, __NV_SATFINITE, __NV_E4M3);
}

// Writes the S slices of every block in the MMA operand layout (K-major
// core matrices of 8 rows x 16 bytes -- 8 BF16 or 16 E4M3 elements -- K core
// matrices 128 B apart, 8-row groups SBO apart).  TRANS = 0: A block, operand
// rows = block rows, K = block columns, row scales.  TRANS = 1: B block,
// operand rows = block columns, K = block rows, column scales.  A CTA stages
// BPI blocks in shared memory at a time (as many as its 128 threads have
// core-matrix rows to make: one at bs 32 BF16, four at bs 16); each thread
// makes one core-matrix row (16 bytes per slice), so a warp writes 512
// contiguous bytes per slice.
// B slices are stored in the operand order of b_pos.  pslot (B only, NULL
// otherwise): the pair slot of each block; the slices of the two sibling
// blocks (I, 2y), (I, 2y+1) of a slot are then interleaved, position p of the
// even sibling at 2p, of the odd one at 2p+1.
template <int BS, int S, int TRANS, int F>
__global__ void __launch_bounds__(128) k_slice(const double *__restrict__ vals,
                                               const uint64_t *__restrict__ keys, int64_t n,
                                               const int *__restrict__ exps,
                                               const int32_t *__restrict__ pslot,
                                               uint8_t *__restrict__ out) {
  using C = Cfg<BS, S, F>;
  constexpr int B = Fmt<F>::BETA;
  constexpr int EPR = 16 / Fmt<F>::EB;  // elements per core-matrix row
  constexpr int KG = BS / EPR;
  constexpr int TASKS = BS * KG;                       // core-matrix rows per block
  constexpr int BPI = TASKS >= 128 ? 1 : 128 / TASKS;  // blocks per iteration
  __shared__ double stage[BPI][BS * (BS + 1)];
  for (int64_t t0 = (int64_t)blockIdx.x * BPI; t0 < n; t0 += (int64_t)gridDim.x * BPI) {
    for (int e = threadIdx.x; e < BPI * BS * BS; e += blockDim.x) {
      const int u = e / (BS * BS), f = e % (BS * BS);
      if (t0 + u < n) stage[u][(f / BS) * (BS + 1) + f % BS] = vals[(t0 + u) * BS * BS + f];
    }
    __syncthreads();
    const int u = BPI > 1 ? (int)threadIdx.x / TASKS : 0;  // this thread's block
    const int64_t t = t0 + u;
    const double *blk = stage[u];
    const uint64_t key = t < n ? keys[t] : 0;
    const int64_t rc = TRANS == 0 ? (int64_t)morton_compact(key >> 1) : (int64_t)morton_compact(key);
    for (int task = BPI > 1 ? (int)threadIdx.x % TASKS : (int)threadIdx.x;
         t < n && task < TASKS; task += BPI > 1 ? TASKS : (int)blockDim.x) {
      const int kg = task % KG, mrow = task / KG;
      const int E = exps[rc * BS + mrow];
      uint32_t w[S][4] = {};
#pragma unroll
      for (int x = 0; x < EPR; x++) {
        const int k = kg * EPR + x;
        const double v = TRANS == 0 ? blk[mrow * (BS + 1) + k] : blk[k * (BS + 1) + mrow];
        int dg[S];
        digits<S, B>(v, E, dg);
#pragma unroll
        for (int i = 0; i < S; i++) {
          if (F == 0)
            w[i][x / 2] |= small_int_to_bf16(dg[i]) << (16 * (x & 1));
          else
            w[i][x / 4] |= small_int_to_e4m3(dg[i]) << (8 * (x & 3));
        }
      }
      const uint32_t off = (mrow >> 3) * C::SBO + kg * 128 + (mrow & 7) * 16;  // bytes
      uint8_t *base = pslot ? out + ((int64_t)pslot[t] * 2 * S + (key & 1)) * C::SLICE
                            : out + t * (int64_t)S * C::SLICE;
      const int64_t step = pslot ? 2 * C::SLICE : C::SLICE;
#pragma unroll
      for (int i = 0; i < S; i++) {
        const int pos = TRANS == 0 ? i : b_pos(S, C::DPG, i);  // B: operand order
        *reinterpret_cast<uint4 *>(base + pos * step + off) =
            make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
      }
    }
    __syncthreads();
  }
}

template <int BS, int S, int F>
void launch_slices(bsm_matrix A, bsm_matrix B, const int *rowexp, const int *colexp,
                   uint8_t *asl, uint8_t *bsl, const int32_t *bslot, cudaStream_t s) {
  // (blocks per CTA iteration: 128 / core-matrix rows per block, at least 1)
  constexpr int BPI = BS * (BS / (16 / Fmt<F>::EB)) >= 128 ? 1 : 128 / (BS * (BS / (16 / Fmt<F>::EB)));
  auto grid = [](int64_t n) {
    const int64_t c = (n + BPI - 1) / BPI;
    return (unsigned)(c < 152 * 16 ? c : 152 * 16);
  };
  count_launch(2);
  if (A->nblk)
    k_slice<BS, S, 0, F><<<grid(A->nblk), 128, 0, s>>>(A->vals, A->keys, A->nblk, rowexp,
                                                        nullptr, asl);
  if (B->nblk)
    k_slice<BS, S, 1, F><<<grid(B->nblk), 128, 0, s>>>(B->vals, B->keys, B->nblk, colexp,
                                                        bslot, bsl);
}

// Slice counts with a compiled pair kernel: BF16 3..8 (16- and 32-wide
// blocks), E4M3 4, 6, 8, 12 (32-wide).
inline bool pair_compiled(int bs, int fmt, int slices) {
  if (fmt == 0) return (bs == 16 || bs == 32) && slices >= 3 && slices <= 8;
  return bs == 32 && (slices == 4 || slices == 6 || slices == 8 || slices == 12);
}

inline bool group_compiled(int bs, int fmt, int slices) {
  return bs == 16 && fmt == 0 && slices >= 3 && slices <= 8;
}

// Slice counts with a compiled kernel: 1..8 for BF16, {2,3,4,6,8,12} for E4M3.
inline bool spec_compiled(int fmt, int slices) {
  if (fmt == 0) return slices >= 1 && slices <= 8;
  return slices == 2 || slices == 3 || slices == 4 || slices == 6 || slices == 8 || slices == 12;
}

template <int BS>
void launch_slices_s(bsm_matrix A, bsm_matrix B, const int *rowexp, const int *colexp,
                     uint8_t *asl, uint8_t *bsl, const int32_t *bslot, int fmt, int slices,
                     cudaStream_t s) {
#define BSM_SL(F, S)                                                    \
  if (fmt == F && slices == S) {                                        \
    launch_slices<BS, S, F>(A, B, rowexp, colexp, asl, bsl, bslot, s); \
    return;                                                             \
  }
  BSM_SL(0, 1) BSM_SL(0, 2) BSM_SL(0, 3) BSM_SL(0, 4) BSM_SL(0, 5) BSM_SL(0, 6) BSM_SL(0, 7)
  BSM_SL(0, 8)
  if constexpr (BS == 32) {  // E4M3 needs K = 32 per instruction: one 32-wide block
    BSM_SL(1, 2) BSM_SL(1, 3) BSM_SL(1, 4) BSM_SL(1, 6) BSM_SL(1, 8) BSM_SL(1, 12)
  }
#undef BSM_SL
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
  const ProdDesc *prods;     // product table (device)
  const uint64_t *items;     // work list of (product, C block); NULL: product 0, C blocks 0..
  int64_t nitems;
  int flushk;                // block products per flush: sums < 2^22 (magic conversion)
  int flushk_wide;           // the same for sums <= 2^24 (bitwise conversion), long lists
  unsigned *err;
  unsigned long long *work;  // chunk counter, zero at launch
  int chunk;                 // work items claimed per atomic (1..32)
  int64_t *fold;             // [grid][2 teams][BS*BS][hi, lo]: folded diagonal sums
};
constexpr int kChunk = 32;   // most work items claimed per atomic
// The 32-bit diagonal sums in shared memory take at most kFold flushes of
// magnitude < 2^22 each (kFoldWide of <= 2^24); a C block with more flushes
// folds them every kFold flushes into exact 64-bit (hi, lo) pairs in per-CTA
// global scratch.
constexpr int kFold = 511, kFoldWide = 127;

// Flush mode of a C block with nk block products: a list longer than one
// narrow flush uses wide flushes (4x longer, converted bit by bit).
struct FlushPlan {
  bool wide;
  int fk, nfl, kf;
};
__device__ __forceinline__ FlushPlan flush_plan(int nk, int flushk, int flushk_wide) {
  FlushPlan p;
  p.wide = nk > flushk;
  p.fk = p.wide ? flushk_wide : flushk;
  p.nfl = (nk + p.fk - 1) / p.fk;
  p.kf = p.wide ? kFoldWide : kFold;
  return p;
}

// Exact value of an integer-valued FP32 with |v| <= 2^24, from its bits.
__device__ __forceinline__ int32_t f32_int_exact(uint32_t b) {
  const int e = (int)((b >> 23) & 0xFFu);
  const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
  const int32_t mag = e < 127 ? 0 : (e > 150 ? (int32_t)(m << (e - 150)) : (int32_t)(m >> (150 - e)));
  return (b >> 31) ? -mag : mag;
}

// Per-item work descriptor handed from the producer warp to the MMA threads
// and the epilogue through a shared-memory ring.
constexpr int kSub = 4;  // most C blocks of a work item
struct __align__(16) Meta {
  int64_t c[kSub];      // C block index within its product of each of the item's
                        // C blocks (pairs: even, odd sibling), -1: absent
  double *cv;           // the product's C blocks
  int32_t *nz;          // the product's nonzero flags
  const int *rowexp;    // the product's row / column scale exponents
  const int *colexp;
  int32_t bi[kSub], bj[kSub];  // block row and block column of each C block
  int32_t nkq[kSub];    // grouped items: block products of each C block
  int32_t nk;           // block products of the item (all its lists)
  int32_t nq;           // grouped items: lists multiplied one after another; else 1
  int32_t nfl;          // the item's flushes (flush plan, made once by the producer)
  int16_t fk;           // block products per flush
  int8_t wide, pad;     // wide flushes (partial sums up to 2^24)
};
static_assert(sizeof(Meta) % 16 == 0, "Meta alignment");
constexpr int kMeta = 8;

// sum_d acc_d 2^(B(S-1-d)) for 32-bit acc_d, returned as hi * 2^T + lo: the
// terms with shift < T are summed in lo (< 2^59.1), the rest in hi.
template <int S, int B, int T>
__device__ __forceinline__ void combine_digits(const int32_t (&a)[S], int64_t &hi, int64_t &lo) {
  lo = 0;
  hi = 0;
#pragma unroll
  for (int d = 0; d < S; d++) {
    const int sh = B * (S - 1 - d);
    if (sh < T)
      lo += (int64_t)a[d] << sh;
    else
      hi += (int64_t)a[d] << (sh - T);
  }
}

// Correctly rounded (hi 2^T + lo) 2^X as FP64; 64-bit path when the value
// fits in an int64, 128-bit path otherwise.  The 64-bit path rounds to nearest
// even by adding 2^(sh-1) - 1 plus the kept part's lowest bit before the
// shift, and adds the 53-bit significand (hidden bit included) to the
// exponent field minus one, so that a rounding carry to 2^53 raises the
// exponent by itself.
// The general case (values beyond 64 bits, results in the subnormal or
// overflow range): rare, and kept out of line so that none of its FP64
// instructions is issued, predicated off, on the common path.
__device__ __noinline__ double split_to_double_slow(int64_t hi, int64_t lo, int T, int X) {
  return fixed_to_double(((__int128)hi << T) + (__int128)lo, X);
}

template <int T>
__device__ __forceinline__ double split_to_double(int64_t hi, int64_t lo, int X) {
  if (__builtin_expect(hi > -(1ll << 27) && hi < (1ll << 27), 1)) {
    const int64_t v = (int64_t)((uint64_t)hi << T) + lo;  // |v| < 2^(27+T) + 2^59.1
    if (v == 0) return 0.0;
    const uint64_t sign = (uint64_t)v & (1ull << 63);
    const uint64_t u = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
    const int top = 63 - __clzll((long long)u);
    uint64_t q;
    if (top <= 52) {
      q = u << (52 - top);
    } else {
      const int sh = top - 52;
      q = (u + ((1ull << (sh - 1)) - 1) + ((u >> sh) & 1ull)) >> sh;
    }
    const int be = top + X + 1023;
    if (__builtin_expect(be >= 1 && be <= 2045, 1))
      return __longlong_as_double((long long)(sign | (((uint64_t)(be - 1) << 52) + q)));
  }
  return split_to_double_slow(hi, lo, T, X);
}

constexpr int kEpiWarps = 16;                // epilogue warps (4 per lane quadrant)
// Each epilogue team is the end of a pipeline of its own: a producer warp
// (work claims, descriptors, stage copies), an MMA-issuing thread in a warp
// of its own, and the team.  A thread issues tcgen05.mma instructions no
// faster than one per ~50 cycles (measured), so a second issuer doubles the
// rate at which the short instructions of this kernel (N = 32 or 64) reach
// the tensor core; a second producer halves the per-item work of the warp
// that otherwise paces the kernel on short product lists (one producer warp
// shares its scheduler with four busy epilogue warps).
constexpr int kMaxThreads = (kEpiWarps + 4) * 32;
template <int NTEAM>
constexpr int threads_for() {
  return (kEpiWarps + 2 * NTEAM) * 32;
}

template <int BS, int S, int F, int NP, int NQ>
__global__ void __launch_bounds__(kMaxThreads, 1) k_numeric_split(SplitArgs P) {
  using C = Cfg<BS, S, F, NP, NQ>;
  constexpr int DPG = C::DPG;
  constexpr int G = C::G;
  constexpr int NTEAM = C::NTEAM;
  constexpr int kTeamWarps = kEpiWarps / NTEAM;  // 8 (two teams) or 16 (one)
  constexpr int kTeam = kTeamWarps * 32;         // threads per epilogue team
  constexpr int NB = NP * BS;                    // MMA N: output columns of one list
  constexpr int NSUB = NP * NQ;                  // C blocks of an item
  static_assert(NSUB <= kSub && (NP == 1 || NQ == 1), "item shape");
  constexpr int BETA = Fmt<F>::BETA, TS = Fmt<F>::TSPLIT;
  // one narrow flush of at most kFast block products: the diagonal sums' FP32
  // bit patterns go to shared memory as they are and are combined in wrapping
  // 64-bit arithmetic (the digit bounds keep the combined integer below 2^63)
  constexpr int kFast = narrow_int64_products<S, BETA, BS>();
  // instruction descriptors for N = NB, 2 NB, 3 NB (one to three diagonal groups)
  constexpr uint32_t IDESC1 = F == 0 ? idesc_bf16_f32(128, NB) : idesc_e4m3_f32(128, NB);
  constexpr uint32_t IDESC2 = F == 0 ? idesc_bf16_f32(128, 2 * NB) : idesc_e4m3_f32(128, 2 * NB);
  constexpr uint32_t IDESC3 = F == 0 ? idesc_bf16_f32(128, 3 * NB) : idesc_e4m3_f32(128, 3 * NB);
  static_assert(G <= 3 && G * NB <= 256, "one MMA spans at most three groups, N <= 256");
  // TMEM accumulators: each team owns NBUF buffers of NQ*G*NB columns (list
  // q's group g at (q G + g) NB), two when they fit in the 256 columns we
  // allocate, so that the MMAs of an item's next flush run while the team
  // drains the previous one
  constexpr int NBUF = NTEAM * 2 * NQ * G * NB <= 256 ? 2 : 1;
  constexpr int TCOLS = NTEAM * NBUF * NQ * G * NB;
  static_assert(TCOLS <= 256, "TMEM columns");
  constexpr int NCOLS = TCOLS <= 32 ? 32 : (TCOLS <= 64 ? 64 : (TCOLS <= 128 ? 128 : 256));
  constexpr uint32_t BYTES = (uint32_t)S * C::SLICE;          // one A block's slices
  constexpr uint32_t BYTES_B = (uint32_t)NP * S * C::SLICE;   // B block (pair) slices
  // pipeline b (one per team): stages b NSTP .. b NSTP + NSTP - 1 of the
  // ring and descriptor ring b, each filled and consumed strictly in order
  constexpr int NSTP = C::NST / NTEAM;
  static_assert(NSTP <= 32, "stages per pipeline");
  constexpr int kProd0 = kEpiWarps, kMma0 = kEpiWarps + NTEAM;  // warps of pipeline 0
  extern __shared__ __align__(1024) uint8_t smem[];
  // tfull / tempty: per (team, buffer), index 2 * team + buffer
  __shared__ __align__(8) uint64_t full[C::NST], empty[C::NST], tfull[4], tempty[4], done;
  __shared__ __align__(8) uint64_t meta_full[2][kMeta], meta_empty[2][kMeta];
  __shared__ Meta meta[2][kMeta];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *stages = smem;
  int32_t *comb = reinterpret_cast<int32_t *>(smem + C::NST * C::STAGE);

  // zero the slice ring once: the pad slots stay zero (copies fill only the
  // S slice slots of each stage)
  for (int i = tid; i < C::NST * C::STAGE / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(stages)[i] = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (tid == 0) {
    for (int i = 0; i < C::NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 4; i++) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kTeam);  // buffers 2t, 2t+1 belong to team t
    }
    for (int b = 0; b < 2; b++)
      for (int i = 0; i < kMeta; i++) {
        mbar_init(&meta_full[b][i], 1);
        mbar_init(&meta_empty[b][i], kTeam + 1);  // the pipeline's MMA thread and team
      }
    mbar_init(&done, NTEAM);
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

  if (warp >= kProd0 && warp < kProd0 + NTEAM) {
    // --------------------------------------------------------- producer warp
    // Claims chunks of kChunk consecutive C blocks (Morton order) from a
    // global counter; the chunk's descriptors and its contiguous range of
    // block products are loaded 32 at a time by the whole warp.  Lane 0 does
    // the barrier work and issues the copies.  Two sentinel descriptors
    // (nk = -1) end the consumers.  The epilogue loads the scale exponents
    // itself.
    const int b = warp - kProd0;  // the pipeline
    uint64_t *const mfull = meta_full[b], *const mempty = meta_empty[b];
    Meta *const mring = meta[b];
    uint32_t it = 0, q = 0;
    uint32_t pend = 0, ppar = 0;  // bit s: local stage s has a fill issued / its phase parity
    bool stop = false;
    // the current product's descriptor fields, reloaded when it changes
    int pc = -1;
    const uint8_t *asl = nullptr, *bsl = nullptr;
    const int32_t *tap = nullptr, *tbp = nullptr;
    int64_t na = 0, nb = 0, nt = 0;
    double *cvp = nullptr;
    int32_t *nzp = nullptr;
    const int *rexp = nullptr, *cexp = nullptr;
    // one work item's descriptor into the ring (lane 0 writes; every lane
    // returns whether it was written).  x-th C block: a pair's siblings, or
    // the C blocks of lanes i .. i + nq - 1 (grouped items).
    auto put_meta = [&](const int64_t (&c)[NSUB], const int32_t (&bi)[NSUB],
                        const int32_t (&bj)[NSUB], const int32_t (&nkq)[NSUB], int nq,
                        int nk) -> bool {
      const int m = q % kMeta;
      int okw = 1;
      if (lane == 0) {
        okw = mbar_wait(&mempty[m], ((q / kMeta) & 1u) ^ 1u) && !abort_flag;
        if (!okw) {
          set_err(P.err, DERR_TIMEOUT);
          abort_flag = 1;
        } else {
#pragma unroll
          for (int x = 0; x < NSUB; x++) {
            mring[m].c[x] = c[x];
            mring[m].bi[x] = bi[x];
            mring[m].bj[x] = bj[x];
            if (NQ > 1) mring[m].nkq[x] = nkq[x];
          }
          mring[m].cv = cvp;
          mring[m].nz = nzp;
          mring[m].rowexp = rexp;
          mring[m].colexp = cexp;
          mring[m].nk = nk;
          mring[m].nq = nq;
          // a grouped item is one narrow flush: list lq into its own columns
          const FlushPlan fp = nq > 1 || nk < 0 ? FlushPlan{false, nk, 1, 1}
                                               : flush_plan(nk, P.flushk, P.flushk_wide);
          mring[m].nfl = fp.nfl;
          mring[m].fk = (int16_t)fp.fk;
          mring[m].wide = fp.wide ? 1 : 0;
          mbar_arrive(&mfull[m]);  // release: the descriptor is visible
        }
      }
      okw = __shfl_sync(0xffffffffu, okw, 0);
      q++;
      return okw != 0;
    };
    // grouped items: C blocks of at most gmax products (one narrow flush on
    // the fast combine path) of one product, consecutive in the work list
    const int gmax = NQ > 1 ? min(P.flushk, kFast) : 0;
    // window of 32 consecutive products (ta, tb) of one product table entry
    int wp = -1;
    int32_t tw = 0, ta_w = 0, tb_w = 0;
    while (!stop) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(P.work, (unsigned long long)P.chunk);
      base = __shfl_sync(0xffffffffu, base, 0);
      if ((int64_t)base >= P.nitems) break;
      const int n = (int)min((int64_t)P.chunk, P.nitems - (int64_t)base);
      // lane i: descriptor of work item base + i
      int pi = 0;
      int64_t ci = 0;
      int32_t s0 = 0, s1 = 0;
      int64_t e0 = 0, e1 = -1;  // the item's C blocks (e1: a pair's odd sibling)
      int32_t kbi = 0, kbj = 0;  // block row and column of the item's C block
      if (lane < n) {
        if (P.items) {
          const uint64_t it = P.items[base + lane];
          pi = (int)item_product(it);
          ci = item_cblock(it);
        } else {
          ci = (int64_t)base + lane;
        }
        const ProdDesc *pd = &P.prods[pi];
        s0 = pd->seg[ci];
        s1 = pd->seg[ci + 1];
        const uint64_t key = pd->ckeys[ci];
        kbi = (int32_t)morton_compact(key >> 1);
        kbj = (int32_t)morton_compact(key);
        if (NP == 2) {
          e0 = pd->pairc[2 * ci];
          e1 = pd->pairc[2 * ci + 1];
        } else {
          e0 = ci;
        }
      }
      for (int i = 0; i < n && !stop;) {
        const int p = __shfl_sync(0xffffffffu, pi, i);
        if (p != pc) {  // every lane keeps the product's fields
          const ProdDesc *pd = &P.prods[p];
          pc = p;
          asl = pd->asl;
          bsl = pd->bsl;
          tap = pd->ta;
          tbp = pd->tb;
          na = pd->na;
          nb = pd->nb;
          nt = pd->nt;
          cvp = pd->cv;
          nzp = pd->nz;
          rexp = pd->rowexp;
          cexp = pd->colexp;
        }
        // grouped item: the following items of the same product with short
        // lists (every lane takes the same decisions)
        const int32_t nk0 = __shfl_sync(0xffffffffu, s1, i) - __shfl_sync(0xffffffffu, s0, i);
        int nq = 1;
        if (NQ > 1 && nk0 >= 1 && nk0 <= gmax) {
          while (nq < NQ && i + nq < n) {
            const int j2 = i + nq;
            const int p2 = __shfl_sync(0xffffffffu, pi, j2);
            const int32_t n2 = __shfl_sync(0xffffffffu, s1, j2) - __shfl_sync(0xffffffffu, s0, j2);
            if (p2 != p || n2 < 1 || n2 > gmax) break;
            nq++;
          }
        }
        int64_t c[NSUB];
        int32_t bi[NSUB], bj[NSUB], nkq[NSUB];
        int nk = 0;
#pragma unroll
        for (int x = 0; x < NSUB; x++) {
          const int src = NP == 2 ? i : min(i + x, 31);
          const int64_t cx = __shfl_sync(0xffffffffu, NP == 2 && x == 1 ? e1 : e0, src);
          bi[x] = __shfl_sync(0xffffffffu, kbi, src);
          bj[x] = __shfl_sync(0xffffffffu, kbj, src) + (NP == 2 ? x : 0);  // the odd sibling
          nkq[x] = __shfl_sync(0xffffffffu, s1, src) - __shfl_sync(0xffffffffu, s0, src);
          const bool in = NP == 2 || x < nq;
          c[x] = in ? cx : -1;
          if (!in) nkq[x] = bi[x] = bj[x] = 0;  // (another product's lane)
          if (NP == 2 ? x == 0 : in) nk += nkq[x];
        }
        if (!put_meta(c, bi, bj, nkq, nq, nk)) {
          stop = true;
          break;
        }
        // the item's lists in order, one stage per block product; lane 0
        // issues (a failure stops it and ends the chunk after the item)
        int okc = 1;
        for (int lq = 0; lq < nq; lq++) {
          const int32_t k0 = __shfl_sync(0xffffffffu, s0, i + lq);
          int32_t nkx = NQ > 1 ? nkq[0] : nk;
#pragma unroll
          for (int x = 1; x < NSUB; x++)
            if (NQ > 1 && lq == x) nkx = nkq[x];
          for (int j = 0; j < nkx; j++, it++) {
            const int32_t t = k0 + j;
            if (p != wp || t < tw || t >= tw + 32) {  // refill the window (loads stay below nt)
              wp = p;
              tw = t;
              ta_w = tw + lane < nt ? tap[tw + lane] : 0;
              tb_w = tw + lane < nt ? tbp[tw + lane] : 0;
            }
            const int32_t aa = __shfl_sync(0xffffffffu, ta_w, t - tw);
            const int32_t bb = __shfl_sync(0xffffffffu, tb_w, t - tw);
            if (lane == 0 && okc) {
              const int sl = it % NSTP, st = b * NSTP + sl;  // local and ring stage
              if (!mbar_wait(&empty[st], ((it / NSTP) & 1u) ^ 1u) || abort_flag) {
                set_err(P.err, DERR_TIMEOUT);
                abort_flag = 1;
                okc = 0;
              } else {
                uint8_t *sa = stages + (size_t)st * C::STAGE;
                uint8_t *sb = sa + C::ASLOTS * C::SLICE;
                pend |= 1u << sl;
                ppar = (ppar & ~(1u << sl)) | (((it / NSTP) & 1u) << sl);
                if (aa < 0 || aa >= na || bb < 0 || bb >= nb) {
                  set_err(P.err, DERR_BOUNDS);  // complete the stage without data
                  mbar_arrive(&full[st]);
                } else {
                  mbar_expect_tx(&full[st], BYTES + BYTES_B);
                  bulk_g2s(sa + (DPG - 1) * C::SLICE, asl + (int64_t)aa * BYTES, BYTES, &full[st]);
                  bulk_g2s(sb, bsl + (int64_t)bb * BYTES_B, BYTES_B, &full[st]);
                }
              }
            }
          }
        }
        if (!__shfl_sync(0xffffffffu, okc, 0)) {
          stop = true;
          break;
        }
        i += nq;
      }
    }
    // end marker for the pipeline's MMA thread and team
    if (!stop) {
      int64_t c[NSUB];
      int32_t z[NSUB];
#pragma unroll
      for (int x = 0; x < NSUB; x++) {
        c[x] = -1;
        z[x] = 0;
      }
      put_meta(c, z, z, z, 1, -1);
    }
    // copies still in flight must land before the CTA exits
    if (lane == 0)
      for (int sl = 0; sl < NSTP; sl++)
        if ((pend >> sl) & 1u) mbar_wait(&full[b * NSTP + sl], (ppar >> sl) & 1u);
  } else if (warp >= kMma0 && warp < kMma0 + NTEAM) {
    // ---------------------------------------------------------- MMA issuers
    // Thread b issues the MMAs of pipeline b's items, whose stages it meets
    // in the order its producer filled them.
    if (lane == 0) {
      const int b = warp - kMma0;
      uint64_t *const mfull = meta_full[b], *const mempty = meta_empty[b];
      const Meta *const mring = meta[b];
      uint32_t it = 0, q = 0;
      uint32_t fcb = 0;  // flushes issued for team b
      const uint32_t sbase = smem_u32(stages);
      for (;; q++) {
        int m = q % kMeta;
        if (!mbar_wait(&mfull[m], (q / kMeta) & 1u)) {
          set_err(P.err, DERR_TIMEOUT);
          abort_flag = 1;
          break;
        }
        // (single blocks and pairs: one list, known at compile time)
        const int nk = mring[m].nk, nq = NQ > 1 ? mring[m].nq : 1;
        const bool fwide = mring[m].wide != 0;
        const FlushPlan fp{fwide, mring[m].fk, mring[m].nfl, fwide ? kFoldWide : kFold};
        int nkq[NQ];
#pragma unroll
        for (int x = 0; x < NQ; x++) nkq[x] = NQ > 1 ? mring[m].nkq[x] : nk;
        mbar_arrive(&mempty[m]);
        if (nk < 0 || abort_flag) break;  // end marker
        // the MMAs of the next stage (one block product) into buffer u,
        // list lq's columns; first: the flush's first product
        auto stage_mmas = [&](uint32_t u, int lq, uint32_t first) -> bool {
          const int st = b * NSTP + it % NSTP;
          if (!mbar_wait(&full[st], (it / NSTP) & 1u)) return false;
          tc_fence_after();
          // descriptors differ only in the start-address field (16-byte
          // units, < 2^14 inside shared memory): build them once per stage
          const uint32_t sa = sbase + st * C::STAGE;
          const uint64_t ad0 = smem_desc(sa, C::LBO, C::SBO);
          const uint64_t bd0 = smem_desc(sa + C::ASLOTS * C::SLICE, C::LBO, C::SBO);
          // (g, t): Toeplitz A tile of group g at offset t times the nbk B
          // slices of residue t, into groups g .. g + nbk - 1.  The first
          // instruction (g = t = h = 0) spans every group and starts the
          // accumulation of a flush.
#pragma unroll
          for (int g = 0; g < G; g++) {
            const uint32_t dt = tbase + (uint32_t)((((b * NBUF + u) * NQ + lq) * G + g) * NB);
#pragma unroll
            for (int t = 0; t < DPG; t++) {
              const int nbk = b_count(S, DPG, t) < G - g ? b_count(S, DPG, t) : G - g;
              if (nbk <= 0 || g * DPG - t >= S) continue;  // B slices or A rows all zero
              const uint32_t idesc = nbk == 1 ? IDESC1 : (nbk == 2 ? IDESC2 : IDESC3);
#pragma unroll
              for (int h = 0; h < BS / Fmt<F>::KPI; h++) {
                // one instruction's K = two core matrices = 256 bytes
                const uint64_t aoff = (uint64_t)(((DPG - 1 + g * DPG - t) * C::SLICE + h * 256) >> 4);
                // B: positions b_off(t) .. + nbk - 1, each one block's slice
                // or a pair's two slices side by side (N rows 0..bs-1 and
                // bs..2bs-1 of each position)
                const uint64_t boff =
                    (uint64_t)((NP * b_off(S, DPG, t) * C::SLICE + h * 256) >> 4);
                const uint32_t acc = (g | t | h) ? 1u : first;
                if (F == 0)
                  tc_mma_bf16(dt, ad0 + aoff, bd0 + boff, idesc, acc);
                else
                  tc_mma_f8(dt, ad0 + aoff, bd0 + boff, idesc, acc);
              }
            }
          }
          tc_commit(&empty[st]);  // stage reusable once these MMAs are done
          it++;
          return true;
        };
        for (int f = 0; f < fp.nfl && !abort_flag; f++) {
          const uint32_t fb = fcb++;
          const uint32_t u = fb % NBUF, use = fb / NBUF;  // buffer and its use count
          if (!mbar_wait(&tempty[2 * b + u], (use & 1u) ^ 1u)) {
            set_err(P.err, DERR_TIMEOUT);
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          bool ok = true;
          if (NQ > 1 && nq > 1) {
#pragma unroll
            for (int lq = 0; lq < NQ; lq++)
              for (int j = 0; lq < nq && j < nkq[lq] && ok; j++)
                ok = stage_mmas(u, lq, j == 0 ? 0u : 1u);
          } else {
            const int jend = min(nk, (f + 1) * fp.fk);
            for (int j = f * fp.fk; j < jend && ok; j++)
              ok = stage_mmas(u, 0, j == f * fp.fk ? 0u : 1u);
          }
          if (!ok) {
            set_err(P.err, DERR_TIMEOUT);
            abort_flag = 1;
          }
          tc_commit(&tfull[2 * b + u]);  // flush ready for the epilogue
        }
      }
      // no MMA may still be running when TMEM is released
      tc_commit(&done);
      if (!mbar_wait(&done, 0)) set_err(P.err, DERR_TIMEOUT);
    }
  } else {
    // ----------------------------------------------------------- epilogue
    // Single C blocks: two teams of eight warps, each at the end of its own
    // pipeline (its producer's items, its own TMEM buffers); pairs: one team
    // of sixteen warps.  Warp w of a team drains lane quadrant w % 4,
    // a slice of HC columns, and accumulates the exact diagonal sums straight
    // into the team's shared-memory buffer [d][r][c]; the team then combines
    // the diagonals of each output element.  With two teams one team's
    // recombination overlaps the other team's drain and the MMAs.
    constexpr int HC = NB / (kTeamWarps / 4);       // 16 columns per warp at bs 32
    constexpr int LG4 = NB * BS / 4;                // 4-column groups of one list
    constexpr int NG4 = NQ * LG4;                   // ... of an item
    constexpr int GRP = (NG4 + kTeam - 1) / kTeam;  // combine: groups per thread
    static_assert(NQ == 1 || G == 1, "grouped items: one diagonal group");
    const int team = warp / kTeamWarps, tw = warp % kTeamWarps, ttid = tid % kTeam;
    const int wq = tw & 3;
    const int row = wq * 32 + lane;       // TMEM lane = operand row
    const int L = row / BS, r = row % BS;
    const int c0 = (tw >> 2) * HC;
    const uint32_t lane_addr = (uint32_t)(wq * 32) << 16;
    int32_t *tcomb = comb + team * (C::COMB / 4);
    const int bar_id = 1 + team;
    uint32_t fct = 0;                     // flushes drained by this team
    uint64_t *const mfull = meta_full[team], *const mempty = meta_empty[team];
    const Meta *const mring = meta[team];
    for (uint32_t q = 0;; q++) {
      int m = q % kMeta;
      bool okm = mbar_wait(&mfull[m], (q / kMeta) & 1u);
      // every decision below is uniform across the warp (tcgen05.ld is
      // .sync.aligned) and, at the named barriers, across the team.  This
      // barrier also ends the previous item: its shared-memory diagonal
      // buffer is free.
      if (named_bar_or(bar_id, kTeam, !okm || abort_flag != 0)) {
        set_err(P.err, DERR_TIMEOUT);
        abort_flag = 1;
        break;
      }
      const int nk = mring[m].nk, nq = NQ > 1 ? mring[m].nq : 1;
      if (nk < 0) {  // end marker
        mbar_arrive(&mempty[m]);
        break;
      }
      const bool fwide = mring[m].wide != 0;
      const FlushPlan fplan{fwide, mring[m].fk, mring[m].nfl, fwide ? kFoldWide : kFold};
      int64_t cblk[NSUB];
#pragma unroll
      for (int x = 0; x < NSUB; x++) cblk[x] = mring[m].c[x];
      double *const cvp = mring[m].cv;
      int32_t *const nzp = mring[m].nz;
      const int *const rowexp = mring[m].rowexp, *const colexp = mring[m].colexp;
      // this thread's output elements: 4-column group g4 = ttid + i kTeam is
      // list g4 / LG4, row rr and list columns cn .. cn + 3 of it; item column
      // c4 = list * NB + cn lies in C block blk = c4 / BS of the item (a
      // pair's odd sibling follows the even one), at its column cc.  The
      // scale exponents are loaded here so that their latency hides behind
      // the first flush.
      // The descriptor's fields go to registers first and the slot is
      // released before the exponent loads: the arrive has release semantics
      // and would wait for every earlier load, the global ones included.
      int erow[GRP], oblk[GRP];
      int4 fcol[GRP];
      int64_t eoff[GRP], foff[GRP];
#pragma unroll
      for (int i = 0; i < GRP; i++) {
        const int g4 = min(ttid + i * kTeam, NG4 - 1);
        const int rem = g4 % LG4, rr = rem / (NB / 4);
        const int c4 = (g4 / LG4) * NB + (rem % (NB / 4)) * 4, blk = c4 / BS;
        int32_t bi = mring[m].bi[0], bj = mring[m].bj[0];
#pragma unroll
        for (int x = 1; x < NSUB; x++)
          if (blk == x) {
            bi = mring[m].bi[x];
            bj = mring[m].bj[x];
          }
        oblk[i] = blk;
        eoff[i] = (int64_t)bi * BS + rr;
        foff[i] = (int64_t)bj * BS + c4 % BS;
      }
      mbar_arrive(&mempty[m]);
#pragma unroll
      for (int i = 0; i < GRP; i++) {
        erow[i] = rowexp[eoff[i]];
        fcol[i] = *reinterpret_cast<const int4 *>(colexp + foff[i]);
      }
      // (a grouped item is one narrow flush on the fast path: every list has
      // at most kFast products)
      const int nfl = fplan.nfl, kf = fplan.kf;
      const bool wide = fplan.wide;
      const bool fast = nq > 1 || (!wide && nk <= kFast);  // uniform over the team
      const int ng4 = nq * LG4;                            // the item's groups
      int64_t *const fold = P.fold + ((int64_t)blockIdx.x * 2 + team) * (NB * BS * 2);
      bool ok = true;
      // Every warp runs all nfl iterations (doing no work once `ok` is false)
      // so that the team meets the same fold barriers whatever happened.
      for (int f = 0; f < nfl; f++, fct++) {
        if (ok) {
          bool w = mbar_wait(&tfull[2 * team + fct % NBUF], (fct / NBUF) & 1u);
          if (!__all_sync(0xffffffffu, w && abort_flag == 0)) {
            set_err(P.err, DERR_TIMEOUT);
            abort_flag = 1;
            ok = false;
          }
        }
        if (ok) {
          tc_fence_after();
          for (int lq = 0; lq < nq; lq++) {
#pragma unroll
            for (int g = 0; g < G; g++) {
              uint32_t v[HC];
              const uint32_t col =
                  (uint32_t)((((team * NBUF + fct % NBUF) * NQ + lq) * G + g) * NB + c0);
              if constexpr (HC == 16)
                tmem_ld16(tbase + lane_addr + col, v);
              else
                tmem_ld8(tbase + lane_addr + col, v);
              tmem_ld_wait();
              const int d = g * DPG + L;
              if (d < S) {
                // exact integer value of each FP32 sum (|D| < 2^22: magic add;
                // wide flushes, |D| <= 2^24: from the bits)
                int32_t *dst = tcomb + (d * BS + r) * C::CROW + lq * NB + c0;
#pragma unroll
                for (int x = 0; x < HC; x += 4) {
                  int4 val;
                  if (fast) {  // bit patterns of D + 1.5 2^23 (one flush)
                    val = make_int4((int32_t)__float_as_uint(__uint_as_float(v[x]) + kMagicF),
                                    (int32_t)__float_as_uint(__uint_as_float(v[x + 1]) + kMagicF),
                                    (int32_t)__float_as_uint(__uint_as_float(v[x + 2]) + kMagicF),
                                    (int32_t)__float_as_uint(__uint_as_float(v[x + 3]) + kMagicF));
                  } else if (!wide) {
                    val = make_int4(
                        (int32_t)(__float_as_uint(__uint_as_float(v[x]) + kMagicF) - kMagic),
                        (int32_t)(__float_as_uint(__uint_as_float(v[x + 1]) + kMagicF) - kMagic),
                        (int32_t)(__float_as_uint(__uint_as_float(v[x + 2]) + kMagicF) - kMagic),
                        (int32_t)(__float_as_uint(__uint_as_float(v[x + 3]) + kMagicF) - kMagic));
                  } else {
                    val = make_int4(f32_int_exact(v[x]), f32_int_exact(v[x + 1]),
                                    f32_int_exact(v[x + 2]), f32_int_exact(v[x + 3]));
                  }
                  if (f % kf != 0) {
                    const int4 old = *reinterpret_cast<const int4 *>(dst + x);
                    val.x += old.x;
                    val.y += old.y;
                    val.z += old.z;
                    val.w += old.w;
                  }
                  *reinterpret_cast<int4 *>(dst + x) = val;
                }
              }
            }
          }
          tc_fence_before();
          mbar_arrive(&tempty[2 * team + fct % NBUF]);
        }
        if ((f + 1) % kf == 0 && f + 1 < nfl) {
          // the 32-bit sums are full: fold them into this thread's (hi, lo)
          // pairs (items of several flushes have one list: c4 = cn < NB).
          // The barrier's OR makes `ok` uniform across the team.
          if (named_bar_or(bar_id, kTeam, !ok || abort_flag != 0)) {
            ok = false;
          } else {
#pragma unroll
            for (int i = 0; i < GRP; i++) {
              const int g4 = ttid + i * kTeam;
              if (g4 >= LG4) break;
              const int rr = g4 / (NB / 4), c4 = (g4 % (NB / 4)) * 4;
              int4 dv[S];
#pragma unroll
              for (int d = 0; d < S; d++)
                dv[d] = *reinterpret_cast<const int4 *>(tcomb + (d * BS + rr) * C::CROW + c4);
#pragma unroll
              for (int x = 0; x < 4; x++) {
                int32_t dg[S];
#pragma unroll
                for (int d = 0; d < S; d++)
                  dg[d] = x == 0 ? dv[d].x : x == 1 ? dv[d].y : x == 2 ? dv[d].z : dv[d].w;
                int64_t hi, lo;
                combine_digits<S, BETA, TS>(dg, hi, lo);
                int64_t *fp = fold + (rr * NB + c4 + x) * 2;
                if (f + 1 > kf) {
                  hi += fp[0];
                  lo += fp[1];
                }
                hi += lo >> TS;  // keep lo in [0, 2^TS): hi 2^TS + lo unchanged
                lo &= (1ll << TS) - 1;
                fp[0] = hi;
                fp[1] = lo;
              }
            }
            named_bar(bar_id, kTeam);  // folded before the next drain overwrites
          }
        }
      }
      if (named_bar_or(bar_id, kTeam, !ok || abort_flag != 0)) break;
      uint32_t any = 0;  // bit x: C block x of the item has an entry != 0
      constexpr int XS = BETA * (S + 1);
#pragma unroll
      for (int i = 0; i < GRP; i++) {
        const int g4 = ttid + i * kTeam;
        if (g4 >= ng4) break;  // bs 16: part of the team idles here
        const int rem = g4 % LG4, rr = rem / (NB / 4);
        const int c4 = (g4 / LG4) * NB + (rem % (NB / 4)) * 4, cc = c4 % BS;
        const int blk = oblk[i];
        int4 dv[S];
#pragma unroll
        for (int d = 0; d < S; d++)
          dv[d] = *reinterpret_cast<const int4 *>(tcomb + (d * BS + rr) * C::CROW + c4);
        double out[4];
        bool nzq = false;
        if (kFast > 0 && fast) {
#pragma unroll
          for (int x = 0; x < 4; x++) {
            uint32_t pat[S];
#pragma unroll
            for (int d = 0; d < S; d++)
              pat[d] = (uint32_t)(x == 0 ? dv[d].x : x == 1 ? dv[d].y : x == 2 ? dv[d].z : dv[d].w);
            const int64_t vv = narrow_combine<S, BETA>(pat);
            const int fx = x == 0 ? fcol[i].x : x == 1 ? fcol[i].y : x == 2 ? fcol[i].z : fcol[i].w;
            const int X = erow[i] + fx - XS;
            if (!int64_scaled_to_double(vv, X, out[x]))  // subnormal or overflow range
              out[x] = split_to_double_slow(vv >> TS, vv & ((1ll << TS) - 1), TS, X);
            nzq |= nonzero_f64(out[x]);
          }
        } else {
#pragma unroll
          for (int x = 0; x < 4; x++) {
            int32_t dg[S];
#pragma unroll
            for (int d = 0; d < S; d++)
              dg[d] = x == 0 ? dv[d].x : x == 1 ? dv[d].y : x == 2 ? dv[d].z : dv[d].w;
            int64_t hi, lo;
            combine_digits<S, BETA, TS>(dg, hi, lo);
            if (nfl > kf) {
              const int64_t *fp = fold + (rr * NB + c4 + x) * 2;
              hi += fp[0];
              lo += fp[1];
            }
            const int fx = x == 0 ? fcol[i].x : x == 1 ? fcol[i].y : x == 2 ? fcol[i].z : fcol[i].w;
            out[x] = split_to_double<TS>(hi, lo, erow[i] + fx - XS);
            nzq |= nonzero_f64(out[x]);
          }
        }
        int64_t cb = cblk[0];
#pragma unroll
        for (int x = 1; x < NSUB; x++)
          if (blk == x) cb = cblk[x];
        any |= (uint32_t)nzq << blk;
        if (cb >= 0) {  // a pair's absent sibling is computed as zero and dropped
          double2 *dst = reinterpret_cast<double2 *>(cvp + cb * (int64_t)BS * BS + rr * BS + cc);
          dst[0] = make_double2(out[0], out[1]);
          dst[1] = make_double2(out[2], out[3]);
        }
      }
      // nonzero flags (zeroed before the launch): any warp that saw an entry
      // != 0 of a C block marks it
#pragma unroll
      for (int x = 0; x < NSUB; x++) {
        const bool a = __any_sync(0xffffffffu, (any >> x) & 1u);
        if (lane == 0 && a && cblk[x] >= 0) nzp[cblk[x]] = 1;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, NCOLS);
  }
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int BS, int S, int F, int NP, int NQ = 1>
bsm_status launch_split(const SplitArgs &a, cudaStream_t s) {
  using C = Cfg<BS, S, F, NP, NQ>;
  static std::atomic<uint64_t> attr{0};
  BSM_TRY(once_per_device(attr, [&] {
    return cuda_status(cudaFuncSetAttribute(
        k_numeric_split<BS, S, F, NP, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  }));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t chunks = (a.nitems + a.chunk - 1) / a.chunk;
  int64_t grid = chunks < sms ? chunks : sms;
  if (grid < 1) return BSM_OK;
  if (!a.fold) return BSM_ERR_INVALID_ARG;  // sized by split_fold_bytes: grid <= SM count
  count_launch();
  k_numeric_split<BS, S, F, NP, NQ><<<(unsigned)grid, threads_for<C::NTEAM>(), C::SMEM, s>>>(a);
  return cuda_status(cudaGetLastError());
}

template <int BS>
bsm_status launch_split_s(const SplitArgs &a, int fmt, int slices, int np, cudaStream_t s) {
#define BSM_LS(F, S) \
  if (np == 1 && fmt == F && slices == S) return launch_split<BS, S, F, 1>(a, s);
#define BSM_LP(F, S) \
  if (np == 2 && fmt == F && slices == S) return launch_split<BS, S, F, 2>(a, s);
#define BSM_LG(F, S) \
  if (np == 4 && fmt == F && slices == S) return launch_split<BS, S, F, 1, 4>(a, s);
  BSM_LS(0, 1) BSM_LS(0, 2) BSM_LS(0, 3) BSM_LS(0, 4) BSM_LS(0, 5) BSM_LS(0, 6) BSM_LS(0, 7)
  BSM_LS(0, 8)
  if constexpr (BS == 32) {
    BSM_LS(1, 2) BSM_LS(1, 3) BSM_LS(1, 4) BSM_LS(1, 6) BSM_LS(1, 8) BSM_LS(1, 12)
    BSM_LP(0, 3) BSM_LP(0, 4) BSM_LP(0, 5) BSM_LP(0, 6) BSM_LP(0, 7) BSM_LP(0, 8)
    BSM_LP(1, 4) BSM_LP(1, 6) BSM_LP(1, 8) BSM_LP(1, 12)
  }
  if constexpr (BS == 16) {
    BSM_LP(0, 3) BSM_LP(0, 4) BSM_LP(0, 5) BSM_LP(0, 6) BSM_LP(0, 7) BSM_LP(0, 8)
    BSM_LG(0, 3) BSM_LG(0, 4) BSM_LG(0, 5) BSM_LG(0, 6) BSM_LG(0, 7) BSM_LG(0, 8)
  }
#undef BSM_LS
#undef BSM_LP
#undef BSM_LG
  return BSM_ERR_INVALID_ARG;
}

// ----------------------------------------------------------- pair items
// Siblings: keys that differ only in bit 0 (the block column's lowest bit).
__global__ void k_pair_heads(const uint64_t *__restrict__ keys, int64_t n,
                             int32_t *__restrict__ head) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = i == 0 || (keys[i] >> 1) != (keys[i - 1] >> 1);
}

// Pair index of every key; optionally pairc[2 p + (key & 1)] = i and the
// pair's even key.
__global__ void k_pair_assign(const uint64_t *__restrict__ keys, int64_t n,
                              const int32_t *__restrict__ head, const int32_t *__restrict__ hpos,
                              int32_t *__restrict__ slot, int32_t *__restrict__ pairc,
                              uint64_t *__restrict__ pkeys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t p = hpos[i] + head[i] - 1;
  if (slot) slot[i] = p;
  if (pairc) pairc[2 * (int64_t)p + (keys[i] & 1)] = (int32_t)i;
  if (pkeys && head[i]) pkeys[p] = keys[i] & ~1ull;
}

__device__ __forceinline__ uint32_t row_of(const uint64_t *bkeys, int32_t b) {
  return morton_compact(bkeys[b] >> 1);
}

// Merged product list of each C pair: the union over K of the two siblings'
// lists (both sorted by K); an entry is (A block, B pair slot).  write = 0:
// count only.
__global__ void k_pair_merge(const int32_t *__restrict__ pairc, int64_t npairs,
                             const int32_t *__restrict__ seg, const int32_t *__restrict__ ta,
                             const int32_t *__restrict__ tb, const uint64_t *__restrict__ bkeys,
                             const int32_t *__restrict__ bslot, int32_t *__restrict__ cnt,
                             const int32_t *__restrict__ mseg, int32_t *__restrict__ mta,
                             int32_t *__restrict__ mtb, int write) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int32_t c0 = pairc[2 * p], c1 = pairc[2 * p + 1];
  int32_t i0 = c0 >= 0 ? seg[c0] : 0, e0 = c0 >= 0 ? seg[c0 + 1] : 0;
  int32_t i1 = c1 >= 0 ? seg[c1] : 0, e1 = c1 >= 0 ? seg[c1 + 1] : 0;
  int32_t o = write ? mseg[p] : 0, n = 0;
  while (i0 < e0 || i1 < e1) {
    int32_t a, b;
    if (i1 >= e1) {
      a = ta[i0];
      b = tb[i0++];
    } else if (i0 >= e0) {
      a = ta[i1];
      b = tb[i1++];
    } else {
      const uint32_t k0 = row_of(bkeys, tb[i0]), k1 = row_of(bkeys, tb[i1]);
      if (k0 <= k1) {
        a = ta[i0];
        b = tb[i0++];
        if (k0 == k1) i1++;  // same A block, sibling B block of the same slot
      } else {
        a = ta[i1];
        b = tb[i1++];
      }
    }
    if (write) {
      mta[o + n] = a;
      mtb[o + n] = bslot[b];
    }
    n++;
  }
  if (!write) cnt[p] = n;
}

}  // namespace

// Largest group of k-products whose diagonal sums stay within 2^bound_log2
// (22: below the magic-number conversion's limit; 24: the largest integers
// FP32 holds exactly) in the FP32 accumulator: with digit base 2^B, d = 0
// sums terms up to 2^(2B); d >= 1 at most (d + 3) 2^(2B-2) per inner element.
int split_flush_group(int bs, int spec, int bound_log2) {
  const int beta = split_spec_fmt(spec) == 0 ? Fmt<0>::BETA : Fmt<1>::BETA;
  const int s = split_spec_slices(spec);
  int maxel = (1 << bound_log2) >> (2 * beta);                  // d = 0
  int m2 = ((1 << bound_log2) >> (2 * beta - 2)) / (s + 2);     // d = s - 1
  if (m2 < maxel) maxel = m2;
  int g = maxel / bs;
  return g < 1 ? 1 : g;
}

// Work items per claim.  Short product lists: 32 consecutive C blocks per
// atomic keep the claiming cheap.  Long lists: one C block per claim, so that
// the CTAs work on neighbouring C blocks (in Morton order) at the same time and
// share the slices of their A rows and B columns in L2 instead of each
// streaming its own region from HBM.
int split_chunk_for(int64_t nt, int64_t nc) {
  const int64_t avg = nc > 0 ? nt / nc : 0;
  return avg >= 16 ? 1 : (avg >= 4 ? 8 : 32);
}

size_t split_fold_bytes(int bs) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // per CTA and team: (hi, lo) for every output of an item (a pair: 2 bs^2)
  return (size_t)(sms > 0 ? sms : 1) * 2 * bs * (2 * bs) * 2 * sizeof(int64_t);
}

bsm_status split_supported(int bs, int spec) {
  if (bs != 16 && bs != 32) return BSM_ERR_UNSUPPORTED;
  const int fmt = split_spec_fmt(spec), slices = split_spec_slices(spec);
  if (fmt == 1 && bs != 32) return BSM_ERR_UNSUPPORTED;  // one E4M3 instruction spans K = 32
  if (fmt < 0 || fmt > 1) return BSM_ERR_INVALID_ARG;
  if (slices < 1 || slices > (fmt ? Fmt<1>::MAXS : Fmt<0>::MAXS)) return BSM_ERR_INVALID_ARG;
  if (!spec_compiled(fmt, slices)) return BSM_ERR_UNSUPPORTED;
  return BSM_OK;
}

// Buffers of the split form of one product: scale exponents of A's rows and
// B's columns and the digit slices of A and B.  Fills the split fields of `d`;
// the allocations are appended to `owned` for the caller to release.
bsm_status split_alloc(bsm_matrix A, bsm_matrix B, int spec, ProdDesc &d,
                       std::vector<void *> &owned, cudaStream_t s) {
  const int bs = A->bs;
  const size_t eb = split_spec_fmt(spec) == 0 ? 2 : 1, slices = split_spec_slices(spec);
  int *rowexp = nullptr, *colexp = nullptr;
  uint8_t *asl = nullptr, *bsl = nullptr;
  bsm_status st;
  if ((st = dev_alloc((void **)&rowexp, 4 * A->mb * bs, s)) != BSM_OK) return st;
  owned.push_back(rowexp);
  if ((st = dev_alloc((void **)&colexp, 4 * B->nb * bs, s)) != BSM_OK) return st;
  owned.push_back(colexp);
  if ((st = dev_alloc((void **)&asl, eb * slices * bs * bs * A->nblk, s)) != BSM_OK)
    return st;
  owned.push_back(asl);
  if ((st = dev_alloc((void **)&bsl, eb * slices * bs * bs * B->nblk, s)) != BSM_OK)
    return st;
  owned.push_back(bsl);
  d.asl = asl;
  d.bsl = bsl;
  d.rowexp = rowexp;
  d.colexp = colexp;
  return BSM_OK;
}

// Computes the exponents and slices into the buffers of `d` (no allocation;
// may be captured in a CUDA graph).
bsm_status split_compute(bsm_matrix A, bsm_matrix B, int spec, const ProdDesc &d,
                         unsigned *errword, cudaStream_t s, const int32_t *bslot) {
  const int fmt = split_spec_fmt(spec), slices = split_spec_slices(spec);
  const int bs = A->bs;
  int *rowexp = const_cast<int *>(d.rowexp), *colexp = const_cast<int *>(d.colexp);
  cudaMemsetAsync(rowexp, 0x80, 4 * A->mb * bs, s);  // 0x80808080: below any exponent
  cudaMemsetAsync(colexp, 0x80, 4 * B->nb * bs, s);
  if (A->nblk) {
    count_launch(1);
    k_row_exp<<<grid_for(A->nblk, 8), 256, 0, s>>>(A->vals, A->keys, A->nblk, bs, rowexp, errword);
  }
  if (B->nblk) {
    count_launch(1);
    k_col_exp<<<grid_for(B->nblk * bs, 256), 256, 0, s>>>(B->vals, B->keys, B->nblk, bs, colexp,
                                                         errword);
  }
  uint8_t *asl = const_cast<uint8_t *>(d.asl), *bsl = const_cast<uint8_t *>(d.bsl);
  if (bs == 16)
    launch_slices_s<16>(A, B, rowexp, colexp, asl, bsl, bslot, fmt, slices, s);
  else
    launch_slices_s<32>(A, B, rowexp, colexp, asl, bsl, bslot, fmt, slices, s);
  return cuda_status(cudaGetLastError());
}

// Longest product list of a task list, atomically maxed into *dmax_dev.
void launch_max_seg(const SymbolicResult &sym, int *dmax_dev, cudaStream_t s) {
  if (sym.nc == 0) return;
  count_launch(1);
  k_max_seg<<<grid_for(sym.nc, 256), 256, 0, s>>>(sym.seg, sym.nc, dmax_dev);
}

bsm_status split_prepare(bsm_matrix A, bsm_matrix B, int slices, unsigned *errword, ProdDesc &d,
                         std::vector<void *> &owned, cudaStream_t s) {
  BSM_TRY(split_alloc(A, B, slices, d, owned, s));
  return split_compute(A, B, slices, d, errword, s);
}

bsm_status split_launch(int bs, int spec, const ProdDesc *prods_dev, const uint64_t *items,
                        int64_t nitems, unsigned long long *work, unsigned *errword,
                        int64_t *fold, cudaStream_t s, int chunk, int np) {
  const int fmt = split_spec_fmt(spec), slices = split_spec_slices(spec);
  SplitArgs a;
  a.fold = fold;
  a.chunk = chunk < 1 ? 1 : (chunk > kChunk ? kChunk : chunk);
  a.prods = prods_dev;
  a.items = items;
  a.nitems = nitems;
  a.flushk = split_flush_group(bs, spec, 22);
  a.flushk_wide = split_flush_group(bs, spec, 24);
  a.err = errword;
  a.work = work;
  // item shape: 1 the default (grouped where split_use_groups), -1 single C
  // blocks, 4 grouped where compiled, 2 sibling pairs
  const bool gc = group_compiled(bs, fmt, slices);
  if (np == 1) np = split_use_groups(bs, spec) ? 4 : 1;
  else if (np == 4) np = gc ? 4 : 1;
  else if (np == -1) np = 1;
  return bs == 16 ? launch_split_s<16>(a, fmt, slices, np, s)
                  : launch_split_s<32>(a, fmt, slices, np, s);
}

ProdDesc make_desc(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, double *cvals,
                   int32_t *nz) {
  ProdDesc d = {};
  d.seg = sym.seg;
  d.ta = sym.ta;
  d.tb = sym.tb;
  d.ckeys = sym.ckeys;
  d.av = A->vals;
  d.bv = B->vals;
  d.cv = cvals;
  d.nz = nz;
  d.na = A->nblk;
  d.nb = B->nblk;
  d.nc = sym.nc;
  d.nt = sym.nt;
  return d;
}

// Grouped items (up to four C blocks of at most one narrow flush each share
// one work item) wherever compiled; the producer groups only C blocks of short
// lists, so the kernel is the single-block kernel for the others.
// BSM_SPLIT_GROUPS=0 in the environment turns them off.
bool split_groups_compiled(int bs, int spec) {
  return group_compiled(bs, split_spec_fmt(spec), split_spec_slices(spec));
}
bool split_use_groups(int bs, int spec) {
  if (!split_groups_compiled(bs, spec)) return false;
  const char *e = getenv("BSM_SPLIT_GROUPS");
  return !(e && e[0] == '0');
}

// Pair items (two sibling C blocks per MMA, N = 2 bs) for long product lists:
// each A tile then serves twice the outputs.  BSM_SPLIT_PAIRS=0 / 1 in the
// environment turns them off / on regardless of the list length.
bool split_use_pairs(int bs, int spec, int64_t nt, int64_t nc) {
  if (!pair_compiled(bs, split_spec_fmt(spec), split_spec_slices(spec))) return false;
  const char *e = getenv("BSM_SPLIT_PAIRS");
  if (e && e[0] == '0') return false;
  if (e && e[0] == '1') return true;
  return nc > 0 && nt >= 16 * nc;
}

// Pair items of one product: B pair slots, C sibling pairs and their merged
// product lists (structure only; no values).  Fills the task-list fields of
// `d` (seg, ta, tb, ckeys, nc, nt, nb, pairc), allocates the A slices, the B
// slices in pair slots (zeroed: absent siblings stay zero) and the exponents
// (one spare block column), and returns the B pair slot of every B block for
// split_compute.  Allocations are appended to `owned`.
bsm_status split_pairs_prepare(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, int spec,
                               ProdDesc &d, int32_t **bslot_out, std::vector<void *> &owned,
                               cudaStream_t s) {
  const int bs = A->bs, fmt = split_spec_fmt(spec);
  const int64_t slices = split_spec_slices(spec), eb = fmt == 0 ? 2 : 1;
  const int64_t nb = B->nblk, nc = sym.nc;
  *bslot_out = nullptr;
  auto grab = [&](void **p, size_t bytes) -> bsm_status {
    bsm_status r = dev_alloc(p, bytes > 0 ? bytes : 16, s);
    if (r == BSM_OK) owned.push_back(*p);
    return r;
  };
  int32_t *h32 = (int32_t *)host_scratch().get(64);
  if (!h32) return BSM_ERR_OOM;
  int32_t *bhead, *bpos, *bslot, *chead, *cpos, *pairc, *cnt, *mseg, *mta, *mtb;
  uint64_t *pkeys;
  BSM_TRY(grab((void **)&bhead, 4 * nb));
  BSM_TRY(grab((void **)&bpos, 4 * nb));
  BSM_TRY(grab((void **)&bslot, 4 * nb));
  BSM_TRY(grab((void **)&chead, 4 * nc));
  BSM_TRY(grab((void **)&cpos, 4 * nc));
  count_launch(2);
  if (nb) k_pair_heads<<<grid_for(nb, 256), 256, 0, s>>>(B->keys, nb, bhead);
  if (nc) k_pair_heads<<<grid_for(nc, 256), 256, 0, s>>>(sym.ckeys, nc, chead);
  BSM_TRY(scan_exclusive_i32(bhead, bpos, nb, s));
  BSM_TRY(scan_exclusive_i32(chead, cpos, nc, s));
  h32[0] = h32[1] = h32[2] = h32[3] = 0;
  if (nb) {
    readback(h32 + 0, bpos + nb - 1, 4, s);
    readback(h32 + 1, bhead + nb - 1, 4, s);
  }
  if (nc) {
    readback(h32 + 2, cpos + nc - 1, 4, s);
    readback(h32 + 3, chead + nc - 1, 4, s);
  }
  BSM_CUDA(cudaStreamSynchronize(s));
  const int64_t npb = (int64_t)h32[0] + h32[1], npc = (int64_t)h32[2] + h32[3];
  BSM_TRY(grab((void **)&pairc, 8 * npc));
  BSM_TRY(grab((void **)&pkeys, 8 * npc));
  BSM_TRY(grab((void **)&cnt, 4 * (npc + 1)));
  BSM_TRY(grab((void **)&mseg, 4 * (npc + 1)));
  cudaMemsetAsync(pairc, 0xFF, 8 * npc, s);  // -1: absent sibling
  cudaMemsetAsync(cnt + npc, 0, 4, s);
  count_launch(3);
  if (nb)
    k_pair_assign<<<grid_for(nb, 256), 256, 0, s>>>(B->keys, nb, bhead, bpos, bslot, nullptr,
                                                    nullptr);
  if (nc) {
    k_pair_assign<<<grid_for(nc, 256), 256, 0, s>>>(sym.ckeys, nc, chead, cpos, nullptr, pairc,
                                                    pkeys);
    k_pair_merge<<<grid_for(npc, 128), 128, 0, s>>>(pairc, npc, sym.seg, sym.ta, sym.tb, B->keys,
                                                    bslot, cnt, nullptr, nullptr, nullptr, 0);
  }
  BSM_TRY(scan_exclusive_i32(cnt, mseg, npc + 1, s));
  readback(h32, mseg + npc, 4, s);
  BSM_CUDA(cudaStreamSynchronize(s));
  const int64_t mt = h32[0];
  BSM_TRY(grab((void **)&mta, 4 * mt));
  BSM_TRY(grab((void **)&mtb, 4 * mt));
  if (npc) {
    count_launch();
    k_pair_merge<<<grid_for(npc, 128), 128, 0, s>>>(pairc, npc, sym.seg, sym.ta, sym.tb, B->keys,
                                                    bslot, nullptr, mseg, mta, mtb, 1);
  }
  int *rowexp, *colexp;
  uint8_t *asl, *bsl;
  const size_t slice_bytes = (size_t)eb * bs * bs;
  // colexp has one spare block column: the odd sibling of a pair in the last
  // block column reads its (unused) exponents there
  BSM_TRY(grab((void **)&rowexp, 4 * A->mb * bs));
  BSM_TRY(grab((void **)&colexp, 4 * (B->nb + 1) * bs));
  BSM_TRY(grab((void **)&asl, slice_bytes * slices * A->nblk));
  BSM_TRY(grab((void **)&bsl, slice_bytes * 2 * slices * npb));
  cudaMemsetAsync(bsl, 0, slice_bytes * 2 * slices * npb, s);
  d.asl = asl;
  d.bsl = bsl;
  d.rowexp = rowexp;
  d.colexp = colexp;
  d.seg = mseg;
  d.ta = mta;
  d.tb = mtb;
  d.ckeys = pkeys;
  d.nb = npb;
  d.nc = npc;
  d.nt = mt;
  d.pairc = pairc;
  *bslot_out = bslot;
  return cuda_status(cudaGetLastError());
}

// The numeric phase of one product over pairs of sibling C blocks.
static bsm_status numeric_split_pairs(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym,
                                      int spec, double *cvals, int32_t *nzflag, unsigned *errword,
                                      cudaStream_t s) {
  const int bs = A->bs;
  std::vector<void *> owned;
  auto cleanup = [&]() {
    for (void *p : owned) dev_free(p, s);  // stream-ordered: after the kernel
  };
  ProdDesc d = make_desc(A, B, sym, cvals, nzflag);
  int32_t *bslot = nullptr;
  bsm_status st = split_pairs_prepare(A, B, sym, spec, d, &bslot, owned, s);
  if (st == BSM_OK) st = split_compute(A, B, spec, d, errword, s, bslot);
  int *scr = nullptr;
  int64_t *fold = nullptr;
  if (st == BSM_OK && (st = dev_alloc((void **)&scr, 16 + sizeof(ProdDesc), s)) == BSM_OK)
    owned.push_back(scr);
  if (st == BSM_OK && (st = dev_alloc((void **)&fold, split_fold_bytes(bs), s)) == BSM_OK)
    owned.push_back(fold);
  void *h = host_scratch().get(sizeof(ProdDesc) + 64);
  if (st == BSM_OK && !h) st = BSM_ERR_OOM;
  if (st == BSM_OK) {
    cudaMemsetAsync(scr, 0, 16, s);
    memcpy(h, &d, sizeof(ProdDesc));
    cudaMemcpyAsync(scr + 4, h, sizeof(ProdDesc), cudaMemcpyHostToDevice, s);
    st = cuda_status(cudaStreamSynchronize(s));  // the host staging buffer is reused
  }
  if (st == BSM_OK) {
    cudaMemsetAsync(nzflag, 0, 4 * sym.nc, s);  // the kernel marks the nonzero C blocks
    st = split_launch(bs, spec, reinterpret_cast<const ProdDesc *>(scr + 4), nullptr, d.nc,
                      reinterpret_cast<unsigned long long *>(scr + 2), errword, fold, s,
                      split_chunk_for(d.nt, d.nc), 2);
  }
  cleanup();
  return st;
}

bsm_status numeric_split(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, int slices,
                         double *cvals, int32_t *nzflag, unsigned *errword, cudaStream_t s) {
  const int bs = A->bs;
  BSM_TRY(split_supported(bs, slices));
  if (sym.nc == 0) return BSM_OK;
  if (split_use_pairs(bs, slices, sym.nt, sym.nc))
    return numeric_split_pairs(A, B, sym, slices, cvals, nzflag, errword, s);
  std::vector<void *> owned;
  auto cleanup = [&]() {
    for (void *p : owned) dev_free(p, s);  // stream-ordered: after the kernel
  };
  // scratch: [2..3] chunk counter, then the product table
  int *scr = nullptr;
  bsm_status st = dev_alloc((void **)&scr, 16 + sizeof(ProdDesc), s);
  if (st != BSM_OK) return st;
  owned.push_back(scr);
  cudaMemsetAsync(scr, 0, 16, s);
  ProdDesc d = make_desc(A, B, sym, cvals, nzflag);
  st = split_prepare(A, B, slices, errword, d, owned, s);
  int *h = (int *)host_scratch().get(16 + sizeof(ProdDesc));
  if (st == BSM_OK && !h) st = BSM_ERR_OOM;
  if (st == BSM_OK) {
    memcpy(h + 4, &d, sizeof(ProdDesc));
    cudaMemcpyAsync(scr + 4, h + 4, sizeof(ProdDesc), cudaMemcpyHostToDevice, s);
    st = cuda_status(cudaStreamSynchronize(s));  // the host staging buffer is reused
  }
  int64_t *fold = nullptr;
  if (st == BSM_OK && (st = dev_alloc((void **)&fold, split_fold_bytes(bs), s)) == BSM_OK)
    owned.push_back(fold);
  if (st == BSM_OK) {
    cudaMemsetAsync(nzflag, 0, 4 * sym.nc, s);  // the kernel marks the nonzero C blocks
    st = split_launch(bs, slices, reinterpret_cast<const ProdDesc *>(scr + 4), nullptr, sym.nc,
                      reinterpret_cast<unsigned long long *>(scr + 2), errword, fold, s,
                      split_chunk_for(sym.nt, sym.nc));
  }
  cleanup();
  return st;
}
