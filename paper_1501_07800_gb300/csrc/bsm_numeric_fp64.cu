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
// pair's FP64 arithmetic: scalar DFMA by default (each thread a tile of
// outputs summed one k at a time), or the FP64 tensor path (mma.sync m8n8k4
// f64).  tcgen05 has no f64 kind, and on GB300 both forms share one FP64 pipe
// of about 1.1-1.26 TFLOP/s, far below what the copies can feed, so the kernel
// only has to keep that pipe busy; DFMA keeps it busier.  The epilogue also
// raises the C block's nonzero flag (exact-zero detection).
//
// Two launch forms share the per-C-block body: one CTA per C block of a single
// product, and a persistent form that walks a global work list of
// (product, C block) items of many independent products (batched products),
// claiming items from an atomic counter in the list's order.
#include <cstdlib>

#include "bsm_batch.cuh"
#include "bsm_fp64_body.cuh"
#include "bsm_ptx.cuh"

// Arithmetic form of the FP64 body (0: DMMA, 1: DFMA).  On GB300 scalar DFMA
// outruns the FP64 tensor path (measured: 1.257 against 1.102 TFLOP/s on
// every SM at 2070 MHz, the two sharing one FP64 pipe), so DFMA is the
// default; BSM_FP64_MODE=dmma or dfma in the environment chooses the form for
// the process.
int fp64_mode() {
  static const int mode = [] {
    const char *e = getenv("BSM_FP64_MODE");
    if (e && e[0] == 'd' && e[1] == 'm') return 0;
    return 1;
  }();
  return mode;
}

namespace {

constexpr int kStages = kFp64Stages;

template <int BS, int MODE>
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
  cblock_fp64<BS, MODE>(seg, ta, tb, c, na, nb, Av, Bv, Cv, nzflag, err, smem, full, use0, use1);
}

// Persistent form over a global work list of (product, C block) items.
template <int BS, int MODE>
__global__ void __launch_bounds__(128, 4) k_numeric_fp64_batched(const ProdDesc *__restrict__ prods,
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
    if (!cblock_fp64<BS, MODE>(p.seg, p.ta, p.tb, item_cblock(it), p.na, p.nb, p.av, p.bv, p.cv,
                               p.nz, err, smem, full, use0, use1))
      break;
  }
}

template <int BS, int MODE>
bsm_status launch(const SymbolicResult &sym, bsm_matrix A, bsm_matrix B, double *Cv, int32_t *nz,
                  unsigned *err, cudaStream_t s) {
  size_t smem = (size_t)kStages * 2 * BS * BS * sizeof(double);
  static std::atomic<uint64_t> attr{0};
  BSM_TRY(once_per_device(attr, [&] {
    return cuda_status(cudaFuncSetAttribute(
        k_numeric_fp64<BS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }));
  // one CTA per C block (nc < 2^31 is checked by the caller)
  count_launch();
  k_numeric_fp64<BS, MODE><<<(unsigned)sym.nc, 128, smem, s>>>(
      sym.seg, sym.ta, sym.tb, sym.nc, A->nblk, B->nblk, A->vals, B->vals, Cv, nz, err);
  return cuda_status(cudaGetLastError());
}

template <int BS, int MODE>
bsm_status launch_batched(const ProdDesc *prods, const uint64_t *items, int64_t nitems,
                          unsigned long long *counter, unsigned *err, int ctas_per_sm,
                          cudaStream_t s) {
  size_t smem = (size_t)kStages * 2 * BS * BS * sizeof(double);
  static std::atomic<uint64_t> attr{0};
  BSM_TRY(once_per_device(attr, [&] {
    return cuda_status(cudaFuncSetAttribute(
        k_numeric_fp64_batched<BS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)smem));
  }));
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  BSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_numeric_fp64_batched<BS, MODE>,
                                                         128, smem));
  if (occ < 1) occ = 1;
  if (ctas_per_sm <= 0 || ctas_per_sm > occ) ctas_per_sm = occ;
  int64_t grid = (int64_t)sms * ctas_per_sm;
  if (grid > nitems) grid = nitems;
  if (grid < 1) return BSM_OK;
  count_launch();
  k_numeric_fp64_batched<BS, MODE><<<(unsigned)grid, 128, smem, s>>>(prods, items, nitems,
                                                                     counter, err);
  return cuda_status(cudaGetLastError());
}

}  // namespace

bsm_status numeric_fp64(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, double *cvals,
                        int32_t *nzflag, unsigned *errword, cudaStream_t s) {
  if (sym.nc == 0) return BSM_OK;
  if (sym.nc > 0x7FFFFFFF) return BSM_ERR_UNSUPPORTED;
  const bool f = fp64_mode() == 1;
  switch (A->bs) {
    case 16: return f ? launch<16, 1>(sym, A, B, cvals, nzflag, errword, s)
                      : launch<16, 0>(sym, A, B, cvals, nzflag, errword, s);
    case 32: return f ? launch<32, 1>(sym, A, B, cvals, nzflag, errword, s)
                      : launch<32, 0>(sym, A, B, cvals, nzflag, errword, s);
    case 64: return f ? launch<64, 1>(sym, A, B, cvals, nzflag, errword, s)
                      : launch<64, 0>(sym, A, B, cvals, nzflag, errword, s);
  }
  return BSM_ERR_BLOCKSIZE;
}

bsm_status numeric_fp64_batched(int bs, const ProdDesc *prods, const uint64_t *items,
                                int64_t nitems, unsigned long long *counter, unsigned *errword,
                                int ctas_per_sm, cudaStream_t s, int form) {
  if (nitems == 0) return BSM_OK;
  // form: 0 DMMA; 1, 2, 3 DFMA tiles of BS/8, BS/16, BS/4 columns per thread
  const int f = form < 0 ? fp64_mode() : form;
#define BSM_LB(B)                                                                                \
  return f == 1   ? launch_batched<B, 1>(prods, items, nitems, counter, errword, ctas_per_sm, s) \
         : f == 2 ? launch_batched<B, 2>(prods, items, nitems, counter, errword, ctas_per_sm, s) \
         : f == 3 ? launch_batched<B, 3>(prods, items, nitems, counter, errword, ctas_per_sm, s) \
                  : launch_batched<B, 0>(prods, items, nitems, counter, errword, ctas_per_sm, s)
  switch (bs) {
    case 16: BSM_LB(16);
    case 32: BSM_LB(32);
    case 64: BSM_LB(64);
  }
#undef BSM_LB
  return BSM_ERR_BLOCKSIZE;
}
