// bsm_block_products_fp64_noalloc: the FP64 numeric phase over a caller's task
// list, with no allocation of any kind.
//
// Who needs this: code that must not call cudaMalloc (or cudaMallocAsync,
// cudaMallocHost, or an allocating library routine) on its hot path -- for
// example a process whose device memory is entirely reserved up front by
// another allocator, so that any new allocation fails, or a latency-critical
// loop where an allocation's implicit synchronisation is not acceptable.  The
// caller passes every input and output buffer; the only other memory used is
// the file-scope scratch array below.
//
// The scratch array is a static device array: every GPU on which a call was
// made holds it (about 4 MiB) from that first call -- which loads the module
// and may therefore allocate -- until the process exits.  All calls share it
// and it keeps the last call's contents, so calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race on it
// and must be serialised by the caller.  The error word is cleared on the
// stream at the start of every call; the flags are fully rewritten for the C
// blocks of each call.
#include <mutex>

#include "bsm_fp64_body.cuh"
#include "bsm_ptx.cuh"

namespace {

constexpr int kErrWords = 64;  // word 0: device error code; the rest pads to 256 B

// [flags of up to BSM_NOALLOC_MAX_CBLOCKS C blocks | error word + padding]
static __device__ __align__(256) int32_t g_scratch[BSM_NOALLOC_MAX_CBLOCKS + kErrWords];

// The library's FP64 per-C-block body (one CTA per C block, bulk-copy ring,
// DMMA, bounds check and bounded waits); the nonzero flag goes to the
// scratch array, and a C block whose CTA gave up (bad index or timed-out
// wait) has its flag cleared, so that only the error word reports it.
template <int BS, int MODE>
__global__ void __launch_bounds__(128) k_products_fp64_noalloc(
    const int32_t *__restrict__ seg, const int32_t *__restrict__ ta, const int32_t *__restrict__ tb,
    int64_t nc, int64_t na, int64_t nb, const double *__restrict__ Av,
    const double *__restrict__ Bv, double *__restrict__ Cv, int32_t *__restrict__ flags,
    unsigned *__restrict__ err) {
  extern __shared__ __align__(128) double smem[];
  __shared__ __align__(8) uint64_t full[kFp64Stages];
  const int64_t c = blockIdx.x;
  if (c >= nc) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kFp64Stages; s++) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t use0 = 0, use1 = 0;
  if (!cblock_fp64<BS, MODE>(seg, ta, tb, c, na, nb, Av, Bv, Cv, flags, err, smem, full, use0,
                             use1) &&
      threadIdx.x == 0)
    flags[c] = 0;
}

// One CTA: counts the nonzero flags; writes -1 if any CTA recorded an error.
__global__ void k_count_flags_noalloc(const int32_t *__restrict__ flags, int64_t nc,
                                      const unsigned *__restrict__ err,
                                      int64_t *__restrict__ out) {
  __shared__ int64_t part[32];
  int64_t n = 0;
  for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) n += flags[i] != 0;
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    *out = (*err != DERR_NONE) ? -1 : t;
  }
}

template <int BS>
constexpr size_t smem_bytes() {
  return (size_t)kFp64Stages * 2 * BS * BS * sizeof(double);
}

// Per-device set-up, done once per device by the first call made with that
// device current: the device address of g_scratch (in host code the symbol
// itself is only a host-side stand-in, not a device address) and the
// kernels' shared-memory attributes.  Under lazy module loading this is also
// when the module -- the scratch array and the kernels of every block size --
// is loaded onto the device, which may allocate device memory: the first call
// on each device must therefore come before the caller reserves all device
// memory and before any stream capture.
std::mutex g_mu;
int32_t *g_ptr[64] = {};

bsm_status setup_current_device(int32_t **out) {
  int dev = 0;
  BSM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BSM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorUnknown : e);
    BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<16, 0>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<16>()));
    BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<32, 0>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<32>()));
    BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<64, 0>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<64>()));
    BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<16, 1>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<16>()));
    BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<32, 1>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<32>()));
    BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<64, 1>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<64>()));
    cudaFuncAttributes fa;
    BSM_CUDA(cudaFuncGetAttributes(&fa, k_count_flags_noalloc));
    g_ptr[dev] = (int32_t *)p;
  }
  *out = g_ptr[dev];
  return BSM_OK;
}

template <int BS>
bsm_status launch(int64_t nc, const int32_t *seg, const int32_t *ta, const int32_t *tb,
                  const double *a, int64_t na, const double *b, int64_t nb, double *c,
                  int32_t *flags, unsigned *err, cudaStream_t s) {
  if (nc > 0 && fp64_mode() == 1)
    k_products_fp64_noalloc<BS, 1><<<(unsigned)nc, 128, smem_bytes<BS>(), s>>>(
        seg, ta, tb, nc, na, nb, a, b, c, flags, err);
  else if (nc > 0)
    k_products_fp64_noalloc<BS, 0><<<(unsigned)nc, 128, smem_bytes<BS>(), s>>>(
        seg, ta, tb, nc, na, nb, a, b, c, flags, err);
  return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" bsm_status bsm_block_products_fp64_noalloc(int bs, int64_t nc, const int32_t *seg,
                                                      const int32_t *ta, const int32_t *tb,
                                                      const double *a_vals, int64_t na,
                                                      const double *b_vals, int64_t nb,
                                                      double *c_vals, int64_t *nnz_out,
                                                      void *stream) {
  if (bs != 16 && bs != 32 && bs != 64) return BSM_ERR_BLOCKSIZE;
  if (nc < 0 || na < 0 || nb < 0 || !nnz_out) return BSM_ERR_INVALID_ARG;
  if (nc > BSM_NOALLOC_MAX_CBLOCKS) return BSM_ERR_UNSUPPORTED;  // beyond the scratch array
  if (nc > 0 && (!seg || !ta || !tb || !a_vals || !b_vals || !c_vals)) return BSM_ERR_INVALID_ARG;
  // blocks are staged by bulk copies and stored with 16-byte vector stores
  if (((uintptr_t)a_vals | (uintptr_t)b_vals | (uintptr_t)c_vals) & 15) return BSM_ERR_INVALID_ARG;
  int32_t *scratch = nullptr;
  BSM_TRY(setup_current_device(&scratch));
  int32_t *flags = scratch;
  unsigned *err = (unsigned *)(scratch + BSM_NOALLOC_MAX_CBLOCKS);
  cudaStream_t s = (cudaStream_t)stream;
  BSM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));  // must start at zero every call
  bsm_status st = BSM_OK;
  switch (bs) {
    case 16: st = launch<16>(nc, seg, ta, tb, a_vals, na, b_vals, nb, c_vals, flags, err, s); break;
    case 32: st = launch<32>(nc, seg, ta, tb, a_vals, na, b_vals, nb, c_vals, flags, err, s); break;
    default: st = launch<64>(nc, seg, ta, tb, a_vals, na, b_vals, nb, c_vals, flags, err, s); break;
  }
  if (st != BSM_OK) return st;
  k_count_flags_noalloc<<<1, 1024, 0, s>>>(flags, nc, err, nnz_out);
  return cuda_status(cudaGetLastError());
}
