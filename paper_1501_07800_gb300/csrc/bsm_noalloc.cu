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
// The scratch array is a static device array: every GPU that loads this
// library holds it (about 4 MiB) until the process exits.  All calls share it
// and it keeps the last call's contents, so calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race on it
// and must be serialised by the caller.  The error word is cleared on the
// stream at the start of every call; the flags are fully rewritten for the C
// blocks of each call.
#include <mutex>

#include "bsm_ptx.cuh"

namespace {

constexpr int kStages = 2;
constexpr int kErrWords = 64;  // word 0: device error code; the rest pads to 256 B

// [flags of up to BSM_NOALLOC_MAX_CBLOCKS C blocks | error word + padding]
static __device__ __align__(256) int32_t g_scratch[BSM_NOALLOC_MAX_CBLOCKS + kErrWords];

__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// Same work as the library's FP64 numeric kernel: one CTA sums the products of
// one C block on DMMA from bulk-copied blocks.  Its nonzero flag goes to the
// scratch array instead of a caller or pool buffer.
template <int BS>
__global__ void __launch_bounds__(128) k_products_fp64_noalloc(
    const int32_t *__restrict__ seg, const int32_t *__restrict__ ta, const int32_t *__restrict__ tb,
    int64_t nc, int64_t na, int64_t nb, const double *__restrict__ Av,
    const double *__restrict__ Bv, double *__restrict__ Cv, int32_t *__restrict__ flags,
    unsigned *__restrict__ err) {
  constexpr int BB = BS * BS;
  constexpr int WT = BS / 2;
  constexpr int TW = WT / 8;
  extern __shared__ __align__(128) double smem[];
  __shared__ __align__(8) uint64_t full[kStages];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wr = warp >> 1, wc = warp & 1;
  const int64_t c = blockIdx.x;
  if (c >= nc) return;
  const int32_t k0 = seg[c], nk = seg[c + 1] - k0;
  bool bad = nk < 0;
  for (int j = tid; j < nk; j += blockDim.x)
    bad |= ta[k0 + j] < 0 || ta[k0 + j] >= na || tb[k0 + j] < 0 || tb[k0 + j] >= nb;
  if (__syncthreads_or(bad)) {
    if (tid == 0) {
      set_err(err, DERR_BOUNDS);
      flags[c] = 0;
    }
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
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
    int s = j % kStages;
    if (!mbar_wait(&full[s], (uint32_t)(j / kStages) & 1u)) ok = false;
    if (__syncthreads_or(!ok)) {
      ok = false;
      jfail = j;
      break;
    }
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
    __syncthreads();
    if (tid == 0 && j + kStages < nk) issue(j + kStages);
  }
  if (!ok) {
    if (tid == 0) {
      set_err(err, DERR_TIMEOUT);
      flags[c] = 0;
      for (int j = jfail; j < jfail + kStages && j < nk; j++)
        mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
    }
    return;
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
  if (tid == 0) flags[c] = nzb;
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

// Device address of g_scratch, looked up once per device with that device
// current (a host-side use of the symbol itself would not be a device address).
std::mutex g_mu;
int32_t *g_ptr[64] = {};
bool g_attr[64][3] = {};

bsm_status scratch_for_current_device(int32_t **out, int *dev_out) {
  int dev = 0;
  BSM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BSM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorUnknown : e);
    g_ptr[dev] = (int32_t *)p;
  }
  *out = g_ptr[dev];
  *dev_out = dev;
  return BSM_OK;
}

template <int BS>
bsm_status launch(int dev, int64_t nc, const int32_t *seg, const int32_t *ta, const int32_t *tb,
                  const double *a, int64_t na, const double *b, int64_t nb, double *c,
                  int32_t *flags, unsigned *err, cudaStream_t s) {
  size_t smem = (size_t)kStages * 2 * BS * BS * sizeof(double);
  {
    std::lock_guard<std::mutex> g(g_mu);
    int slot = BS == 16 ? 0 : BS == 32 ? 1 : 2;
    if (!g_attr[dev][slot]) {
      BSM_CUDA(cudaFuncSetAttribute(k_products_fp64_noalloc<BS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      g_attr[dev][slot] = true;
    }
  }
  if (nc > 0)
    k_products_fp64_noalloc<BS><<<(unsigned)nc, 128, smem, s>>>(seg, ta, tb, nc, na, nb, a, b, c,
                                                               flags, err);
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
  int dev = 0;
  BSM_TRY(scratch_for_current_device(&scratch, &dev));
  int32_t *flags = scratch;
  unsigned *err = (unsigned *)(scratch + BSM_NOALLOC_MAX_CBLOCKS);
  cudaStream_t s = (cudaStream_t)stream;
  BSM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));  // must start at zero every call
  bsm_status st = BSM_OK;
  switch (bs) {
    case 16: st = launch<16>(dev, nc, seg, ta, tb, a_vals, na, b_vals, nb, c_vals, flags, err, s); break;
    case 32: st = launch<32>(dev, nc, seg, ta, tb, a_vals, na, b_vals, nb, c_vals, flags, err, s); break;
    default: st = launch<64>(dev, nc, seg, ta, tb, a_vals, na, b_vals, nb, c_vals, flags, err, s); break;
  }
  if (st != BSM_OK) return st;
  k_count_flags_noalloc<<<1, 1024, 0, s>>>(flags, nc, err, nnz_out);
  return cuda_status(cudaGetLastError());
}
