// Peak probes: the rates that bound this library's kernels, measured on the
// device they run on (the paper has no counterpart; they give the roofline
// denominators that no vendor table states for this chip).
//
//   bsm_probe_fp64     FP64 tensor-core MMA (mma.sync f64, four shapes) and
//                      DFMA, register operands, every SM busy, many
//                      independent accumulator chains per warp
//   bsm_probe_tcgen05  tcgen05.mma kind::f16 (BF16) / kind::f8f6f4 (E4M3),
//                      M = 128, a given N, operands in shared memory in the
//                      layout of the split kernel, FP32 accumulators in TMEM,
//                      issued back to back by one thread per SM
//   bsm_probe_bulk_copy  1-D bulk copies (cp.async.bulk) streaming a buffer
//                      from HBM into a shared-memory ring, every SM
//
// Each call runs one launch, times it with CUDA events on the caller's stream
// and returns the work done (flops or bytes) and the time.  Every mbarrier
// wait is bounded; a wait that gives up makes the call return TIMEOUT.
#include "../../include/bsm_probe.h"
#include "bsm_ptx.cuh"

namespace {

constexpr int kChains = 8;  // independent accumulators per thread

template <int SHAPE>
struct Dmma;
// m8n8k4: A 1, B 1, C 2 registers per thread; 512 flops per warp instruction
template <>
struct Dmma<0> {
  static constexpr int NA = 1, NB = 1, NC = 2, FLOPS = 2 * 8 * 8 * 4;
  __device__ static void mma(double (&c)[NC], const double (&a)[NA], const double (&b)[NB]) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a[0]), "d"(b[0]));
  }
};
// m16n8k4: A 2, B 1, C 4
template <>
struct Dmma<1> {
  static constexpr int NA = 2, NB = 1, NC = 4, FLOPS = 2 * 16 * 8 * 4;
  __device__ static void mma(double (&c)[NC], const double (&a)[NA], const double (&b)[NB]) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(b[0]));
  }
};
// m16n8k8: A 4, B 2, C 4
template <>
struct Dmma<2> {
  static constexpr int NA = 4, NB = 2, NC = 4, FLOPS = 2 * 16 * 8 * 8;
  __device__ static void mma(double (&c)[NC], const double (&a)[NA], const double (&b)[NB]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
  }
};
// m16n8k16: A 8, B 4, C 4
template <>
struct Dmma<3> {
  static constexpr int NA = 8, NB = 4, NC = 4, FLOPS = 2 * 16 * 8 * 16;
  __device__ static void mma(double (&c)[NC], const double (&a)[NA], const double (&b)[NB]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]),
          "d"(a[7]), "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
};

// Operands come from memory (so nothing folds), values small enough that the
// accumulators stay finite; the sums are written out so nothing is dropped.
template <int SHAPE>
__global__ void __launch_bounds__(256) k_probe_dmma(const double *__restrict__ in, int64_t iters,
                                                    double *__restrict__ out) {
  using D = Dmma<SHAPE>;
  const int lane = threadIdx.x & 31;
  double a[D::NA], b[D::NB], c[kChains][D::NC];
#pragma unroll
  for (int i = 0; i < D::NA; i++) a[i] = in[(lane + i) & 31];
#pragma unroll
  for (int i = 0; i < D::NB; i++) b[i] = in[32 + ((lane + i) & 31)];
#pragma unroll
  for (int q = 0; q < kChains; q++)
#pragma unroll
    for (int i = 0; i < D::NC; i++) c[q][i] = 0.0;
  for (int64_t it = 0; it < iters; it++) {
#pragma unroll
    for (int q = 0; q < kChains; q++) D::mma(c[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; q++)
#pragma unroll
    for (int i = 0; i < D::NC; i++) s += c[q][i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_dfma(const double *__restrict__ in, int64_t iters,
                                                    double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const double x = in[lane], y = in[32 + lane];
  double c[kChains];
#pragma unroll
  for (int q = 0; q < kChains; q++) c[q] = in[q];
  for (int64_t it = 0; it < iters; it++) {
#pragma unroll
    for (int q = 0; q < kChains; q++) c[q] = fma(x, c[q], y);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; q++) s += c[q];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Even warps DMMA m8n8k4, odd warps DFMA (`ratio` DFMA rounds per DMMA
// round): whether the two share one FP64 pipe.
__global__ void __launch_bounds__(256) k_probe_mixed(const double *__restrict__ in, int64_t iters,
                                                     int ratio, double *__restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s = 0.0;
  if ((warp & 1) == 0) {
    double a[1] = {in[lane]}, b[1] = {in[32 + lane]}, c[kChains][2];
#pragma unroll
    for (int q = 0; q < kChains; q++) c[q][0] = c[q][1] = 0.0;
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
      for (int q = 0; q < kChains; q++) Dmma<0>::mma(c[q], a, b);
    }
#pragma unroll
    for (int q = 0; q < kChains; q++) s += c[q][0] + c[q][1];
  } else {
    const double x = in[lane], y = in[32 + lane];
    double c[kChains];
#pragma unroll
    for (int q = 0; q < kChains; q++) c[q] = in[q];
    for (int64_t it = 0; it < iters * ratio; it++) {
#pragma unroll
      for (int q = 0; q < kChains; q++) c[q] = fma(x, c[q], y);
    }
#pragma unroll
    for (int q = 0; q < kChains; q++) s += c[q];
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One CTA per SM: warp 0 allocates TMEM; thread 0 issues `iters` groups of
// four MMAs (M = 128, N = n) alternating between two accumulators, then
// commits and waits (bounded) for the tensor core to finish.
template <int F>
__global__ void __launch_bounds__(128, 1) k_probe_tc(int n, int tiles, int issuers, int64_t iters,
                                                    unsigned *err) {
  // `tiles` operand pairs: A tile t at t * 4 KiB, B tile t after all A tiles
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar[4];
  __shared__ uint32_t tbase_sh;
  // small integer operands, as the split kernel's digits: the bytes 0x40
  // read as BF16 (0x4040) are 3.0, read as E4M3 2.0
  const uint32_t word = 0x40404040u;
  const int bytes = tiles * (4096 + n * 32);
  for (int i = threadIdx.x; i < bytes / 4; i += blockDim.x)
    reinterpret_cast<uint32_t *>(smem)[i] = word;
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int w = 0; w < 4; w++) mbar_init(&bar[w], 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tmem_alloc(&tbase_sh, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_sh;
  const int wi = threadIdx.x >> 5;  // issuing warps 0 .. issuers-1, lane 0 each
  if ((threadIdx.x & 31) == 0 && wi < issuers) {
    // K-major, no swizzle: core matrices of 8 rows x 16 bytes, the two along
    // K 128 bytes apart, 8-row groups 256 bytes apart
    const uint32_t sa = smem_u32(smem);
    const uint64_t ad = smem_desc(sa, 128, 256);
    const uint64_t bd = smem_desc(sa + tiles * 4096, 128, 256);
    const uint32_t idesc = F == 0 ? idesc_bf16_f32(128, n) : idesc_e4m3_f32(128, n);
    if (tiles == 1) {  // one operand pair: nothing computed between instructions
      for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const uint32_t d = tbase + (uint32_t)((2 * wi + (u & 1)) * n);
          const uint32_t acc = (it > 0 || u > 1) ? 1u : 0u;
          if (F == 0)
            tc_mma_bf16(d, ad, bd, idesc, acc);
          else
            tc_mma_f8(d, ad, bd, idesc, acc);
        }
      }
    } else {
      int t = 0;
      for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const uint32_t d = tbase + (uint32_t)((2 * wi + (u & 1)) * n);
          const uint32_t acc = (it > 0 || u > 1) ? 1u : 0u;
          // descriptor start addresses are in 16-byte units
          const uint64_t at = ad + (uint64_t)(t * 256), bt = bd + (uint64_t)(t * n * 2);
          if (F == 0)
            tc_mma_bf16(d, at, bt, idesc, acc);
          else
            tc_mma_f8(d, at, bt, idesc, acc);
          t = t + 1 == tiles ? 0 : t + 1;
        }
      }
    }
    tc_commit(&bar[wi]);
    if (!mbar_wait(&bar[wi], 0)) set_err(err, DERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// CTA b streams chunks b, b + grid, b + 2 grid, ... of `stage` bytes through a
// ring of `nst` shared-memory stages (thread 0 issues, and re-issues a stage
// once its previous copy has landed).
__global__ void __launch_bounds__(32, 1) k_probe_bulk(const uint8_t *__restrict__ src,
                                                      int64_t nchunks, int stage, int nst,
                                                      unsigned *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[8];
  if (threadIdx.x != 0) return;
  for (int s = 0; s < nst; s++) mbar_init(&full[s], 1);
  fence_mbar_init();
  int64_t j = 0;  // copies issued
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, j++) {
    const int s = (int)(j % nst);
    if (j >= nst && !mbar_wait(&full[s], (uint32_t)((j / nst - 1) & 1))) {
      set_err(err, DERR_TIMEOUT);
      break;
    }
    mbar_expect_tx(&full[s], (uint32_t)stage);
    bulk_g2s(smem + (size_t)s * stage, src + ch * (int64_t)stage, (uint32_t)stage, &full[s]);
  }
  // the last copy of every stage lands before the CTA exits (also after a
  // timeout: shared memory must not be released under a copy in flight)
  for (int64_t k = (j > nst ? j - nst : 0); k < j; k++) {
    const int s = (int)(k % nst);
    if (!mbar_wait(&full[s], (uint32_t)((k / nst) & 1))) set_err(err, DERR_TIMEOUT);
  }
}

struct Timed {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Timed() {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  ~Timed() {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
};

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Launches `launch` between two events, waits, and reads the error word.
template <typename L>
bsm_status timed_launch(L launch, unsigned *err, float *ms, cudaStream_t s) {
  Timed t;
  cudaEventRecord(t.e0, s);
  launch();
  cudaEventRecord(t.e1, s);
  BSM_CUDA(cudaGetLastError());
  BSM_CUDA(cudaEventSynchronize(t.e1));
  BSM_CUDA(cudaEventElapsedTime(ms, t.e0, t.e1));
  if (err) {
    unsigned h = 0;
    BSM_CUDA(cudaMemcpy(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h == DERR_TIMEOUT) return BSM_ERR_TIMEOUT;
    if (h != DERR_NONE) return BSM_ERR_CUDA;
  }
  return BSM_OK;
}

template <typename K>
int64_t fp64_grid(K kernel) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0);
  return (int64_t)sm_count() * (occ > 0 ? occ : 1);
}

}  // namespace

extern "C" bsm_status bsm_probe_fp64(int kind, int64_t iters, double *flops, float *ms,
                                     void *stream) {
  if (kind < BSM_PROBE_DMMA_M8N8K4 || kind > BSM_PROBE_MIXED || iters < 1 || !flops || !ms)
    return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double *in = nullptr, *out = nullptr;
  BSM_TRY(dev_alloc((void **)&in, 64 * sizeof(double), s));
  double h[64];
  for (int i = 0; i < 64; i++) h[i] = (i < 32 ? 1e-3 : 1e-9) * (1 + (i % 5));
  bsm_status st = cuda_status(cudaMemcpyAsync(in, h, sizeof(h), cudaMemcpyHostToDevice, s));
  int64_t grid = 0, per_thread = 0;
  switch (kind) {
    case BSM_PROBE_DMMA_M8N8K4: grid = fp64_grid(k_probe_dmma<0>); per_thread = Dmma<0>::FLOPS / 32; break;
    case BSM_PROBE_DMMA_M16N8K4: grid = fp64_grid(k_probe_dmma<1>); per_thread = Dmma<1>::FLOPS / 32; break;
    case BSM_PROBE_DMMA_M16N8K8: grid = fp64_grid(k_probe_dmma<2>); per_thread = Dmma<2>::FLOPS / 32; break;
    case BSM_PROBE_DMMA_M16N8K16: grid = fp64_grid(k_probe_dmma<3>); per_thread = Dmma<3>::FLOPS / 32; break;
    case BSM_PROBE_DFMA: grid = fp64_grid(k_probe_dfma); per_thread = 2; break;
    default: grid = fp64_grid(k_probe_mixed); break;
  }
  constexpr int kRatio = 8;  // DFMA rounds per DMMA round in the mixed probe
  if (st == BSM_OK) st = dev_alloc((void **)&out, (size_t)grid * 256 * sizeof(double), s);
  if (st == BSM_OK) {
    count_launch();
    st = timed_launch(
        [&] {
          switch (kind) {
            case BSM_PROBE_DMMA_M8N8K4: k_probe_dmma<0><<<(unsigned)grid, 256, 0, s>>>(in, iters, out); break;
            case BSM_PROBE_DMMA_M16N8K4: k_probe_dmma<1><<<(unsigned)grid, 256, 0, s>>>(in, iters, out); break;
            case BSM_PROBE_DMMA_M16N8K8: k_probe_dmma<2><<<(unsigned)grid, 256, 0, s>>>(in, iters, out); break;
            case BSM_PROBE_DMMA_M16N8K16: k_probe_dmma<3><<<(unsigned)grid, 256, 0, s>>>(in, iters, out); break;
            case BSM_PROBE_DFMA: k_probe_dfma<<<(unsigned)grid, 256, 0, s>>>(in, iters, out); break;
            default: k_probe_mixed<<<(unsigned)grid, 256, 0, s>>>(in, iters, kRatio, out); break;
          }
        },
        nullptr, ms, s);
  }
  *flops = kind == BSM_PROBE_MIXED
               ? (double)grid * 128 * (double)iters * kChains * (Dmma<0>::FLOPS / 32 + 2.0 * kRatio)
               : (double)grid * 256 * (double)iters * kChains * (double)per_thread;
  dev_free(out, s);
  dev_free(in, s);
  return st;
}

extern "C" bsm_status bsm_probe_tcgen05(int fmt, int n, int tiles, int issuers, int64_t iters,
                                        double *flops, float *ms, void *stream) {
  if ((fmt != 0 && fmt != 1) || n < 16 || n > 256 || n % 16 || tiles < 1 || tiles > 8 ||
      issuers < 1 || issuers > 4 || 2 * issuers * n > 512 || iters < 1 || !flops || !ms)
    return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // more shared memory than two CTAs could share: one CTA (one issuing
  // thread, 512 TMEM columns) per SM
  const int smem = 120 * 1024;
  auto kern = fmt == 0 ? k_probe_tc<0> : k_probe_tc<1>;
  BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  unsigned *err = nullptr;
  BSM_TRY(dev_alloc((void **)&err, sizeof(unsigned), s));
  cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  const int grid = sm_count();
  count_launch();
  bsm_status st =
      timed_launch([&] { kern<<<grid, 128, smem, s>>>(n, tiles, issuers, iters, err); }, err, ms,
                   s);
  const double k = fmt == 0 ? 16 : 32;
  *flops = (double)grid * issuers * (double)iters * 4 * 2.0 * 128 * n * k;
  dev_free(err, s);
  return st;
}

extern "C" bsm_status bsm_probe_bulk_copy(int64_t bytes, int stage_bytes, int stages,
                                          double *bytes_moved, float *ms, void *stream) {
  if (stage_bytes < 1024 || stage_bytes % 16 || stages < 2 || stages > 8 ||
      (int64_t)stage_bytes * stages > 200 * 1024 || bytes < stage_bytes || !bytes_moved || !ms)
    return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nch = bytes / stage_bytes;
  uint8_t *src = nullptr;
  unsigned *err = nullptr;
  BSM_TRY(dev_alloc((void **)&src, (size_t)nch * stage_bytes, s));
  bsm_status st = dev_alloc((void **)&err, sizeof(unsigned), s);
  if (st == BSM_OK) {
    cudaMemsetAsync(src, 1, (size_t)nch * stage_bytes, s);
    cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    const int smem = stage_bytes * stages;
    st = cuda_status(cudaFuncSetAttribute(k_probe_bulk,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = sm_count();
    count_launch();
    if (st == BSM_OK)
      st = timed_launch([&] { k_probe_bulk<<<grid, 32, smem, s>>>(src, nch, stage_bytes, stages, err); },
                        err, ms, s);
  }
  *bytes_moved = (double)nch * stage_bytes;
  dev_free(err, s);
  dev_free(src, s);
  return st;
}
