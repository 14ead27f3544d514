// Diagnostic: exercises the bounded-wait path of the kernels on the GPU.
//
// Every mbarrier wait in this library gives up after a time limit, records
// DERR_TIMEOUT in the launch's error word and unwinds, so that a lost arrival
// becomes BSM_ERR_TIMEOUT on the host instead of a hung GPU.  This entry point
// runs one CTA that waits on a barrier nothing will ever complete, with a
// caller-chosen limit, and reports what the host reads back.
#include "bsm_ptx.cuh"

namespace {

__global__ void k_wait_probe(uint64_t limit_ns, unsigned *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival that never comes
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = mbar_try_wait(&bar, 0);
    const uint64_t t0 = globaltimer_ns();
    while (!done && globaltimer_ns() - t0 <= limit_ns) done = mbar_try_wait(&bar, 0);
    if (!done) set_err(err, DERR_TIMEOUT);
  }
}

}  // namespace

extern "C" bsm_status bsm_selftest_wait_timeout(int limit_ms, void *stream) {
  if (limit_ms < 1 || limit_ms > 5000) return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned *err = nullptr;
  BSM_TRY(dev_alloc((void **)&err, sizeof(unsigned), s));
  cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  count_launch();
  k_wait_probe<<<1, 32, 0, s>>>((uint64_t)limit_ms * 1000000ull, err);
  unsigned *h = (unsigned *)host_scratch().get(16);
  bsm_status st = h ? cuda_status(cudaGetLastError()) : BSM_ERR_OOM;
  if (st == BSM_OK) {
    readback(h, err, sizeof(unsigned), s);
    st = cuda_status(cudaStreamSynchronize(s));
  }
  dev_free(err, s);
  if (st != BSM_OK) return st;
  return h[0] == DERR_TIMEOUT ? BSM_ERR_TIMEOUT : (h[0] == DERR_NONE ? BSM_OK : BSM_ERR_CUDA);
}
