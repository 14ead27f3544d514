// Quadtree construction on the device: Morton keys, radix sort, zero-block
// removal, payload gather, per-level child bitmasks; block extraction.
//
// The paper's Matrix chunk (Sec. 3.1) is a node with four child ids, NIL for a
// zero submatrix at any level.  Here level h (height above the leaves) is the
// sorted array of nonzero node keys key >> 2h, each with a 4-bit mask of its
// non-NIL children (bit c = child 2*rowhalf + colhalf) and the index of its
// first child in level h-1.  Children of a node are contiguous because keys
// are in Morton order.
#include <cstring>
#include <mutex>

#include "bsm_internal.cuh"

// ------------------------------------------------------------------ kernels
// One warp per listed block: range check, key, and whether the block holds an
// entry != 0.0.  stage (or NULL): receives a copy of every block it reads (the
// values of pinned host input then cross the host link once).
__global__ void k_make_keys(const int32_t *__restrict__ brow, const int32_t *__restrict__ bcol,
                            const double *__restrict__ vals, int64_t n, int64_t mb, int64_t nb,
                            int bs, uint64_t *__restrict__ keys, int32_t *__restrict__ idx,
                            uint8_t *__restrict__ nz, unsigned *__restrict__ err,
                            double *__restrict__ stage) {
  int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  const double2 *b = reinterpret_cast<const double2 *>(vals + w * (int64_t)bs * bs);
  int n2 = bs * bs / 2;
  bool any = false;
  double2 *st = stage ? reinterpret_cast<double2 *>(stage + w * (int64_t)bs * bs) : nullptr;
  for (int t = lane; t < n2; t += 32) {
    double2 v = b[t];
    any |= nonzero_f64(v.x) | nonzero_f64(v.y);
    if (st) st[t] = v;
  }
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) {
    int64_t I = brow[w], J = bcol[w];
    if (I < 0 || I >= mb || J < 0 || J >= nb) {
      atomicCAS(err, DERR_NONE, DERR_OUT_OF_RANGE);
      I = 0;
      J = 0;
    }
    keys[w] = morton_key((uint64_t)I, (uint64_t)J);
    idx[w] = (int32_t)w;
    nz[w] = any ? 1 : 0;
  }
}

__global__ void k_dup_keep(const uint64_t *__restrict__ skeys, const int32_t *__restrict__ sidx,
                           const uint8_t *__restrict__ nz, int64_t n, int32_t *__restrict__ keep,
                           unsigned *__restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i > 0 && skeys[i] == skeys[i - 1]) atomicCAS(err, DERR_NONE, DERR_DUPLICATE);
  keep[i] = nz[sidx[i]];
}

__global__ void k_compact_keys(const uint64_t *__restrict__ skeys, const int32_t *__restrict__ sidx,
                               const int32_t *__restrict__ keep, const int32_t *__restrict__ pos,
                               int64_t n, uint64_t *__restrict__ okeys,
                               int32_t *__restrict__ oidx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  okeys[pos[i]] = skeys[i];
  oidx[pos[i]] = sidx[i];
}

// dst[t] = src[idx[t]]; each CTA copies whole blocks with 16-byte accesses.
__global__ void k_gather_blocks(const double *__restrict__ src, const int32_t *__restrict__ idx,
                                double *__restrict__ dst, int64_t n, int bs) {
  int64_t per = (int64_t)bs * bs / 2;  // double2 per block
  for (int64_t t = blockIdx.x; t < n; t += gridDim.x) {
    const double2 *s = reinterpret_cast<const double2 *>(src + (int64_t)idx[t] * bs * bs);
    double2 *d = reinterpret_cast<double2 *>(dst + t * (int64_t)bs * bs);
    for (int64_t e = threadIdx.x; e < per; e += blockDim.x) d[e] = __ldg(s + e);
  }
}

void launch_gather_blocks(const double *src, const int32_t *idx, double *dst, int64_t n, int bs,
                          cudaStream_t s, int64_t max_ctas) {
  if (n <= 0) return;
  const int64_t cap = max_ctas > 0 ? max_ctas : 152 * 32;
  int64_t grid = n < cap ? n : cap;
  count_launch();
  k_gather_blocks<<<(unsigned)grid, 256, 0, s>>>(src, idx, dst, n, bs);
}

// Level h from level h-1 (child keys K, count *nchild): heads of runs of equal
// parent key.
__global__ void k_level_heads(const uint64_t *__restrict__ K, const int64_t *__restrict__ nchild,
                              int64_t cap, int32_t *__restrict__ head) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  int64_t n = *nchild;
  head[i] = (i < n) && (i == 0 || (K[i] >> 2) != (K[i - 1] >> 2));
}

__global__ void k_level_write(const uint64_t *__restrict__ K, const int64_t *__restrict__ nchild,
                              const int32_t *__restrict__ head, const int32_t *__restrict__ hpos,
                              uint64_t *__restrict__ pkeys, uint8_t *__restrict__ pmask,
                              int32_t *__restrict__ pcstart, int64_t *__restrict__ nparent) {
  // launched over the child level's capacity; *nchild <= that capacity
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = *nchild;
  if (i >= n) return;
  if (i == n - 1) *nparent = hpos[i] + head[i];
  if (!head[i]) return;
  uint64_t pk = K[i] >> 2;
  unsigned mask = 0;
  for (int64_t j = i; j < n && j < i + 4 && (K[j] >> 2) == pk; j++) mask |= 1u << (K[j] & 3);
  int32_t p = hpos[i];
  pkeys[p] = pk;
  pmask[p] = (uint8_t)mask;
  pcstart[p] = (int32_t)i;
}

__global__ void k_rowmajor_keys(const uint64_t *__restrict__ keys, int64_t n,
                                uint64_t *__restrict__ rm, int32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k = keys[i];
  uint64_t I = morton_compact(k >> 1), J = morton_compact(k);
  rm[i] = (I << 32) | J;
  idx[i] = (int32_t)i;
}

__global__ void k_rowmajor_coords(const uint64_t *__restrict__ rm, int64_t off, int64_t n,
                                  int32_t *__restrict__ brow, int32_t *__restrict__ bcol) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k = rm[off + i];
  if (brow) brow[i] = (int32_t)(k >> 32);
  if (bcol) bcol[i] = (int32_t)(k & 0xFFFFFFFFu);
}

static inline unsigned nblocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Keys of a COO list in (I, J) -> Morton form, with range checks.
__global__ void k_coo_keys(const int32_t *__restrict__ brow, const int32_t *__restrict__ bcol,
                           int64_t n, int64_t mb, int64_t nb, uint64_t *__restrict__ keys,
                           int32_t *__restrict__ idx, unsigned *__restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t I = brow[i], J = bcol[i];
  if (I < 0 || I >= mb || J < 0 || J >= nb) {
    atomicCAS(err, DERR_NONE, DERR_OUT_OF_RANGE);
    I = 0;
    J = 0;
  }
  keys[i] = morton_key((uint64_t)I, (uint64_t)J);
  idx[i] = (int32_t)i;
}

// Sorted update keys must equal the handle's keys one for one.
__global__ void k_keys_equal(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b,
                             int64_t n, unsigned *__restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && a[i] != b[i]) atomicCAS(err, DERR_NONE, DERR_BOUNDS);
}

// --------------------------------------------------------------- host side
bsm_status build_levels(bsm_matrix M, cudaStream_t s) {
  for (int h = 0; h <= BSM_MAXH; h++) M->nlev[h] = 0;
  M->nlev[0] = M->nblk;
  if (M->nblk == 0 || M->L == 0) return BSM_OK;
  int L = M->L;
  int64_t *dcount = nullptr;  // device counts per level
  BSM_TRY(dev_alloc((void **)&dcount, sizeof(int64_t) * (L + 1), s));
  M->owned.push_back(dcount);
  BSM_CUDA(cudaMemcpyAsync(dcount, &M->nblk, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  int64_t cap_prev = M->nblk;
  int32_t *head = nullptr, *hpos = nullptr;
  BSM_TRY(dev_alloc((void **)&head, sizeof(int32_t) * cap_prev, s));
  bsm_status st = dev_alloc((void **)&hpos, sizeof(int32_t) * cap_prev, s);
  if (st != BSM_OK) {
    dev_free(head, s);
    return st;
  }
  const uint64_t *K = M->keys;
  for (int h = 1; h <= L && st == BSM_OK; h++) {
    int64_t maxnodes = (2 * (L - h) >= 62) ? INT64_MAX : ((int64_t)1 << (2 * (L - h)));
    int64_t cap = cap_prev < maxnodes ? cap_prev : maxnodes;
    void *pk = nullptr, *pm = nullptr, *pc = nullptr;
    if ((st = dev_alloc(&pk, sizeof(uint64_t) * cap, s)) != BSM_OK) break;
    M->owned.push_back(pk);
    if ((st = dev_alloc(&pm, sizeof(uint8_t) * cap, s)) != BSM_OK) break;
    M->owned.push_back(pm);
    if ((st = dev_alloc(&pc, sizeof(int32_t) * cap, s)) != BSM_OK) break;
    M->owned.push_back(pc);
    M->lkeys[h] = (uint64_t *)pk;
    M->lmask[h] = (uint8_t *)pm;
    M->lcstart[h] = (int32_t *)pc;
    count_launch();
    k_level_heads<<<nblocks_for(cap_prev, 256), 256, 0, s>>>(K, dcount + h - 1, cap_prev, head);
    if ((st = scan_exclusive_i32(head, hpos, cap_prev, s)) != BSM_OK) break;
    count_launch();
    k_level_write<<<nblocks_for(cap_prev, 256), 256, 0, s>>>(K, dcount + h - 1, head, hpos,
                                                             M->lkeys[h], M->lmask[h],
                                                             M->lcstart[h], dcount + h);
    K = M->lkeys[h];
    cap_prev = cap;
  }
  dev_free(head, s);
  dev_free(hpos, s);
  if (st != BSM_OK) return st;
  BSM_CUDA(cudaGetLastError());
  int64_t *hc = (int64_t *)host_scratch().get(sizeof(int64_t) * (L + 1));
  if (!hc) return BSM_ERR_OOM;
  BSM_TRY(readback(hc, dcount, sizeof(int64_t) * (L + 1), s));
  BSM_CUDA(cudaStreamSynchronize(s));
  for (int h = 0; h <= L; h++) M->nlev[h] = hc[h];
  return BSM_OK;
}

static void destroy_matrix(bsm_matrix M, cudaStream_t s) {
  if (!M) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != M->device) cudaSetDevice(M->device);
  for (void *p : M->owned) dev_free(p, s);
  if (cur != M->device) cudaSetDevice(cur);
  delete M;
}

static bool bs_supported(int bs) { return bs == 16 || bs == 32 || bs == 64; }

// Allocates and fills a new handle from device COO arrays.
// stage (or NULL): device buffer of nblk blocks that the key kernel fills
// with the input values, the gather's source then (for pinned host input).
static bsm_status build_from_device(int64_t nrows, int64_t ncols, int bs, int64_t nblk,
                                    const int32_t *brow, const int32_t *bcol, const double *vals,
                                    cudaStream_t s, bsm_matrix *out, double *stage = nullptr) {
  bsm_matrix M = new bsm_matrix_s();
  cudaGetDevice(&M->device);
  M->nrows = nrows;
  M->ncols = ncols;
  M->bs = bs;
  M->mb = (nrows + bs - 1) / bs;
  M->nb = (ncols + bs - 1) / bs;
  int64_t side = M->mb > M->nb ? M->mb : M->nb;
  M->L = ceil_log2_i64(side < 1 ? 1 : side);
  if (M->L > BSM_MAXH) {
    delete M;
    return BSM_ERR_INVALID_ARG;
  }
  bsm_status st = BSM_OK;
  uint64_t *keys = nullptr, *skeys = nullptr;
  int32_t *idx = nullptr, *sidx = nullptr, *keep = nullptr, *pos = nullptr;
  uint8_t *nz = nullptr;
  unsigned *err = nullptr;
  int64_t nkeep = 0;
  auto cleanup = [&]() {
    dev_free(keys, s);
    dev_free(skeys, s);
    dev_free(idx, s);
    dev_free(sidx, s);
    dev_free(keep, s);
    dev_free(pos, s);
    dev_free(nz, s);
    dev_free(err, s);
  };
  if (nblk > 0) {
    if ((st = dev_alloc((void **)&keys, 8 * nblk, s)) ||
        (st = dev_alloc((void **)&skeys, 8 * nblk, s)) ||
        (st = dev_alloc((void **)&idx, 4 * nblk, s)) ||
        (st = dev_alloc((void **)&sidx, 4 * nblk, s)) ||
        (st = dev_alloc((void **)&keep, 4 * nblk, s)) ||
        (st = dev_alloc((void **)&pos, 4 * nblk, s)) || (st = dev_alloc((void **)&nz, nblk, s)) ||
        (st = dev_alloc((void **)&err, sizeof(unsigned), s))) {
      cleanup();
      delete M;
      return st;
    }
    cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    count_launch();
    k_make_keys<<<nblocks_for(nblk, 8), 256, 0, s>>>(brow, bcol, vals, nblk, M->mb, M->nb, bs,
                                                     keys, idx, nz, err, stage);
    st = sort_keys_u64(keys, skeys, idx, sidx, nblk, 2 * M->L, s);
    if (st == BSM_OK) {
      count_launch();
      k_dup_keep<<<nblocks_for(nblk, 256), 256, 0, s>>>(skeys, sidx, nz, nblk, keep, err);
      st = scan_exclusive_i32(keep, pos, nblk, s);
    }
    if (st == BSM_OK) {
      int32_t *h = (int32_t *)host_scratch().get(16);
      if (!h) st = BSM_ERR_OOM;
      if (st == BSM_OK) {
        readback(h, pos + nblk - 1, 4, s);
        readback(h + 1, keep + nblk - 1, 4, s);
        readback(h + 2, err, 4, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e);
        unsigned derr = (unsigned)h[2];
        if (st == BSM_OK && derr == DERR_OUT_OF_RANGE) st = BSM_ERR_OUT_OF_RANGE;
        if (st == BSM_OK && derr == DERR_DUPLICATE) st = BSM_ERR_DUPLICATE;
        nkeep = (int64_t)h[0] + h[1];
      }
    }
    if (st != BSM_OK) {
      cleanup();
      delete M;
      return st;
    }
  }
  M->nblk = nkeep;
  if (nkeep > 0) {
    if ((st = dev_alloc((void **)&M->keys, 8 * nkeep, s)) == BSM_OK) M->owned.push_back(M->keys);
    if (st == BSM_OK &&
        (st = dev_alloc((void **)&M->vals, sizeof(double) * bs * bs * nkeep, s)) == BSM_OK)
      M->owned.push_back(M->vals);
    if (st == BSM_OK) {
      // reuse idx as the compacted source index
      count_launch();
      k_compact_keys<<<nblocks_for(nblk, 256), 256, 0, s>>>(skeys, sidx, keep, pos, nblk, M->keys,
                                                            idx);
      launch_gather_blocks(stage ? stage : vals, idx, M->vals, nkeep, bs, s);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_status(e);
    }
  }
  if (st == BSM_OK) st = build_levels(M, s);
  cleanup();
  if (st != BSM_OK) {
    destroy_matrix(M, s);
    return st;
  }
  *out = M;
  return BSM_OK;
}

// The device address of a pinned (page-locked, device-mapped) host buffer,
// if it has one with the given alignment; nullptr for any other pointer.
static void *mapped_device_ptr(const void *p, uintptr_t align) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return (uintptr_t)a.devicePointer % align ? nullptr : a.devicePointer;
}

extern "C" bsm_status bsm_build(int64_t nrows, int64_t ncols, int bs, int64_t nblk,
                                const int32_t *brow, const int32_t *bcol, const double *vals,
                                int on_device, void *stream, bsm_matrix *out) {
  NvtxRange range("bsm_build");
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (nrows < 0 || ncols < 0 || nblk < 0 || (on_device != 0 && on_device != 1))
    return BSM_ERR_INVALID_ARG;
  if (!bs_supported(bs)) return BSM_ERR_BLOCKSIZE;
  if (nblk > 0 && (!brow || !bcol || !vals)) return BSM_ERR_INVALID_ARG;
  if (nblk > INT32_MAX) return BSM_ERR_UNSUPPORTED;
  // device payloads are read with 16-byte vector loads
  if (on_device && nblk > 0 &&
      (((uintptr_t)vals & 15) || ((uintptr_t)brow & 3) || ((uintptr_t)bcol & 3)))
    return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (on_device || nblk == 0)
    return build_from_device(nrows, ncols, bs, nblk, brow, bcol, vals, s, out);
  // pinned host input: the key kernel reads it in place over the host link
  // (no copy-engine upload, which would queue behind other streams' copies)
  // and copies the values into a device buffer for the gather, so they cross
  // the link once; the call returns once the last read is done
  {
    const int32_t *mr = (const int32_t *)mapped_device_ptr(brow, 4);
    const int32_t *mc = (const int32_t *)mapped_device_ptr(bcol, 4);
    const double *mv = (const double *)mapped_device_ptr(vals, 16);
    if (mr && mc && mv) {
      double *stage = nullptr;
      bsm_status st = dev_alloc((void **)&stage, sizeof(double) * bs * bs * nblk, s);
      if (st != BSM_OK) return st;
      st = build_from_device(nrows, ncols, bs, nblk, mr, mc, mv, s, out, stage);
      dev_free(stage, s);
      if (st == BSM_OK) st = cuda_status(cudaStreamSynchronize(s));
      if (st != BSM_OK && *out) {
        destroy_matrix(*out, s);
        *out = nullptr;
      }
      return st;
    }
  }
  // other host input: stage on the device
  int32_t *dr = nullptr, *dc = nullptr;
  double *dv = nullptr;
  size_t vb = sizeof(double) * bs * bs * nblk;
  bsm_status st;
  if ((st = dev_alloc((void **)&dr, 4 * nblk, s)) || (st = dev_alloc((void **)&dc, 4 * nblk, s)) ||
      (st = dev_alloc((void **)&dv, vb, s))) {
    dev_free(dr, s);
    dev_free(dc, s);
    dev_free(dv, s);
    return st;
  }
  cudaMemcpyAsync(dr, brow, 4 * nblk, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dc, bcol, 4 * nblk, cudaMemcpyHostToDevice, s);
  cudaError_t e = cudaMemcpyAsync(dv, vals, vb, cudaMemcpyHostToDevice, s);
  st = cuda_status(e);
  if (st == BSM_OK) st = build_from_device(nrows, ncols, bs, nblk, dr, dc, dv, s, out);
  dev_free(dr, s);
  dev_free(dc, s);
  dev_free(dv, s);
  return st;
}

// Asynchronous downloads run on a stream of the library's own, one per
// device, at the device's greatest priority: the block scheduler then places
// the download's short gather launches ahead of the pending CTAs of a long
// kernel on another stream (a product), so the copy engine is kept fed while
// the product runs.  The caller's stream is joined both ways by one event.
struct SideStream {
  cudaStream_t caller = nullptr, side = nullptr;
  cudaEvent_t ev = nullptr;
  bsm_status fork(cudaStream_t s) {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0, lo = 0, hi = 0;
    BSM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return BSM_ERR_UNSUPPORTED;
    {
      std::lock_guard<std::mutex> g(mu);
      if (!streams[dev]) {
        BSM_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        BSM_CUDA(cudaStreamCreateWithPriority(&streams[dev], cudaStreamNonBlocking, hi));
      }
    }
    BSM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    caller = s;
    side = streams[dev];
    cudaEventRecord(ev, caller);
    cudaStreamWaitEvent(side, ev, 0);
    return BSM_OK;
  }
  // everything queued on the side stream so far precedes later work on the
  // caller's stream
  ~SideStream() {
    if (!ev) return;
    cudaEventRecord(ev, side);
    cudaStreamWaitEvent(caller, ev, 0);
    cudaEventDestroy(ev);
  }
};

// Blocks per chunk of an asynchronous download and CTAs of its gathers: one
// 512 MB staging buffer, one CTA per SM.
constexpr size_t kDownloadChunkBytes = (size_t)512 << 20;
constexpr int64_t kDownloadGatherCtas = 152;

extern "C" bsm_status bsm_to_blocks(bsm_matrix M, int64_t *nblk_inout, int32_t *brow,
                                    int32_t *bcol, double *vals, int on_device, void *stream) {
  NvtxRange range("bsm_to_blocks");
  if (!M || !nblk_inout || on_device < 0 || on_device > 2) return BSM_ERR_INVALID_ARG;
  int64_t cap = *nblk_inout;
  *nblk_inout = M->nblk;
  if (!brow && !bcol && !vals) return BSM_OK;
  if (cap < M->nblk) return BSM_ERR_BUFFER_TOO_SMALL;
  if (M->nblk == 0) return BSM_OK;
  // device outputs are written with 16-byte vector stores
  if (on_device && (((uintptr_t)vals & 15) || ((uintptr_t)brow & 3) || ((uintptr_t)bcol & 3)))
    return BSM_ERR_INVALID_ARG;
  // host output into pinned (page-locked, device-mapped) buffers: the gather
  // and coordinate kernels write straight into them over the host link, with
  // no staging copy
  auto mapped = [](void *p, uintptr_t align) -> void * { return mapped_device_ptr(p, align); };
  double *mv = nullptr;
  int32_t *mr = nullptr, *mc = nullptr;
  bool all_mapped = false;
  if (on_device != 1) {
    mv = (double *)mapped(vals, 16);
    mr = (int32_t *)mapped(brow, 4);
    mc = (int32_t *)mapped(bcol, 4);
    all_mapped = (!vals || mv) && (!brow || mr) && (!bcol || mc);
  }
  // asynchronous host output needs page-locked buffers (checked before any work)
  if (on_device == 2 && !all_mapped) return BSM_ERR_INVALID_ARG;
  const bool async_host = on_device == 2;
  cudaStream_t s = (cudaStream_t)stream;
  SideStream side;
  if (async_host) {
    BSM_TRY(side.fork(s));
    s = side.side;
  }
  int64_t n = M->nblk;
  int bs = M->bs;
  uint64_t *rm = nullptr, *rms = nullptr;
  int32_t *idx = nullptr, *sidx = nullptr;
  bsm_status st;
  auto cleanup = [&]() {
    dev_free(rm, s);
    dev_free(rms, s);
    dev_free(idx, s);
    dev_free(sidx, s);
  };
  if ((st = dev_alloc((void **)&rm, 8 * n, s)) || (st = dev_alloc((void **)&rms, 8 * n, s)) ||
      (st = dev_alloc((void **)&idx, 4 * n, s)) || (st = dev_alloc((void **)&sidx, 4 * n, s))) {
    cleanup();
    return st;
  }
  count_launch();
  k_rowmajor_keys<<<nblocks_for(n, 256), 256, 0, s>>>(M->keys, n, rm, idx);
  int endbit = 32 + ceil_log2_i64(M->nb < 1 ? 1 : M->nb) + 1;
  if (endbit > 64) endbit = 64;
  if ((st = sort_keys_u64(rm, rms, idx, sidx, n, endbit, s)) != BSM_OK) {
    cleanup();
    return st;
  }
  if (on_device == 1) {
    count_launch();
    k_rowmajor_coords<<<nblocks_for(n, 256), 256, 0, s>>>(rms, 0, n, brow, bcol);
    if (vals) launch_gather_blocks(M->vals, sidx, vals, n, bs, s);
    st = cuda_status(cudaGetLastError());
    cleanup();
    return st;
  }
  if (async_host) {
    // gather on the device in chunks through one small staging buffer, each
    // chunk followed by a copy-engine transfer into the caller's page-locked
    // buffers.  The gathers are short and narrow and the transfers hold no
    // SM, so a product on another stream runs beside the download nearly
    // undisturbed; the staging is a fixed 512 MB, not the size of the
    // output.  All ordered on the side stream; nothing waits here.
    size_t bblk = sizeof(double) * bs * bs;
    int64_t chunk = (int64_t)(kDownloadChunkBytes / bblk);
    if (chunk < 1) chunk = 1;
    if (chunk > n) chunk = n;
    double *stage = nullptr;
    int32_t *crd = nullptr;
    if ((st = dev_alloc((void **)&stage, vals ? bblk * chunk : 16, s)) ||
        (st = dev_alloc((void **)&crd, 8 * n, s))) {
      dev_free(stage, s);
      cleanup();
      return st;
    }
    count_launch();
    k_rowmajor_coords<<<nblocks_for(n, 256), 256, 0, s>>>(rms, 0, n, crd, crd + n);
    if (brow) cudaMemcpyAsync(brow, crd, 4 * n, cudaMemcpyDeviceToHost, s);
    if (bcol) cudaMemcpyAsync(bcol, crd + n, 4 * n, cudaMemcpyDeviceToHost, s);
    if (vals)
      for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        int64_t m = n - c0 < chunk ? n - c0 : chunk;
        launch_gather_blocks(M->vals, sidx + c0, stage, m, bs, s, kDownloadGatherCtas);
        cudaMemcpyAsync(vals + c0 * bs * bs, stage, bblk * m, cudaMemcpyDeviceToHost, s);
      }
    dev_free(stage, s);
    dev_free(crd, s);
    cleanup();
    return cuda_status(cudaGetLastError());
  }
  if (all_mapped) {
    if (brow || bcol) {
      count_launch();
      k_rowmajor_coords<<<nblocks_for(n, 256), 256, 0, s>>>(rms, 0, n, mr, mc);
    }
    if (vals) launch_gather_blocks(M->vals, sidx, mv, n, bs, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cleanup();
    return cuda_status(e == cudaSuccess ? cudaGetLastError() : e);
  }
  // other host output: gather through a bounded device staging buffer
  size_t bblk = sizeof(double) * bs * bs;
  int64_t chunk = (int64_t)((size_t)1 << 30) / (int64_t)bblk;
  if (chunk > n) chunk = n;
  double *stage = nullptr;
  int32_t *crd = nullptr;
  if ((st = dev_alloc((void **)&stage, bblk * chunk, s)) ||
      (st = dev_alloc((void **)&crd, 8 * n, s))) {
    dev_free(stage, s);
    cleanup();
    return st;
  }
  count_launch();
  k_rowmajor_coords<<<nblocks_for(n, 256), 256, 0, s>>>(rms, 0, n, crd, crd + n);
  if (brow) cudaMemcpyAsync(brow, crd, 4 * n, cudaMemcpyDeviceToHost, s);
  if (bcol) cudaMemcpyAsync(bcol, crd + n, 4 * n, cudaMemcpyDeviceToHost, s);
  if (vals)
    for (int64_t o = 0; o < n; o += chunk) {
      int64_t m = n - o < chunk ? n - o : chunk;
      launch_gather_blocks(M->vals, sidx + o, stage, m, bs, s);
      cudaMemcpyAsync(vals + o * bs * bs, stage, bblk * m, cudaMemcpyDeviceToHost, s);
    }
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(stage, s);
  dev_free(crd, s);
  cleanup();
  return cuda_status(e == cudaSuccess ? cudaGetLastError() : e);
}

extern "C" bsm_status bsm_update_values(bsm_matrix M, int64_t nblk, const int32_t *brow,
                                        const int32_t *bcol, const double *vals, int on_device,
                                        void *stream) {
  if (!M || nblk < 0 || (on_device != 0 && on_device != 1)) return BSM_ERR_INVALID_ARG;
  if (nblk != M->nblk) return BSM_ERR_INVALID_ARG;  // the block set must be the same
  if (nblk == 0) return BSM_OK;
  if (!brow || !bcol || !vals) return BSM_ERR_INVALID_ARG;
  if (on_device && (((uintptr_t)vals & 15) || ((uintptr_t)brow & 3) || ((uintptr_t)bcol & 3)))
    return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int bs = M->bs;
  const size_t vb = sizeof(double) * bs * bs * nblk;
  int32_t *dr = nullptr, *dc = nullptr, *idx = nullptr, *sidx = nullptr;
  double *dv = nullptr;
  uint64_t *keys = nullptr, *skeys = nullptr;
  unsigned *err = nullptr;
  bsm_status st;
  auto cleanup = [&]() {
    if (!on_device) {
      dev_free(dr, s);
      dev_free(dc, s);
      dev_free(dv, s);
    }
    dev_free(idx, s);
    dev_free(sidx, s);
    dev_free(keys, s);
    dev_free(skeys, s);
    dev_free(err, s);
  };
  if (on_device) {
    dr = const_cast<int32_t *>(brow);
    dc = const_cast<int32_t *>(bcol);
    dv = const_cast<double *>(vals);
  } else if ((st = dev_alloc((void **)&dr, 4 * nblk, s)) ||
             (st = dev_alloc((void **)&dc, 4 * nblk, s)) || (st = dev_alloc((void **)&dv, vb, s))) {
    cleanup();
    return st;
  } else {
    cudaMemcpyAsync(dr, brow, 4 * nblk, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dc, bcol, 4 * nblk, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dv, vals, vb, cudaMemcpyHostToDevice, s);
  }
  if ((st = dev_alloc((void **)&idx, 4 * nblk, s)) || (st = dev_alloc((void **)&sidx, 4 * nblk, s)) ||
      (st = dev_alloc((void **)&keys, 8 * nblk, s)) ||
      (st = dev_alloc((void **)&skeys, 8 * nblk, s)) ||
      (st = dev_alloc((void **)&err, sizeof(unsigned), s))) {
    cleanup();
    return st;
  }
  cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  count_launch();
  k_coo_keys<<<nblocks_for(nblk, 256), 256, 0, s>>>(dr, dc, nblk, M->mb, M->nb, keys, idx, err);
  st = sort_keys_u64(keys, skeys, idx, sidx, nblk, 2 * M->L, s);
  if (st == BSM_OK) {
    count_launch();
    k_keys_equal<<<nblocks_for(nblk, 256), 256, 0, s>>>(skeys, M->keys, nblk, err);
    unsigned *h = (unsigned *)host_scratch().get(16);
    if (!h) st = BSM_ERR_OOM;
    if (st == BSM_OK) {
      readback(h, err, 4, s);
      st = cuda_status(cudaStreamSynchronize(s));
    }
    if (st == BSM_OK && h[0] == DERR_OUT_OF_RANGE) st = BSM_ERR_OUT_OF_RANGE;
    if (st == BSM_OK && h[0] != DERR_NONE) st = BSM_ERR_INVALID_ARG;  // different block set
  }
  if (st == BSM_OK) {
    launch_gather_blocks(dv, sidx, M->vals, nblk, bs, s);
    st = cuda_status(cudaGetLastError());
  }
  cleanup();
  return st;
}

extern "C" bsm_status bsm_info(bsm_matrix M, int64_t *nrows, int64_t *ncols, int *bs,
                               int64_t *nblk) {
  if (!M) return BSM_ERR_INVALID_ARG;
  if (nrows) *nrows = M->nrows;
  if (ncols) *ncols = M->ncols;
  if (bs) *bs = M->bs;
  if (nblk) *nblk = M->nblk;
  return BSM_OK;
}

extern "C" bsm_status bsm_level_counts(bsm_matrix M, int64_t *counts, int cap, int *nlev) {
  if (!M || !nlev) return BSM_ERR_INVALID_ARG;
  *nlev = M->L + 1;
  if (!counts) return BSM_OK;
  if (cap < M->L + 1) return BSM_ERR_BUFFER_TOO_SMALL;
  for (int l = 0; l <= M->L; l++) counts[l] = M->nblk == 0 ? 0 : M->nlev[M->L - l];
  return BSM_OK;
}

extern "C" bsm_status bsm_destroy(bsm_matrix M) {
  if (!M) return BSM_OK;
  cudaStream_t s = 0;
  destroy_matrix(M, s);
  return BSM_OK;
}

// Creates an empty handle shell (used by the multiply to assemble C).
bsm_matrix new_matrix_shell(int64_t nrows, int64_t ncols, int bs, int L) {
  bsm_matrix M = new bsm_matrix_s();
  cudaGetDevice(&M->device);
  M->nrows = nrows;
  M->ncols = ncols;
  M->bs = bs;
  M->mb = (nrows + bs - 1) / bs;
  M->nb = (ncols + bs - 1) / bs;
  M->L = L;
  return M;
}
void free_matrix_shell(bsm_matrix M, cudaStream_t s) { destroy_matrix(M, s); }
