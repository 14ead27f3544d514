// Transposition and addition of quadtree matrices.
//
// C = A + B is Algorithm 2: where both operands have a block the blocks are
// added (the leaf add), where only one has it that block is taken (the
// fallback), NIL where neither has one.  On the Morton-ordered key lists this
// is a merge: concatenate, sort, and add runs of equal keys; sums that come
// out exactly zero are dropped (zero blocks are never stored).
// A^T is A with every key's row and column bits swapped and every block
// transposed; with it the transposed products of Sec. 3.2 (A^T B, A B^T,
// A^T B^T) are ordinary products.
#include "bsm_internal.cuh"

namespace {

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ uint64_t swap_rowcol(uint64_t k) {
  return ((k & 0x5555555555555555ull) << 1) | ((k >> 1) & 0x5555555555555555ull);
}

constexpr uint32_t kTransFlag = 0x80000000u;

__global__ void k_transpose_keys(const uint64_t *__restrict__ keys, int64_t n,
                                 uint64_t *__restrict__ tk, int32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  tk[i] = swap_rowcol(keys[i]);
  idx[i] = (int32_t)((uint32_t)i | kTransFlag);
}

// dst[t] = src[idx[t]] (transposed when the flag bit is set), one CTA per
// block at a time, through a padded shared-memory tile.
__global__ void k_gather_blocks_t(const double *__restrict__ src, const int32_t *__restrict__ idx,
                                  double *__restrict__ dst, int64_t n, int bs) {
  extern __shared__ double tile[];  // bs x (bs+1)
  for (int64_t t = blockIdx.x; t < n; t += gridDim.x) {
    const uint32_t id = (uint32_t)idx[t];
    const bool tr = id & kTransFlag;
    const double *s = src + (int64_t)(id & ~kTransFlag) * bs * bs;
    double *d = dst + t * (int64_t)bs * bs;
    if (!tr) {
      for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) d[e] = s[e];
      continue;  // uniform over the CTA: no barrier is skipped by part of it
    }
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) tile[(e / bs) * (bs + 1) + e % bs] = s[e];
    __syncthreads();
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) d[e] = tile[(e % bs) * (bs + 1) + e / bs];
    __syncthreads();
  }
}

// Merge of two sorted key lists: (key, source index with operand in bit 31).
__global__ void k_add_tag(const uint64_t *__restrict__ ka, int64_t na,
                          const uint64_t *__restrict__ kb, int64_t nb, uint64_t *__restrict__ keys,
                          uint32_t *__restrict__ src) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < na) {
    keys[i] = ka[i];
    src[i] = (uint32_t)i;
  } else if (i < na + nb) {
    keys[i] = kb[i - na];
    src[i] = (uint32_t)(i - na) | 0x80000000u;
  }
}

// Heads of runs of equal keys in the sorted list.
__global__ void k_add_heads(const uint64_t *__restrict__ keys, int64_t n, int32_t *__restrict__ head) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = i == 0 || keys[i] != keys[i - 1];
}

// One CTA per output block: sum of the one or two source blocks; nonzero flag.
__global__ void k_add_blocks(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ src,
                             const int32_t *__restrict__ head, const int32_t *__restrict__ hpos,
                             int64_t n, const double *__restrict__ av, const double *__restrict__ bv,
                             int bs, uint64_t *__restrict__ okeys, double *__restrict__ ovals,
                             int32_t *__restrict__ nz) {
  int64_t i = blockIdx.x;
  if (i >= n || !head[i]) return;
  const int32_t o = hpos[i];
  const bool two = (i + 1 < n) && keys[i + 1] == keys[i];
  auto blk = [&](uint32_t s) {
    return (s & 0x80000000u) ? bv + (int64_t)(s & 0x7FFFFFFFu) * bs * bs : av + (int64_t)s * bs * bs;
  };
  const double *x = blk(src[i]);
  const double *y = two ? blk(src[i + 1]) : nullptr;
  double *d = ovals + (int64_t)o * bs * bs;
  bool any = false;
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    double v = two ? x[e] + y[e] : x[e];
    d[e] = v;
    any |= nonzero_f64(v);
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    okeys[o] = keys[i];
    nz[o] = any;
  }
}

__global__ void k_compact_flagged(const int32_t *__restrict__ nz, const int32_t *__restrict__ pos,
                                  int64_t n, const uint64_t *__restrict__ keys,
                                  uint64_t *__restrict__ okeys, int32_t *__restrict__ idx) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || !nz[c]) return;
  okeys[pos[c]] = keys[c];
  idx[pos[c]] = (int32_t)c;
}

}  // namespace

void launch_gather_blocks_t(const double *src, const int32_t *idx, double *dst, int64_t n, int bs,
                            cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  const int64_t grid = n < 152 * 16 ? n : 152 * 16;
  k_gather_blocks_t<<<(unsigned)grid, 256, sizeof(double) * bs * (bs + 1), s>>>(src, idx, dst, n,
                                                                                  bs);
}

extern "C" bsm_status bsm_transpose(bsm_matrix M, bsm_matrix *out, void *stream) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!M) return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int bs = M->bs;
  const int64_t n = M->nblk;
  bsm_matrix T = new_matrix_shell(M->ncols, M->nrows, bs, M->L);
  bsm_status st = BSM_OK;
  uint64_t *tk = nullptr;
  int32_t *idx = nullptr, *sidx = nullptr;
  auto owned_alloc = [&](void **p, size_t bytes) {
    bsm_status r = dev_alloc(p, bytes, s);
    if (r == BSM_OK) T->owned.push_back(*p);
    return r;
  };
  if (n > 0 &&
      (st = dev_alloc((void **)&tk, 8 * n, s)) == BSM_OK &&
      (st = dev_alloc((void **)&idx, 4 * n, s)) == BSM_OK &&
      (st = dev_alloc((void **)&sidx, 4 * n, s)) == BSM_OK &&
      (st = owned_alloc((void **)&T->keys, 8 * n)) == BSM_OK &&
      (st = owned_alloc((void **)&T->vals, sizeof(double) * bs * bs * n)) == BSM_OK) {
    count_launch();
    k_transpose_keys<<<grid_for(n, 256), 256, 0, s>>>(M->keys, n, tk, idx);
    st = sort_keys_u64(tk, T->keys, idx, sidx, n, 2 * M->L, s);
    if (st == BSM_OK) {
      launch_gather_blocks_t(M->vals, sidx, T->vals, n, bs, s);
      st = cuda_status(cudaGetLastError());
    }
  }
  dev_free(tk, s);
  dev_free(idx, s);
  dev_free(sidx, s);
  T->nblk = n;
  if (st == BSM_OK) st = build_levels(T, s);
  if (st != BSM_OK) {
    free_matrix_shell(T, s);
    return st;
  }
  *out = T;
  return BSM_OK;
}

extern "C" bsm_status bsm_add(bsm_matrix A, bsm_matrix B, bsm_matrix *out, void *stream) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || !B) return BSM_ERR_INVALID_ARG;
  if (A->nrows != B->nrows || A->ncols != B->ncols) return BSM_ERR_DIM_MISMATCH;
  if (A->bs != B->bs) return BSM_ERR_BLOCKSIZE;
  if (A->nblk + B->nblk > 0x7FFFFFFF) return BSM_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int bs = A->bs;
  const int64_t n = A->nblk + B->nblk;
  bsm_matrix C = new_matrix_shell(A->nrows, A->ncols, bs, A->L > B->L ? A->L : B->L);
  bsm_status st = BSM_OK;
  uint64_t *k0 = nullptr, *k1 = nullptr, *sk = nullptr;
  uint32_t *s0 = nullptr, *s1 = nullptr;
  int32_t *head = nullptr, *hpos = nullptr, *nz = nullptr, *pos = nullptr, *idx = nullptr;
  double *sums = nullptr;
  auto cleanup = [&]() {
    for (void *p : {(void *)k0, (void *)k1, (void *)sk, (void *)s0, (void *)s1, (void *)head,
                    (void *)hpos, (void *)nz, (void *)pos, (void *)idx, (void *)sums})
      dev_free(p, s);
  };
  int64_t nu = 0, nkeep = 0;
  if (n > 0) {
    if ((st = dev_alloc((void **)&k0, 8 * n, s)) || (st = dev_alloc((void **)&k1, 8 * n, s)) ||
        (st = dev_alloc((void **)&s0, 4 * n, s)) || (st = dev_alloc((void **)&s1, 4 * n, s)) ||
        (st = dev_alloc((void **)&head, 4 * n, s)) || (st = dev_alloc((void **)&hpos, 4 * n, s))) {
      cleanup();
      free_matrix_shell(C, s);
      return st;
    }
    count_launch(2);
    k_add_tag<<<grid_for(n, 256), 256, 0, s>>>(A->keys, A->nblk, B->keys, B->nblk, k0, s0);
    st = sort_keys_u64(k0, k1, reinterpret_cast<int32_t *>(s0), reinterpret_cast<int32_t *>(s1), n,
                       2 * C->L, s);
    if (st == BSM_OK) {
      k_add_heads<<<grid_for(n, 256), 256, 0, s>>>(k1, n, head);
      st = scan_exclusive_i32(head, hpos, n, s);
    }
    int32_t *h = (int32_t *)host_scratch().get(16);
    if (st == BSM_OK && !h) st = BSM_ERR_OOM;
    if (st == BSM_OK) {
      readback(h, hpos + n - 1, 4, s);
      readback(h + 1, head + n - 1, 4, s);
      st = cuda_status(cudaStreamSynchronize(s));
      nu = (int64_t)h[0] + h[1];
    }
    if (st == BSM_OK && (st = dev_alloc((void **)&sk, 8 * nu, s)) == BSM_OK &&
        (st = dev_alloc((void **)&sums, sizeof(double) * bs * bs * nu, s)) == BSM_OK &&
        (st = dev_alloc((void **)&nz, 4 * nu, s)) == BSM_OK &&
        (st = dev_alloc((void **)&pos, 4 * nu, s)) == BSM_OK) {
      count_launch();
      k_add_blocks<<<(unsigned)n, 128, 0, s>>>(k1, s1, head, hpos, n, A->vals, B->vals, bs, sk,
                                                sums, nz);
      st = scan_exclusive_i32(nz, pos, nu, s);
    }
    if (st == BSM_OK) {
      readback(h, pos + nu - 1, 4, s);
      readback(h + 1, nz + nu - 1, 4, s);
      st = cuda_status(cudaStreamSynchronize(s));
      nkeep = (int64_t)h[0] + h[1];
    }
    if (st == BSM_OK && nkeep == nu) {
      C->keys = sk;
      C->vals = sums;
      sk = nullptr;
      sums = nullptr;
    } else if (st == BSM_OK && nkeep > 0) {
      if ((st = dev_alloc((void **)&C->keys, 8 * nkeep, s)) == BSM_OK &&
          (st = dev_alloc((void **)&C->vals, sizeof(double) * bs * bs * nkeep, s)) == BSM_OK &&
          (st = dev_alloc((void **)&idx, 4 * nkeep, s)) == BSM_OK) {
        count_launch();
        k_compact_flagged<<<grid_for(nu, 256), 256, 0, s>>>(nz, pos, nu, sk, C->keys, idx);
        launch_gather_blocks(sums, idx, C->vals, nkeep, bs, s);
      }
    }
    if (C->keys) C->owned.push_back(C->keys);
    if (C->vals) C->owned.push_back(C->vals);
  }
  cleanup();
  C->nblk = st == BSM_OK ? nkeep : 0;
  if (st == BSM_OK) st = build_levels(C, s);
  if (st != BSM_OK) {
    free_matrix_shell(C, s);
    return st;
  }
  *out = C;
  return BSM_OK;
}

// ------------------------------------------------------------- re-blocking
// A matrix re-cut into leaf blocks of another side (16, 32 or 64; the ratio is
// a power of two).  Splitting a block of side bs into f x f blocks of side
// bs/f: the sub-block (i, j) of block (I, J) is block (I f + i, J f + j), whose
// Morton key is key(I, J) << 2 log2 f | key(i, j); taking the sub-blocks of
// each block in Morton order keeps the list sorted, and all-zero sub-blocks
// are dropped.  Merging f x f blocks into one: block (I, J) goes to
// (I / f, J / f), key >> 2 log2 f, and the f^2 children of one merged block
// are contiguous in Morton order; absent children are zero.
namespace {

// flag[t f^2 + q] = 1 if sub-block q (Morton index) of block t is kept: it
// has an entry != 0 (mode 0), it lies inside the matrix (mode 1), or it has an
// entry != 0 and lies on or above the diagonal (mode 2).  One warp per
// sub-block.
__global__ void k_split_flags(const double *__restrict__ vals, const uint64_t *__restrict__ keys,
                              int64_t n, int bs, int nbs, int keep_all, int64_t mb, int64_t nb,
                              int32_t *__restrict__ flag) {
  const int f = bs / nbs, f2 = f * f;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n * f2) return;
  const int64_t t = w / f2;
  const int q = (int)(w % f2);
  const int i = (int)morton_compact((uint64_t)q >> 1), j = (int)morton_compact((uint64_t)q);
  const int64_t I = (int64_t)morton_compact(keys[t] >> 1) * f + i;
  const int64_t J = (int64_t)morton_compact(keys[t]) * f + j;
  if (keep_all == 1) {
    if (lane == 0) flag[w] = I < mb && J < nb;
    return;
  }
  const double *b = vals + t * bs * bs + (int64_t)(i * nbs) * bs + j * nbs;
  bool any = false;
  for (int e = lane; e < nbs * nbs; e += 32) any |= nonzero_f64(b[(e / nbs) * bs + e % nbs]);
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) flag[w] = any && (keep_all != 2 || I <= J);
}

__global__ void k_split_keys(const uint64_t *__restrict__ keys, int64_t n, int f,
                             const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                             uint64_t *__restrict__ okeys, int32_t *__restrict__ map) {
  const int f2 = f * f, sh = 2 * (31 - __clz(f));
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n * f2 || !flag[w]) return;
  okeys[pos[w]] = (keys[w / f2] << sh) | (uint64_t)(w % f2);
  map[pos[w]] = (int32_t)w;
}

// dst[o] = sub-block map[o] % f^2 of block map[o] / f^2 (one CTA per block).
__global__ void k_split_gather(const double *__restrict__ src, const int32_t *__restrict__ map,
                               int64_t nout, int bs, int nbs, double *__restrict__ dst) {
  const int f = bs / nbs, f2 = f * f;
  for (int64_t o = blockIdx.x; o < nout; o += gridDim.x) {
    const int64_t w = map[o];
    const int q = (int)(w % f2);
    const int i = (int)morton_compact((uint64_t)q >> 1), j = (int)morton_compact((uint64_t)q);
    const double *b = src + (w / f2) * bs * bs + (int64_t)(i * nbs) * bs + j * nbs;
    double *d = dst + o * nbs * nbs;
    for (int e = threadIdx.x; e < nbs * nbs; e += blockDim.x) d[e] = b[(e / nbs) * bs + e % nbs];
  }
}

__global__ void k_merge_heads(const uint64_t *__restrict__ keys, int64_t n, int sh,
                              int32_t *__restrict__ head) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  head[t] = t == 0 || (keys[t] >> sh) != (keys[t - 1] >> sh);
}

__global__ void k_merge_keys(const uint64_t *__restrict__ keys, int64_t n, int sh,
                             const int32_t *__restrict__ head, const int32_t *__restrict__ hpos,
                             uint64_t *__restrict__ okeys, int32_t *__restrict__ dst_of) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int32_t o = hpos[t] + head[t] - 1;  // index of this block's merged block
  dst_of[t] = o;
  if (head[t]) okeys[o] = keys[t] >> sh;
}

// Block t goes to sub-position key & (f^2 - 1) of merged block dst_of[t]
// (zero-filled beforehand).  One CTA per source block.
__global__ void k_merge_scatter(const double *__restrict__ src, const uint64_t *__restrict__ keys,
                                const int32_t *__restrict__ dst_of, int64_t n, int bs, int nbs,
                                double *__restrict__ dst) {
  const int f = nbs / bs;
  for (int64_t t = blockIdx.x; t < n; t += gridDim.x) {
    const uint64_t q = keys[t] & (uint64_t)(f * f - 1);
    const int i = (int)morton_compact(q >> 1), j = (int)morton_compact(q);
    double *d = dst + (int64_t)dst_of[t] * nbs * nbs + (int64_t)(i * bs) * nbs + j * bs;
    const double *b = src + t * bs * bs;
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) d[(e / bs) * nbs + e % bs] = b[e];
  }
}

inline unsigned grid_blocks(int64_t n) { return (unsigned)(n < 152 * 16 ? n : 152 * 16); }

}  // namespace

// Core of re-blocking.  keep_all (splitting only): 0 drops all-zero
// sub-blocks; 1 keeps every sub-block inside the matrix (the structure then
// depends only on A's structure); 2 also drops sub-blocks below the diagonal.
// map_out, if not NULL, receives the index map that reblock_refresh needs
// (caller frees).
bsm_status reblock_impl(bsm_matrix A, int bs, int keep_all, bsm_matrix *out, int32_t **map_out,
                        cudaStream_t s) {
  *out = nullptr;
  if (map_out) *map_out = nullptr;
  const int obs = A->bs;
  const int64_t n = A->nblk;
  const int64_t mb = (A->nrows + bs - 1) / bs, nb = (A->ncols + bs - 1) / bs;
  const int64_t side = mb > nb ? mb : nb;
  bsm_matrix R = new_matrix_shell(A->nrows, A->ncols, bs, ceil_log2_i64(side < 1 ? 1 : side));
  bsm_status st = BSM_OK;
  int32_t *flag = nullptr, *pos = nullptr, *map = nullptr;
  int64_t nout = 0;
  auto owned_alloc = [&](void **p, size_t bytes) {
    bsm_status r = dev_alloc(p, bytes, s);
    if (r == BSM_OK) R->owned.push_back(*p);
    return r;
  };
  int32_t *h = (int32_t *)host_scratch().get(16);
  if (!h) st = BSM_ERR_OOM;
  if (st == BSM_OK && n > 0 && bs == obs) {
    nout = n;
    if ((st = owned_alloc((void **)&R->keys, 8 * n)) == BSM_OK &&
        (st = owned_alloc((void **)&R->vals, sizeof(double) * bs * bs * n)) == BSM_OK) {
      cudaMemcpyAsync(R->keys, A->keys, 8 * n, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(R->vals, A->vals, sizeof(double) * bs * bs * n, cudaMemcpyDeviceToDevice, s);
    }
  } else if (st == BSM_OK && n > 0 && bs < obs) {
    const int f = obs / bs;
    const int64_t m = n * f * f;
    if (m > 0x7FFFFFFF) st = BSM_ERR_UNSUPPORTED;
    if (st == BSM_OK && (st = dev_alloc((void **)&flag, 4 * m, s)) == BSM_OK &&
        (st = dev_alloc((void **)&pos, 4 * m, s)) == BSM_OK) {
      count_launch();
      k_split_flags<<<grid_for(m * 32, 256), 256, 0, s>>>(A->vals, A->keys, n, obs, bs, keep_all,
                                                          mb, nb, flag);
      st = scan_exclusive_i32(flag, pos, m, s);
    }
    if (st == BSM_OK) {
      readback(h, pos + m - 1, 4, s);
      readback(h + 1, flag + m - 1, 4, s);
      st = cuda_status(cudaStreamSynchronize(s));
      nout = (int64_t)h[0] + h[1];
    }
    if (st == BSM_OK && nout > 0 && (st = owned_alloc((void **)&R->keys, 8 * nout)) == BSM_OK &&
        (st = owned_alloc((void **)&R->vals, sizeof(double) * bs * bs * nout)) == BSM_OK &&
        (st = dev_alloc((void **)&map, 4 * nout, s)) == BSM_OK) {
      count_launch(2);
      k_split_keys<<<grid_for(m, 256), 256, 0, s>>>(A->keys, n, f, flag, pos, R->keys, map);
      k_split_gather<<<grid_blocks(nout), 256, 0, s>>>(A->vals, map, nout, obs, bs, R->vals);
      st = cuda_status(cudaGetLastError());
    }
  } else if (st == BSM_OK && n > 0) {
    const int f = bs / obs;
    const int sh = 2 * (f == 2 ? 1 : 2);
    if ((st = dev_alloc((void **)&flag, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&pos, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&map, 4 * n, s)) == BSM_OK) {
      count_launch();
      k_merge_heads<<<grid_for(n, 256), 256, 0, s>>>(A->keys, n, sh, flag);
      st = scan_exclusive_i32(flag, pos, n, s);
    }
    if (st == BSM_OK) {
      readback(h, pos + n - 1, 4, s);
      readback(h + 1, flag + n - 1, 4, s);
      st = cuda_status(cudaStreamSynchronize(s));
      nout = (int64_t)h[0] + h[1];
    }
    if (st == BSM_OK && (st = owned_alloc((void **)&R->keys, 8 * nout)) == BSM_OK &&
        (st = owned_alloc((void **)&R->vals, sizeof(double) * bs * bs * nout)) == BSM_OK) {
      cudaMemsetAsync(R->vals, 0, sizeof(double) * bs * bs * nout, s);
      count_launch(2);
      k_merge_keys<<<grid_for(n, 256), 256, 0, s>>>(A->keys, n, sh, flag, pos, R->keys, map);
      k_merge_scatter<<<grid_blocks(n), 256, 0, s>>>(A->vals, A->keys, map, n, obs, bs, R->vals);
      st = cuda_status(cudaGetLastError());
    }
  }
  dev_free(flag, s);
  dev_free(pos, s);
  if (st == BSM_OK && map_out) {
    *map_out = map;
  } else {
    dev_free(map, s);
  }
  R->nblk = st == BSM_OK ? nout : 0;
  if (st == BSM_OK) st = build_levels(R, s);
  if (st != BSM_OK) {
    if (map_out && *map_out) {
      dev_free(*map_out, s);
      *map_out = nullptr;
    }
    free_matrix_shell(R, s);
    return st;
  }
  *out = R;
  return BSM_OK;
}

void reblock_refresh(bsm_matrix src, bsm_matrix dst, const int32_t *map, cudaStream_t s) {
  if (src->nblk == 0 || dst->nblk == 0) return;
  const int obs = src->bs, bs = dst->bs;
  if (obs == bs) {
    cudaMemcpyAsync(dst->vals, src->vals, sizeof(double) * bs * bs * src->nblk,
                    cudaMemcpyDeviceToDevice, s);
  } else if (bs < obs) {
    count_launch();
    k_split_gather<<<grid_blocks(dst->nblk), 256, 0, s>>>(src->vals, map, dst->nblk, obs, bs,
                                                          dst->vals);
  } else {
    cudaMemsetAsync(dst->vals, 0, sizeof(double) * bs * bs * dst->nblk, s);
    count_launch();
    k_merge_scatter<<<grid_blocks(src->nblk), 256, 0, s>>>(src->vals, src->keys, map, src->nblk,
                                                           obs, bs, dst->vals);
  }
}

extern "C" bsm_status bsm_reblock(bsm_matrix A, int bs, bsm_matrix *out, void *stream) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A) return BSM_ERR_INVALID_ARG;
  if (bs != 16 && bs != 32 && bs != 64) return BSM_ERR_BLOCKSIZE;
  return reblock_impl(A, bs, 0, out, nullptr, (cudaStream_t)stream);
}
