// Frobenius norms of quadtree nodes and norm-based truncation.
//
// The paper names per-node Frobenius norms as extra information a quadtree
// can carry (Sec. 7) and truncates its overlap matrices so that the Frobenius
// norm of the error stays below a threshold (Sec. 6.2).  Squared norms are
// summed in one fixed order, with every multiply and add rounded separately
// (no contraction), so results are reproducible bit for bit: a block's squared
// norm is the sum over its rows, in ascending order, of the row's sum of
// squares in ascending column order; a node's is the sum of its children's in
// child (= Morton) order.
//
// Truncation removes the longest run of blocks, in ascending order of squared
// norm (ties in ascending Morton key order), whose squared norms sum to at most
// tau^2.  The running sum is kept in integers so the decision is exact: with
// 2^e = 2^(floor(log2 tau^2) - 63), each squared norm s becomes
// Q = ceil(s / 2^e) (saturating) and the run ends before the prefix sum of the
// Q passes T = floor(tau^2 / 2^e); then sum(s) <= sum(Q) 2^e <= tau^2.
#include <cmath>

#include "bsm_internal.cuh"

namespace {

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// One warp per block: lane r sums rows r and r + 32 in column order, lane 0
// adds the row sums in row order.
template <int BS>
__global__ void k_block_norm2(const double *__restrict__ vals, int64_t n, double *__restrict__ out) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= n) return;  // whole warps leave together
  const double *v = vals + b * BS * BS;
  double r0 = 0.0, r1 = 0.0;
  if (lane < BS) {
    for (int c = 0; c < BS; c++) r0 = __dadd_rn(r0, __dmul_rn(v[lane * BS + c], v[lane * BS + c]));
  }
  if (BS > 32) {
    const int r = lane + 32;
    for (int c = 0; c < BS; c++) r1 = __dadd_rn(r1, __dmul_rn(v[r * BS + c], v[r * BS + c]));
  }
  double t = 0.0;
  for (int r = 0; r < BS; r++) {
    const double x = __shfl_sync(0xffffffffu, r < 32 ? r0 : r1, r & 31);
    t = __dadd_rn(t, x);
  }
  if (lane == 0) out[b] = t;
}

// Nodes of height h from their children at height h - 1 (child order).
__global__ void k_node_norm2(const uint8_t *__restrict__ mask, const int32_t *__restrict__ cstart,
                             int64_t n, const double *__restrict__ child, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = __popc((unsigned)mask[i]);
  const int32_t c0 = cstart[i];
  double t = 0.0;
  for (int c = 0; c < m; c++) t = __dadd_rn(t, child[c0 + c]);
  out[i] = t;
}

__global__ void k_node_coords(const uint64_t *__restrict__ keys, int64_t n, int32_t *__restrict__ I,
                              int32_t *__restrict__ J) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (I) I[i] = (int32_t)morton_compact(keys[i] >> 1);
  if (J) J[i] = (int32_t)morton_compact(keys[i]);
}

// Sort keys: the bits of a nonnegative double order like its value; NaN last.
__global__ void k_norm_keys(const double *__restrict__ n2, int64_t n, uint64_t *__restrict__ key,
                            int32_t *__restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = n2[i];
  key[i] = v != v ? ~0ull : (uint64_t)__double_as_longlong(v);
  idx[i] = (int32_t)i;
}

__global__ void k_quantize(const uint64_t *__restrict__ key, int64_t n, int e,
                           uint64_t *__restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (key[i] == ~0ull) {
    q[i] = ~0ull;  // NaN: never removed
    return;
  }
  const double v = ceil(scalbn(__longlong_as_double((long long)key[i]), -e));
  q[i] = v >= 18446744073709551616.0 ? ~0ull : (uint64_t)v;
}

// Number of leading entries whose prefix sum stays <= T (prefix sums are
// nondecreasing, so it is the first index above T).
__global__ void k_first_above(const uint64_t *__restrict__ cum, int64_t n, uint64_t T,
                              unsigned long long *__restrict__ first) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cum[i] > T) atomicMin(first, (unsigned long long)i);
}

__global__ void k_mark_kept(const int32_t *__restrict__ sidx, int64_t n,
                            const unsigned long long *__restrict__ first,
                            int32_t *__restrict__ keep) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  keep[sidx[t]] = (unsigned long long)t >= *first;
}

__global__ void k_keep_compact(const int32_t *__restrict__ keep, const int32_t *__restrict__ pos,
                               int64_t n, const uint64_t *__restrict__ keys,
                               uint64_t *__restrict__ okeys, int32_t *__restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  okeys[pos[i]] = keys[i];
  idx[pos[i]] = (int32_t)i;
}

void launch_block_norm2(const double *vals, int64_t n, int bs, double *out, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  const unsigned g = grid_for(n * 32, 256);
  if (bs == 16)
    k_block_norm2<16><<<g, 256, 0, s>>>(vals, n, out);
  else if (bs == 32)
    k_block_norm2<32><<<g, 256, 0, s>>>(vals, n, out);
  else
    k_block_norm2<64><<<g, 256, 0, s>>>(vals, n, out);
}

}  // namespace

extern "C" bsm_status bsm_node_norms2(bsm_matrix M, int height, double *norm2, int32_t *I,
                                      int32_t *J, int64_t *n_inout, int on_device, void *stream) {
  if (!M || !n_inout || height < 0 || (on_device != 0 && on_device != 1))
    return BSM_ERR_INVALID_ARG;
  if (height > M->L) return BSM_ERR_OUT_OF_RANGE;
  const int64_t nn = M->nblk == 0 ? 0 : M->nlev[height];
  const int64_t cap = *n_inout;
  *n_inout = nn;
  if (!norm2 && !I && !J) return BSM_OK;
  if (cap < nn) return BSM_ERR_BUFFER_TOO_SMALL;
  if (on_device && ((uintptr_t)norm2 % 8 || (uintptr_t)I % 4 || (uintptr_t)J % 4))
    return BSM_ERR_INVALID_ARG;
  if (nn == 0) return BSM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // squared norms up the levels, two buffers alternating
  double *cur = nullptr, *nxt = nullptr;
  bsm_status st = dev_alloc((void **)&cur, 8 * M->nblk, s);
  if (st != BSM_OK) return st;
  launch_block_norm2(M->vals, M->nblk, M->bs, cur, s);
  for (int h = 1; h <= height && st == BSM_OK; h++) {
    if ((st = dev_alloc((void **)&nxt, 8 * M->nlev[h], s)) != BSM_OK) break;
    count_launch();
    k_node_norm2<<<grid_for(M->nlev[h], 256), 256, 0, s>>>(M->lmask[h], M->lcstart[h],
                                                            M->nlev[h], cur, nxt);
    dev_free(cur, s);
    cur = nxt;
    nxt = nullptr;
  }
  const uint64_t *keys = height == 0 ? M->keys : M->lkeys[height];
  int32_t *dI = nullptr, *dJ = nullptr;
  if (st == BSM_OK && (I || J)) {
    if (on_device) {
      dI = I;
      dJ = J;
    } else if ((st = dev_alloc((void **)&dI, 4 * nn, s)) == BSM_OK) {
      st = dev_alloc((void **)&dJ, 4 * nn, s);
    }
    if (st == BSM_OK) {
      count_launch();
      k_node_coords<<<grid_for(nn, 256), 256, 0, s>>>(keys, nn, I ? dI : nullptr,
                                                       J ? dJ : nullptr);
    }
  }
  if (st == BSM_OK) {
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (norm2) cudaMemcpyAsync(norm2, cur, 8 * nn, k, s);
    if (!on_device) {
      if (I) cudaMemcpyAsync(I, dI, 4 * nn, cudaMemcpyDeviceToHost, s);
      if (J) cudaMemcpyAsync(J, dJ, 4 * nn, cudaMemcpyDeviceToHost, s);
      st = cuda_status(cudaStreamSynchronize(s));
    } else {
      st = cuda_status(cudaGetLastError());
    }
  }
  dev_free(cur, s);
  if (!on_device) {
    dev_free(dI, s);
    dev_free(dJ, s);
  }
  return st;
}

extern "C" bsm_status bsm_truncate(bsm_matrix M, double tau, bsm_matrix *out, int64_t *removed,
                                   double *bound, void *stream) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!M) return BSM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int bs = M->bs;
  const int64_t n = M->nblk;
  if (n > 0x7FFFFFFF) return BSM_ERR_UNSUPPORTED;
  const double t2 = tau * tau;
  // threshold in integer units of 2^e
  const bool none = !(tau > 0.0) || !(t2 > 0.0);
  const bool all = !none && std::isinf(t2);
  int e = 0;
  uint64_t T = 0;
  if (!none && !all) {
    int ex = 0;
    std::frexp(t2, &ex);
    e = ex - 1 - 63;
    T = (uint64_t)std::floor(std::ldexp(t2, -e));
  }
  bsm_matrix R = new_matrix_shell(M->nrows, M->ncols, bs, M->L);
  bsm_status st = BSM_OK;
  double *n2 = nullptr;
  uint64_t *k0 = nullptr, *k1 = nullptr, *q = nullptr;
  int32_t *i0 = nullptr, *i1 = nullptr, *keep = nullptr, *pos = nullptr, *idx = nullptr;
  unsigned long long *first = nullptr;
  int64_t nrem = 0, nkeep = n;
  double bnd = 0.0;
  auto owned_alloc = [&](void **p, size_t bytes) {
    bsm_status r = dev_alloc(p, bytes, s);
    if (r == BSM_OK) R->owned.push_back(*p);
    return r;
  };
  uint64_t *h = (uint64_t *)host_scratch().get(32);
  if (!h) st = BSM_ERR_OOM;
  if (st == BSM_OK && n > 0 && !none) {
    if ((st = dev_alloc((void **)&n2, 8 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&k0, 8 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&k1, 8 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&q, 8 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&i0, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&i1, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&keep, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&pos, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&first, 8, s)) == BSM_OK) {
      launch_block_norm2(M->vals, n, bs, n2, s);
      count_launch();
      k_norm_keys<<<grid_for(n, 256), 256, 0, s>>>(n2, n, k0, i0);
      st = sort_keys_u64(k0, k1, i0, i1, n, 64, s);  // stable: ties stay in Morton order
    }
    if (st == BSM_OK) {
      if (all) {
        // every block with a finite norm: the NaN keys sort last
        h[0] = ~0ull;
        cudaMemcpyAsync(first, h, 8, cudaMemcpyHostToDevice, s);
        count_launch();
        k_first_above<<<grid_for(n, 256), 256, 0, s>>>(k1, n, ~0ull - 1, first);
      } else {
        count_launch();
        k_quantize<<<grid_for(n, 256), 256, 0, s>>>(k1, n, e, q);
        st = scan_inclusive_u64_sat(q, k0, n, s);  // k0 now holds the prefix sums
        if (st == BSM_OK) {
          h[0] = (uint64_t)n;
          cudaMemcpyAsync(first, h, 8, cudaMemcpyHostToDevice, s);
          count_launch();
          k_first_above<<<grid_for(n, 256), 256, 0, s>>>(k0, n, T, first);
        }
      }
    }
    if (st == BSM_OK) {
      count_launch();
      k_mark_kept<<<grid_for(n, 256), 256, 0, s>>>(i1, n, first, keep);
      st = scan_exclusive_i32(keep, pos, n, s);
    }
    if (st == BSM_OK) {
      readback(h + 1, first, 8, s);
      st = cuda_status(cudaStreamSynchronize(s));
      if (all && h[1] == ~0ull) h[1] = (uint64_t)n;  // no NaN norms: everything goes
      nrem = (int64_t)h[1];
      nkeep = n - nrem;
      if (st == BSM_OK && !all && nrem > 0) {
        readback(h + 2, k0 + nrem - 1, 8, s);
        st = cuda_status(cudaStreamSynchronize(s));
        bnd = std::ldexp((double)h[2], e);
      }
      if (all) bnd = t2;
    }
  }
  if (st == BSM_OK && nkeep > 0) {
    if ((st = owned_alloc((void **)&R->keys, 8 * nkeep)) == BSM_OK &&
        (st = owned_alloc((void **)&R->vals, sizeof(double) * bs * bs * nkeep)) == BSM_OK) {
      if (nrem == 0) {
        cudaMemcpyAsync(R->keys, M->keys, 8 * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(R->vals, M->vals, sizeof(double) * bs * bs * n, cudaMemcpyDeviceToDevice,
                        s);
      } else if ((st = dev_alloc((void **)&idx, 4 * nkeep, s)) == BSM_OK) {
        count_launch();
        k_keep_compact<<<grid_for(n, 256), 256, 0, s>>>(keep, pos, n, M->keys, R->keys, idx);
        launch_gather_blocks(M->vals, idx, R->vals, nkeep, bs, s);
        st = cuda_status(cudaGetLastError());
      }
    }
  }
  for (void *p : {(void *)n2, (void *)k0, (void *)k1, (void *)q, (void *)i0, (void *)i1,
                  (void *)keep, (void *)pos, (void *)idx, (void *)first})
    dev_free(p, s);
  R->nblk = st == BSM_OK ? nkeep : 0;
  if (st == BSM_OK) st = build_levels(R, s);
  if (st != BSM_OK) {
    free_matrix_shell(R, s);
    return st;
  }
  if (removed) *removed = nrem;
  if (bound) *bound = bnd;
  *out = R;
  return BSM_OK;
}
