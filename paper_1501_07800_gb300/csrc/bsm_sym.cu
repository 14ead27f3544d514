// Symmetric task types (Sec. 3.3, additional task types for the symmetric
// matrix square): C = A^2 with A symmetric, C = A B with A or B symmetric,
// and the symmetric rank-k products C = A A^T and C = A^T A.
//
// A symmetric matrix is stored as its upper triangle of blocks (I <= J), the
// diagonal blocks in full; a symmetric result is returned the same way.
//
// The paper's scheduler reaches the upper triangle of C by recursing through
// dedicated symmetric-square, symmetric-multiply and rank-k tasks.  Here the
// same result comes from the ordinary product with the symbolic phase
// restricted to C nodes on or above the diagonal: the full operand is
// materialised once (the strictly-upper blocks mirrored, transposed, into the
// lower triangle), and the expansion drops the lower-left quadrant of every
// diagonal C node, which removes the strictly-lower C blocks and all of their
// block products -- the near-halving of the flops that the symmetric
// recursion buys.
#include "bsm_internal.cuh"

namespace {

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ uint64_t swap_rowcol(uint64_t k) {
  return ((k & 0x5555555555555555ull) << 1) | ((k >> 1) & 0x5555555555555555ull);
}

// f[i] = 1 for a strictly-upper block; a block below the diagonal sets *bad.
__global__ void k_strict_upper(const uint64_t *__restrict__ keys, int64_t n,
                               int32_t *__restrict__ f, unsigned *__restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  const uint32_t I = morton_compact(k >> 1), J = morton_compact(k);
  f[i] = I < J;
  if (I > J) atomicOr(bad, 1u);
}

// Full key list: every stored block as it is, then the mirror of each
// strictly-upper block (its index tagged for transposition).
__global__ void k_mirror(const uint64_t *__restrict__ keys, int64_t n,
                         const int32_t *__restrict__ f, const int32_t *__restrict__ pos,
                         uint64_t *__restrict__ okeys, int32_t *__restrict__ oidx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  okeys[i] = keys[i];
  oidx[i] = (int32_t)i;
  if (f[i]) {
    okeys[n + pos[i]] = swap_rowcol(keys[i]);
    oidx[n + pos[i]] = (int32_t)((uint32_t)i | 0x80000000u);
  }
}

}  // namespace

// F = the full symmetric matrix whose upper triangle U stores.
static bsm_status sym_full(bsm_matrix U, bsm_matrix *out, cudaStream_t s) {
  *out = nullptr;
  if (U->nrows != U->ncols) return BSM_ERR_DIM_MISMATCH;
  const int64_t n = U->nblk;
  const int bs = U->bs;
  if (2 * n > 0x7FFFFFFF) return BSM_ERR_UNSUPPORTED;
  bsm_matrix F = new_matrix_shell(U->nrows, U->ncols, bs, U->L);
  bsm_status st = BSM_OK;
  int32_t *f = nullptr, *pos = nullptr, *i0 = nullptr, *i1 = nullptr;
  uint64_t *k0 = nullptr;
  unsigned *bad = nullptr;
  int64_t total = 0;
  if (n > 0) {
    if ((st = dev_alloc((void **)&f, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&pos, 4 * n, s)) == BSM_OK &&
        (st = dev_alloc((void **)&bad, 4, s)) == BSM_OK) {
      cudaMemsetAsync(bad, 0, 4, s);
      count_launch();
      k_strict_upper<<<grid_for(n, 256), 256, 0, s>>>(U->keys, n, f, bad);
      st = scan_exclusive_i32(f, pos, n, s);
    }
    int32_t *h = (int32_t *)host_scratch().get(16);
    if (st == BSM_OK && !h) st = BSM_ERR_OOM;
    if (st == BSM_OK) {
      readback(h, pos + n - 1, 4, s);
      readback(h + 1, f + n - 1, 4, s);
      readback(h + 2, bad, 4, s);
      st = cuda_status(cudaStreamSynchronize(s));
    }
    if (st == BSM_OK && h[2]) st = BSM_ERR_OUT_OF_RANGE;  // a block below the diagonal
    if (st == BSM_OK) total = n + (int64_t)h[0] + h[1];
    if (st == BSM_OK && (st = dev_alloc((void **)&k0, 8 * total, s)) == BSM_OK &&
        (st = dev_alloc((void **)&i0, 4 * total, s)) == BSM_OK &&
        (st = dev_alloc((void **)&i1, 4 * total, s)) == BSM_OK &&
        (st = dev_alloc((void **)&F->keys, 8 * total, s)) == BSM_OK) {
      F->owned.push_back(F->keys);
      if ((st = dev_alloc((void **)&F->vals, sizeof(double) * bs * bs * total, s)) == BSM_OK)
        F->owned.push_back(F->vals);
    }
    if (st == BSM_OK) {
      count_launch();
      k_mirror<<<grid_for(n, 256), 256, 0, s>>>(U->keys, n, f, pos, k0, i0);
      st = sort_keys_u64(k0, F->keys, i0, i1, total, 2 * U->L, s);
    }
    if (st == BSM_OK) {
      launch_gather_blocks_t(U->vals, i1, F->vals, total, bs, s);
      st = cuda_status(cudaGetLastError());
    }
  }
  for (void *p : {(void *)f, (void *)pos, (void *)i0, (void *)i1, (void *)k0, (void *)bad})
    dev_free(p, s);
  F->nblk = st == BSM_OK ? total : 0;
  if (st == BSM_OK) st = build_levels(F, s);
  if (st != BSM_OK) {
    free_matrix_shell(F, s);
    return st;
  }
  *out = F;
  return BSM_OK;
}

static bsm_status sym_opts(const bsm_mult_opts *opts, int bs, int *prec, int *slices) {
  BSM_TRY(check_opts(opts, prec, slices, 0));
  if (opts && opts->bs) return BSM_ERR_INVALID_ARG;  // computed at the operand's size
  if (*prec != BSM_FP64) BSM_TRY(split_supported(split_width(*prec, bs), *slices));
  return BSM_OK;
}

extern "C" bsm_status bsm_sym_to_full(bsm_matrix A, bsm_matrix *out, void *stream) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A) return BSM_ERR_INVALID_ARG;
  return sym_full(A, out, (cudaStream_t)stream);
}

extern "C" bsm_status bsm_sym_square(bsm_matrix A, bsm_matrix *C, const bsm_mult_opts *opts,
                                     void *stream) {
  if (!C) return BSM_ERR_INVALID_ARG;
  *C = nullptr;
  if (!A) return BSM_ERR_INVALID_ARG;
  if (A->nrows != A->ncols) return BSM_ERR_DIM_MISMATCH;
  int prec, slices;
  BSM_TRY(sym_opts(opts, A->bs, &prec, &slices));
  cudaStream_t s = (cudaStream_t)stream;
  bsm_matrix F = nullptr;
  BSM_TRY(sym_full(A, &F, s));
  bsm_status st = multiply_one(F, F, prec, slices, s, C, true);
  bsm_destroy(F);
  return st;
}

extern "C" bsm_status bsm_syrk(bsm_matrix A, int trans, bsm_matrix *C, const bsm_mult_opts *opts,
                               void *stream) {
  if (!C) return BSM_ERR_INVALID_ARG;
  *C = nullptr;
  if (!A || (trans != 0 && trans != 1)) return BSM_ERR_INVALID_ARG;
  int prec, slices;
  BSM_TRY(sym_opts(opts, A->bs, &prec, &slices));
  cudaStream_t s = (cudaStream_t)stream;
  bsm_matrix T = nullptr;
  BSM_TRY(bsm_transpose(A, &T, stream));
  // trans = 0: C = A A^T; trans = 1: C = A^T A
  bsm_status st = trans == 0 ? multiply_one(A, T, prec, slices, s, C, true)
                             : multiply_one(T, A, prec, slices, s, C, true);
  bsm_destroy(T);
  return st;
}

extern "C" bsm_status bsm_sym_multiply(bsm_matrix A, bsm_matrix B, int side, bsm_matrix *C,
                                       const bsm_mult_opts *opts, void *stream) {
  if (!C) return BSM_ERR_INVALID_ARG;
  *C = nullptr;
  if (!A || !B || (side != BSM_SYM_LEFT && side != BSM_SYM_RIGHT)) return BSM_ERR_INVALID_ARG;
  BSM_TRY(check_pair(A, B));
  int prec, slices;
  BSM_TRY(sym_opts(opts, A->bs, &prec, &slices));
  cudaStream_t s = (cudaStream_t)stream;
  bsm_matrix F = nullptr;
  BSM_TRY(sym_full(side == BSM_SYM_LEFT ? A : B, &F, s));
  bsm_status st = side == BSM_SYM_LEFT ? multiply_one(F, B, prec, slices, s, C)
                                       : multiply_one(A, F, prec, slices, s, C);
  bsm_destroy(F);
  return st;
}
