// C = A*B: symbolic phase, numeric phase, exact-zero block removal, C levels.
#include <cstring>
#include <algorithm>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "bsm_internal.cuh"

namespace {

__global__ void k_compact_c(const int32_t *__restrict__ nz, const int32_t *__restrict__ pos,
                            int64_t nc, const uint64_t *__restrict__ ckeys,
                            uint64_t *__restrict__ okeys, int32_t *__restrict__ idx) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc || !nz[c]) return;
  okeys[pos[c]] = ckeys[c];
  idx[pos[c]] = (int32_t)c;
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

bsm_status check_pair(bsm_matrix A, bsm_matrix B) {
  if (!A || !B) return BSM_ERR_INVALID_ARG;
  if (A->ncols != B->nrows) return BSM_ERR_DIM_MISMATCH;
  if (A->bs != B->bs) return BSM_ERR_BLOCKSIZE;
  if (A->device != B->device) return BSM_ERR_INVALID_ARG;
  return BSM_OK;
}

// For split modes *slices receives the split spec (slice count and digit
// format, see split_spec).
bsm_status check_opts(const bsm_mult_opts *o, int *prec, int *slices, int allowed_flags) {
  *prec = BSM_FP64;
  *slices = 0;
  if (!o) return BSM_OK;
  if (o->flags & ~allowed_flags) return BSM_ERR_INVALID_ARG;
  if (o->prec != BSM_FP64 && o->prec != BSM_SPLIT_BF16 && o->prec != BSM_SPLIT_FP8)
    return BSM_ERR_INVALID_ARG;
  const int maxs = o->prec == BSM_SPLIT_FP8 ? 12 : 8;
  if (o->slices < 0 || o->slices > maxs) return BSM_ERR_INVALID_ARG;
  if (o->bs != 0 && o->bs != 16 && o->bs != 32 && o->bs != 64) return BSM_ERR_BLOCKSIZE;
  *prec = o->prec;
  if (o->prec == BSM_SPLIT_BF16) *slices = split_spec(0, o->slices == 0 ? 7 : o->slices);
  if (o->prec == BSM_SPLIT_FP8) *slices = split_spec(1, o->slices == 0 ? 6 : o->slices);
  return BSM_OK;
}

// Assembles C from the numeric result: drops exactly-zero blocks and builds
// the level arrays.  Takes ownership of sym->ckeys and cvals (freed on error).
bsm_status finish_product(bsm_matrix C, SymbolicResult *sym, double *cvals, int32_t *nz,
                          unsigned *err, cudaStream_t s) {
  int64_t nc = sym->nc;
  int bs = C->bs;
  int32_t *pos = nullptr;
  bsm_status st = dev_alloc((void **)&pos, 4 * (nc + 1), s);
  if (st != BSM_OK) {
    dev_free(cvals, s);
    return st;
  }
  st = scan_exclusive_i32(nz, pos, nc, s);
  int32_t *h = (int32_t *)host_scratch().get(16);
  if (st == BSM_OK && !h) st = BSM_ERR_OOM;
  if (st == BSM_OK) {
    readback(h, pos + nc - 1, 4, s);
    readback(h + 1, nz + nc - 1, 4, s);
    readback(h + 2, err, 4, s);
    st = cuda_status(cudaStreamSynchronize(s));
  }
  if (st == BSM_OK && h[2] == DERR_TIMEOUT) st = BSM_ERR_TIMEOUT;
  if (st == BSM_OK && h[2] != DERR_NONE) st = BSM_ERR_CUDA;
  if (st != BSM_OK) {
    dev_free(pos, s);
    dev_free(cvals, s);
    return st;
  }
  int64_t nkeep = (int64_t)h[0] + h[1];
  if (nkeep == nc) {
    C->keys = sym->ckeys;
    C->vals = cvals;
    sym->ckeys = nullptr;
    C->owned.push_back(C->keys);
    C->owned.push_back(C->vals);
  } else {
    uint64_t *okeys = nullptr;
    double *ovals = nullptr;
    int32_t *idx = nullptr;
    if ((st = dev_alloc((void **)&okeys, 8 * (nkeep > 0 ? nkeep : 1), s)) ||
        (st = dev_alloc((void **)&ovals, sizeof(double) * bs * bs * (nkeep > 0 ? nkeep : 1), s)) ||
        (st = dev_alloc((void **)&idx, 4 * (nkeep > 0 ? nkeep : 1), s))) {
      dev_free(okeys, s);
      dev_free(ovals, s);
      dev_free(idx, s);
      dev_free(pos, s);
      dev_free(cvals, s);
      return st;
    }
    count_launch();
    k_compact_c<<<grid_for(nc, 256), 256, 0, s>>>(nz, pos, nc, sym->ckeys, okeys, idx);
    launch_gather_blocks(cvals, idx, ovals, nkeep, bs, s);
    dev_free(idx, s);
    dev_free(cvals, s);
    C->keys = okeys;
    C->vals = ovals;
    C->owned.push_back(okeys);
    C->owned.push_back(ovals);
  }
  dev_free(pos, s);
  C->nblk = nkeep;
  return build_levels(C, s);
}

bsm_status finish_product_copy(bsm_matrix C, const SymbolicResult &sym, const double *cvals,
                               const int32_t *nz, unsigned *err, cudaStream_t s) {
  const int64_t nc = sym.nc;
  const int bs = C->bs;
  if (nc == 0) return build_levels(C, s);
  int32_t *pos = nullptr;
  bsm_status st = dev_alloc((void **)&pos, 4 * (nc + 1), s);
  if (st != BSM_OK) return st;
  st = scan_exclusive_i32(nz, pos, nc, s);
  int32_t *h = (int32_t *)host_scratch().get(16);
  if (st == BSM_OK && !h) st = BSM_ERR_OOM;
  if (st == BSM_OK) {
    readback(h, pos + nc - 1, 4, s);
    readback(h + 1, nz + nc - 1, 4, s);
    readback(h + 2, err, 4, s);
    st = cuda_status(cudaStreamSynchronize(s));
  }
  if (st == BSM_OK && h[2] == DERR_TIMEOUT) st = BSM_ERR_TIMEOUT;
  if (st == BSM_OK && h[2] != DERR_NONE) st = BSM_ERR_CUDA;
  const int64_t nkeep = st == BSM_OK ? (int64_t)h[0] + h[1] : 0;
  uint64_t *okeys = nullptr;
  double *ovals = nullptr;
  int32_t *idx = nullptr;
  if (st == BSM_OK && ((st = dev_alloc((void **)&okeys, 8 * (nkeep > 0 ? nkeep : 1), s)) ||
                       (st = dev_alloc((void **)&ovals,
                                       sizeof(double) * bs * bs * (nkeep > 0 ? nkeep : 1), s)) ||
                       (st = dev_alloc((void **)&idx, 4 * (nkeep > 0 ? nkeep : 1), s)))) {
    dev_free(okeys, s);
    dev_free(ovals, s);
    okeys = nullptr;
    ovals = nullptr;
  }
  if (st == BSM_OK) {
    count_launch();
    k_compact_c<<<grid_for(nc, 256), 256, 0, s>>>(nz, pos, nc, sym.ckeys, okeys, idx);
    launch_gather_blocks(cvals, idx, ovals, nkeep, bs, s);
    C->keys = okeys;
    C->vals = ovals;
    C->owned.push_back(okeys);
    C->owned.push_back(ovals);
    C->nblk = nkeep;
  }
  dev_free(idx, s);
  dev_free(pos, s);
  if (st != BSM_OK) return st;
  return build_levels(C, s);
}

// Compacts the nonzero C blocks of one chunk into new arrays (or takes the
// chunk's arrays when nothing was dropped).
static bsm_status compact_chunk(SymbolicResult &r, double *&cvals, const int32_t *nz,
                                unsigned *err, int bs, uint64_t **okeys_out, double **ovals_out,
                                int64_t *n_out, cudaStream_t s) {
  const int64_t nc = r.nc;
  int32_t *pos = nullptr;
  bsm_status st = dev_alloc((void **)&pos, 4 * (nc + 1), s);
  if (st != BSM_OK) return st;
  st = scan_exclusive_i32(nz, pos, nc, s);
  int32_t *h = (int32_t *)host_scratch().get(16);
  if (st == BSM_OK && !h) st = BSM_ERR_OOM;
  if (st == BSM_OK) {
    readback(h, pos + nc - 1, 4, s);
    readback(h + 1, nz + nc - 1, 4, s);
    readback(h + 2, err, 4, s);
    st = cuda_status(cudaStreamSynchronize(s));
  }
  if (st == BSM_OK && h[2] == DERR_TIMEOUT) st = BSM_ERR_TIMEOUT;
  if (st == BSM_OK && h[2] != DERR_NONE) st = BSM_ERR_CUDA;
  if (st != BSM_OK) {
    dev_free(pos, s);
    return st;
  }
  const int64_t nkeep = (int64_t)h[0] + h[1];
  if (nkeep == nc) {
    *okeys_out = r.ckeys;
    *ovals_out = cvals;
    r.ckeys = nullptr;
    cvals = nullptr;
  } else {
    uint64_t *okeys = nullptr;
    double *ovals = nullptr;
    int32_t *idx = nullptr;
    const int64_t m = nkeep > 0 ? nkeep : 1;
    if ((st = dev_alloc((void **)&okeys, 8 * m, s)) ||
        (st = dev_alloc((void **)&ovals, sizeof(double) * bs * bs * m, s)) ||
        (st = dev_alloc((void **)&idx, 4 * m, s))) {
      dev_free(okeys, s);
      dev_free(ovals, s);
      dev_free(idx, s);
      dev_free(pos, s);
      return st;
    }
    count_launch();
    k_compact_c<<<grid_for(nc, 256), 256, 0, s>>>(nz, pos, nc, r.ckeys, okeys, idx);
    launch_gather_blocks(cvals, idx, ovals, nkeep, bs, s);
    dev_free(idx, s);
    *okeys_out = okeys;
    *ovals_out = ovals;
  }
  dev_free(pos, s);
  *n_out = nkeep;
  return BSM_OK;
}

// One product: the symbolic phase delivers the task list in Morton-range
// chunks (one chunk unless a level exceeds the pair budget); each chunk is
// computed and compacted as it arrives, and C is assembled from the chunks.
static bsm_status multiply_chunked(bsm_matrix A, bsm_matrix B, int prec, int slices,
                                   cudaStream_t s, bsm_matrix *out, int upper, uint64_t key_lo,
                                   uint64_t key_hi);

bsm_status multiply_one(bsm_matrix A, bsm_matrix B, int prec, int slices, cudaStream_t s,
                        bsm_matrix *out, bool upper, uint64_t key_lo, uint64_t key_hi) {
  *out = nullptr;
  const int wb = prec == BSM_SPLIT_FP8 ? 32 : (A->bs == 64 ? 32 : A->bs);  // kernel's width
  if (prec == BSM_FP64 || A->bs == wb)
    return multiply_chunked(A, B, prec, slices, s, out, upper, key_lo, key_hi);
  // The split kernels take 16- and 32-wide blocks (E4M3: 32 only).  Their
  // result does not depend on the leaf size: the scales span whole rows of A
  // and columns of B and the digit sums are exact, so the product at another
  // width is the product of the re-cut operands, cut back.  For an
  // upper-triangle result the pruning applies at the coarser of the two
  // widths, and blocks below the diagonal are dropped when cutting finer.  A
  // key range maps exactly onto finer blocks (each key becomes four).
  const bool coarser = wb < A->bs;  // computing on finer blocks than the operands'
  if (key_hi && !coarser) return BSM_ERR_UNSUPPORTED;
  bsm_matrix a = nullptr, b = nullptr, c = nullptr;
  bsm_status st = reblock_impl(A, wb, 0, &a, nullptr, s);
  if (st == BSM_OK) st = B == A ? (b = a, BSM_OK) : reblock_impl(B, wb, 0, &b, nullptr, s);
  if (st == BSM_OK)
    st = multiply_chunked(a, b, prec, slices, s, &c, upper ? (coarser ? 2 : 1) : 0, key_lo << 2,
                          key_hi << 2);
  if (st == BSM_OK) st = reblock_impl(c, A->bs, upper && !coarser ? 2 : 0, out, nullptr, s);
  bsm_destroy(c);
  if (b != a) bsm_destroy(b);
  bsm_destroy(a);
  return st;
}

static bsm_status multiply_chunked(bsm_matrix A, bsm_matrix B, int prec, int slices,
                                   cudaStream_t s, bsm_matrix *out, int upper, uint64_t key_lo,
                                   uint64_t key_hi) {
  *out = nullptr;
  LastStats &ls = last_stats();
  ls = LastStats();
  const int64_t l0 = launch_counter();
  // timing (when enabled): events only, resolved by bsm_last_phase_ms, so
  // that the product never waits for them
  timing_begin();
  const int t_begin = timing_mark(s);
  const int bs = A->bs;
  struct Chunk {
    uint64_t *keys;
    double *vals;
    int64_t n;
  };
  std::vector<Chunk> chunks;
  unsigned *err = nullptr;
  bsm_status st = dev_alloc((void **)&err, sizeof(unsigned), s);
  if (st == BSM_OK) cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  LeafSink sink = [&](SymbolicResult &r) -> bsm_status {
    ls.triples += r.nt;
    ls.nc_sym += r.nc;
    if (r.nc == 0) return BSM_OK;
    if (r.nc > 0x7FFFFFFF) return BSM_ERR_UNSUPPORTED;
    double *cvals = nullptr;
    int32_t *nz = nullptr;
    bsm_status e;
    if ((e = dev_alloc((void **)&cvals, sizeof(double) * bs * bs * r.nc, s)) ||
        (e = dev_alloc((void **)&nz, 4 * r.nc, s))) {
      dev_free(cvals, s);
      dev_free(nz, s);
      return e;
    }
    const int t_a = timing_mark(s);
    {
      NvtxRange numeric(prec == BSM_FP64 ? "numeric fp64" : "numeric split");
      e = prec == BSM_FP64 ? numeric_fp64(A, B, r, cvals, nz, err, s)
                           : numeric_split(A, B, r, slices, cvals, nz, err, s);
    }
    const int t_b = timing_mark(s);
    Chunk c{nullptr, nullptr, 0};
    if (e == BSM_OK) e = compact_chunk(r, cvals, nz, err, bs, &c.keys, &c.vals, &c.n, s);
    const int t_c = timing_mark(s);
    timing_span(1, t_a, t_b);
    timing_span(2, t_b, t_c);
    dev_free(cvals, s);
    dev_free(nz, s);
    if (e == BSM_OK) {
      if (c.n > 0) {
        chunks.push_back(c);
      } else {
        dev_free(c.keys, s);
        dev_free(c.vals, s);
      }
    }
    return e;
  };
  int H = 0, nch = 0;
  int64_t tasks[BSM_MAXH + 1];
  if (st == BSM_OK)
    st = symbolic_chunks(A, B, sink, tasks, &H, &nch, s, 0, upper, key_lo, key_hi);
  int64_t mb = A->mb, nb = B->nb;
  int64_t side = mb > nb ? mb : nb;
  bsm_matrix C = new_matrix_shell(A->nrows, B->ncols, bs, ceil_log2_i64(side < 1 ? 1 : side));
  // assemble C: chunks are consecutive Morton ranges
  if (st == BSM_OK) {
    int64_t total = 0;
    for (auto &c : chunks) total += c.n;
    if (chunks.size() == 1) {
      C->keys = chunks[0].keys;
      C->vals = chunks[0].vals;
      chunks.clear();
    } else if (total > 0) {
      if ((st = dev_alloc((void **)&C->keys, 8 * total, s)) == BSM_OK &&
          (st = dev_alloc((void **)&C->vals, sizeof(double) * bs * bs * total, s)) == BSM_OK) {
        int64_t off = 0;
        for (auto &c : chunks) {
          cudaMemcpyAsync(C->keys + off, c.keys, 8 * c.n, cudaMemcpyDeviceToDevice, s);
          cudaMemcpyAsync(C->vals + off * bs * bs, c.vals, sizeof(double) * bs * bs * c.n,
                          cudaMemcpyDeviceToDevice, s);
          off += c.n;
        }
      }
    }
    if (C->keys) C->owned.push_back(C->keys);
    if (C->vals) C->owned.push_back(C->vals);
    C->nblk = total;
  }
  for (auto &c : chunks) {
    dev_free(c.keys, s);
    dev_free(c.vals, s);
  }
  dev_free(err, s);
  if (st == BSM_OK) st = build_levels(C, s);
  if (st != BSM_OK) {
    free_matrix_shell(C, s);
  } else {
    *out = C;
  }
  ls.nlev = H + 1;
  for (int l = 0; l <= H; l++) ls.tasks[l] = tasks[H - l];
  ls.chunks = nch;
  timing_rest(0, t_begin, timing_mark(s));  // symbolic phase: the rest of the product
  ls.launches = launch_counter() - l0;
  return st;
}

extern "C" bsm_status bsm_multiply(bsm_matrix A, bsm_matrix B, bsm_matrix *C,
                                   const bsm_mult_opts *opts, void *stream) {
  NvtxRange range("bsm_multiply");
  if (!C) return BSM_ERR_INVALID_ARG;
  *C = nullptr;
  if (!A || !B) return BSM_ERR_INVALID_ARG;
  int prec, slices;
  BSM_TRY(check_opts(opts, &prec, &slices, BSM_FLAG_TRANS_A | BSM_FLAG_TRANS_B));
  const int flags = opts ? opts->flags : 0;
  const int obs = opts ? opts->bs : 0;
  const bool ta = flags & BSM_FLAG_TRANS_A, tb = flags & BSM_FLAG_TRANS_B;
  // op(A) and op(B) dimensions are checked before any transposition is made.
  if ((ta ? A->nrows : A->ncols) != (tb ? B->ncols : B->nrows)) return BSM_ERR_DIM_MISMATCH;
  if (!obs && A->bs != B->bs) return BSM_ERR_BLOCKSIZE;
  if (A->device != B->device) return BSM_ERR_INVALID_ARG;
  const int cbs = obs ? obs : A->bs;  // the leaf size the product is computed at
  if (prec != BSM_FP64) BSM_TRY(split_supported(split_width(prec, cbs), slices));
  cudaStream_t s = (cudaStream_t)stream;
  // Operands of another leaf size are re-cut exactly (same entries, zero
  // blocks dropped), once per distinct handle.
  bsm_matrix Ar = nullptr, Br = nullptr;
  bsm_status st = BSM_OK;
  if (A->bs != cbs) st = reblock_impl(A, cbs, 0, &Ar, nullptr, s);
  if (st == BSM_OK && B->bs != cbs) st = B == A ? (Br = Ar, BSM_OK) : reblock_impl(B, cbs, 0, &Br, nullptr, s);
  bsm_matrix a = Ar ? Ar : A, b = Br ? Br : B;
  // The transposed task types (Sec. 3.2) are the plain product of transposed
  // handles: op(X) is X with its keys' row and column bits swapped and every
  // block transposed, made once here and released after the product.
  bsm_matrix At = nullptr, Bt = nullptr;
  if (st == BSM_OK && ta) st = bsm_transpose(a, &At, stream);
  if (st == BSM_OK && tb) st = (a == b && ta) ? (Bt = At, BSM_OK) : bsm_transpose(b, &Bt, stream);
  if (st == BSM_OK) st = multiply_one(ta ? At : a, tb ? Bt : b, prec, slices, s, C);
  if (Bt && Bt != At) bsm_destroy(Bt);
  if (At) bsm_destroy(At);
  if (Br && Br != Ar) bsm_destroy(Br);
  if (Ar) bsm_destroy(Ar);
  return st;
}

extern "C" bsm_status bsm_multiply_range(bsm_matrix A, bsm_matrix B, uint64_t key_lo,
                                         uint64_t key_hi, bsm_matrix *C,
                                         const bsm_mult_opts *opts, void *stream) {
  if (!C) return BSM_ERR_INVALID_ARG;
  *C = nullptr;
  BSM_TRY(check_pair(A, B));
  if (key_hi <= key_lo) return BSM_ERR_INVALID_ARG;
  int prec, slices;
  BSM_TRY(check_opts(opts, &prec, &slices, 0));
  if (opts && opts->bs) return BSM_ERR_INVALID_ARG;  // keys are those of the operands' size
  if (prec != BSM_FP64) BSM_TRY(split_supported(split_width(prec, A->bs), slices));
  return multiply_one(A, B, prec, slices, (cudaStream_t)stream, C, false, key_lo, key_hi);
}

extern "C" bsm_status bsm_last_chunks(int *nchunks) {
  if (!nchunks) return BSM_ERR_INVALID_ARG;
  *nchunks = last_stats().chunks;
  return BSM_OK;
}

extern "C" bsm_status bsm_last_stats(int64_t *tasks, int cap, int *nlev, int64_t *triples,
                                     int64_t *nc_sym) {
  LastStats &ls = last_stats();
  if (nlev) *nlev = ls.nlev;
  if (triples) *triples = ls.triples;
  if (nc_sym) *nc_sym = ls.nc_sym;
  if (tasks) {
    if (cap < ls.nlev) return BSM_ERR_BUFFER_TOO_SMALL;
    for (int l = 0; l < ls.nlev; l++) tasks[l] = ls.tasks[l];
  }
  return BSM_OK;
}

// LPT order: key = -(product-list length) so an ascending sort puts the
// longest C blocks first.
__global__ void k_batch_items(const int32_t *__restrict__ seg, int64_t nc, uint32_t p,
                              uint32_t *__restrict__ keys, uint64_t *__restrict__ items) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  keys[c] = 0xFFFFFFFFu - (uint32_t)(seg[c + 1] - seg[c]);
  items[c] = make_item(p, (uint64_t)c);
}

// A fixed pool of host threads for per-product host work (created on first
// use, never torn down: its threads idle on a condition variable until the
// process exits, so no thread-local CUDA state is released during static
// destruction).  run(nw, job) calls job(w) for w < nw on the pool's threads
// and returns when all have finished; one job runs at a time.
class WorkerPool {
 public:
  static constexpr int kThreads = 8;
  static WorkerPool &get() {
    static WorkerPool *pool = new WorkerPool();
    return *pool;
  }
  void run(int nw, const std::function<void(int)> &job) {
    std::lock_guard<std::mutex> one(run_mu_);
    std::unique_lock<std::mutex> lk(mu_);
    job_ = &job;
    njob_ = nw;
    next_ = 0;
    pending_ = nw;
    gen_++;
    cv_.notify_all();
    done_cv_.wait(lk, [&] { return pending_ == 0; });
    job_ = nullptr;
  }

 private:
  WorkerPool() {
    for (int t = 0; t < kThreads; t++) std::thread([this] { loop(); }).detach();
  }
  void loop() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return gen_ != seen && next_ < njob_; });
      seen = gen_;
      while (next_ < njob_) {
        const int w = next_++;
        const std::function<void(int)> *job = job_;
        lk.unlock();
        (*job)(w);
        lk.lock();
        if (--pending_ == 0) done_cv_.notify_all();
      }
    }
  }
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)> *job_ = nullptr;
  int njob_ = 0, next_ = 0, pending_ = 0;
  uint64_t gen_ = 0;
};

// Runs f(i, stream) for the products i < n on up to WorkerPool::kThreads host
// threads, each worker with its own stream that starts after the work queued
// so far on `s` and that `s` waits for at the end (events), so that the
// per-product host round trips of the symbolic phase and of C's assembly
// overlap.  Returns the first error; the work of every product that ran stays
// ordered before later work on `s`.
template <typename F>
static bsm_status parallel_products(int n, cudaStream_t s, F f) {
  const int nw = n < WorkerPool::kThreads ? n : WorkerPool::kThreads;
  if (nw <= 1) {
    for (int i = 0; i < n; i++) BSM_TRY(f(i, s));
    return BSM_OK;
  }
  int dev = 0;
  BSM_CUDA(cudaGetDevice(&dev));
  cudaEvent_t ready = nullptr;
  BSM_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  cudaEventRecord(ready, s);
  std::vector<cudaStream_t> ws(nw, nullptr);
  std::vector<cudaEvent_t> done(nw, nullptr);
  std::vector<bsm_status> res(nw, BSM_OK);
  std::vector<int64_t> launches(nw, 0);
  bsm_status st = BSM_OK;
  for (int w = 0; w < nw && st == BSM_OK; w++) {
    st = cuda_status(cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking));
    if (st == BSM_OK) st = cuda_status(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming));
    if (st == BSM_OK) cudaStreamWaitEvent(ws[w], ready, 0);
  }
  if (st == BSM_OK) {
    WorkerPool::get().run(nw, [&](int w) {
      cudaSetDevice(dev);
      const int64_t l0 = launch_counter();
      for (int i = w; i < n && res[w] == BSM_OK; i += nw) res[w] = f(i, ws[w]);
      launches[w] = launch_counter() - l0;
      cudaEventRecord(done[w], ws[w]);
    });
    for (int w = 0; w < nw; w++) {
      cudaStreamWaitEvent(s, done[w], 0);
      count_launch(launches[w]);
      if (st == BSM_OK) st = res[w];
    }
  }
  for (int w = 0; w < nw; w++) {
    if (ws[w]) cudaStreamDestroy(ws[w]);  // released once its work is done
    if (done[w]) cudaEventDestroy(done[w]);
  }
  cudaEventDestroy(ready);
  return st;
}

// ------------------------------------------- one symbolic pass for a batch
// The operands of all products are placed on the diagonal of one quadtree:
// product i's matrices at block offset i * 2^lmax in both coordinates (lmax:
// the largest operand depth), so that their keys are the products' own keys
// with the product index, Morton-spread, in the bits above 2 lmax.  The plain
// level-by-level expansion of this pair of block-diagonal matrices then pairs
// every product's nodes in the same launches (the nodes of different
// products meet only as NIL pairs and are never expanded), and its leaf task
// list is every product's, in product order.

__global__ void k_offset_keys(const uint64_t *__restrict__ src, int64_t n, uint64_t add,
                              uint64_t *__restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + add;  // no carry: the local keys are below 4^lmax
}

// First C block and first product of every product i <= n in the combined
// list (binary search for the product's first key).
__global__ void k_product_bounds(const uint64_t *__restrict__ ckeys, int64_t nc,
                                 const int32_t *__restrict__ seg, int n, int lmax,
                                 int64_t *__restrict__ cb, int64_t *__restrict__ tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const uint64_t lo = i < n ? morton_key((uint64_t)i, (uint64_t)i) << (2 * lmax) : ~0ull;
  int64_t a = 0, b = nc;
  while (a < b) {
    const int64_t m = (a + b) / 2;
    if (ckeys[m] < lo) a = m + 1; else b = m;
  }
  cb[i] = a;
  tb[i] = seg[a];
}

// Back to each product's own numbering: C keys without the product bits, A and
// B block indices relative to the product's first block.
__global__ void k_localize(uint64_t *__restrict__ ckeys, const int32_t *__restrict__ seg,
                           int32_t *__restrict__ ta, int32_t *__restrict__ tb, int64_t nc,
                           int lmax, const int64_t *__restrict__ aoff,
                           const int64_t *__restrict__ boff) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const uint64_t k = ckeys[c];
  const int p = (int)morton_compact(k >> (2 * lmax + 1));
  ckeys[c] = k & ((1ull << (2 * lmax)) - 1);
  const int32_t da = (int32_t)aoff[p], db = (int32_t)boff[p];
  for (int32_t t = seg[c]; t < seg[c + 1]; t++) {
    ta[t] -= da;
    tb[t] -= db;
  }
}

// The symbolic phase of the products idx[0..n) of one block size in one pass.
// On success sym[i] describe product i: nc, nt and ckeys its own (ckeys an
// allocation of its own), seg a view into the combined list (its entries
// index the combined ta / tb, which hold the product's own block indices);
// `whole` owns the combined seg / ta / tb (freed by the caller after the
// numeric phase) and *bound is the length of the combined ta / tb.
static bsm_status batched_symbolic(const std::vector<int> &idx, const bsm_matrix *A,
                                   const bsm_matrix *B, std::vector<SymbolicResult> &sym,
                                   SymbolicResult *whole, int64_t *bound, cudaStream_t s) {
  const int n = (int)idx.size();
  const int bs = A[idx[0]]->bs;
  int lmax = 0;
  int64_t na = 0, nb = 0;
  std::vector<int64_t> aoff(n + 1, 0), boff(n + 1, 0);
  for (int i = 0; i < n; i++) {
    const bsm_matrix a = A[idx[i]], b = B[idx[i]];
    lmax = std::max(lmax, std::max(a->L, b->L));
    aoff[i] = na;
    boff[i] = nb;
    na += a->nblk;
    nb += b->nblk;
  }
  aoff[n] = na;
  boff[n] = nb;
  const int lsup = lmax + ceil_log2_i64(n);
  if (lsup > BSM_MAXH || na > INT32_MAX || nb > INT32_MAX) return BSM_ERR_UNSUPPORTED;
  const int64_t side = (int64_t)n << lmax;  // blocks per side of the combined matrices
  bsm_matrix SA = new_matrix_shell(side * bs, side * bs, bs, lsup);
  bsm_matrix SB = new_matrix_shell(side * bs, side * bs, bs, lsup);
  bsm_status st = BSM_OK;
  auto keys_of = [&](bsm_matrix S, int64_t tot, bool left) -> bsm_status {
    BSM_TRY(dev_alloc((void **)&S->keys, 8 * (tot > 0 ? tot : 1), s));
    S->owned.push_back(S->keys);
    for (int i = 0; i < n; i++) {
      const bsm_matrix M = left ? A[idx[i]] : B[idx[i]];
      if (M->nblk == 0) continue;
      const uint64_t add = morton_key((uint64_t)i, (uint64_t)i) << (2 * lmax);
      count_launch();
      k_offset_keys<<<grid_for(M->nblk, 256), 256, 0, s>>>(M->keys, M->nblk, add,
                                                            S->keys + (left ? aoff[i] : boff[i]));
    }
    S->nblk = tot;
    return build_levels(S, s);
  };
  st = keys_of(SA, na, true);
  if (st == BSM_OK) st = keys_of(SB, nb, false);
  if (st == BSM_OK) st = symbolic_multiply(SA, SB, whole, s);
  free_matrix_shell(SA, s);
  free_matrix_shell(SB, s);
  if (st != BSM_OK) return st;
  *bound = whole->nt;
  int64_t *dv = nullptr;  // [cb (n+1) | tb (n+1) | aoff (n+1) | boff (n+1)]
  BSM_TRY(dev_alloc((void **)&dv, 8 * 4 * (n + 1), s));
  int64_t *h = (int64_t *)host_scratch().get(8 * 4 * (n + 1));
  if (!h) st = BSM_ERR_OOM;
  if (st == BSM_OK) {
    memcpy(h + 2 * (n + 1), aoff.data(), 8 * (n + 1));
    memcpy(h + 3 * (n + 1), boff.data(), 8 * (n + 1));
    cudaMemcpyAsync(dv + 2 * (n + 1), h + 2 * (n + 1), 16 * (n + 1), cudaMemcpyHostToDevice, s);
    count_launch(2);
    k_product_bounds<<<grid_for(n + 1, 128), 128, 0, s>>>(whole->ckeys, whole->nc, whole->seg, n,
                                                          lmax, dv, dv + (n + 1));
    if (whole->nc > 0)
      k_localize<<<grid_for(whole->nc, 256), 256, 0, s>>>(whole->ckeys, whole->seg, whole->ta,
                                                          whole->tb, whole->nc, lmax,
                                                          dv + 2 * (n + 1), dv + 3 * (n + 1));
    readback(h, dv, 16 * (n + 1), s);
    st = cuda_status(cudaStreamSynchronize(s));  // the host copy of aoff/boff is reused below
  }
  dev_free(dv, s);
  for (int i = 0; i < n && st == BSM_OK; i++) {
    SymbolicResult &r = sym[i];
    r = SymbolicResult();
    r.nc = h[i + 1] - h[i];
    r.nt = h[(n + 1) + i + 1] - h[(n + 1) + i];
    r.seg = whole->seg + h[i];
    r.ta = whole->ta;
    r.tb = whole->tb;
    r.H = whole->H;
    if (r.nc == 0) continue;
    if ((st = dev_alloc((void **)&r.ckeys, 8 * r.nc, s)) != BSM_OK) break;
    cudaMemcpyAsync(r.ckeys, whole->ckeys + h[i], 8 * r.nc, cudaMemcpyDeviceToDevice, s);
  }
  return st;
}

// Products of one block size: one symbolic pass over all of them, then one
// persistent numeric launch over all their C blocks in longest-first order,
// then zero removal and level build per product (concurrently, one host
// thread and stream per worker).
static bsm_status batched_group(const std::vector<int> &idx, const bsm_matrix *A,
                                const bsm_matrix *B, bsm_matrix *C, int prec, int slices,
                                cudaStream_t s) {
  const int n = (int)idx.size();
  const int bs = A[idx[0]]->bs;
  LastStats &ls = last_stats();
  const int t0 = timing_mark(s);  // timing: events only, resolved by bsm_last_phase_ms
  std::vector<SymbolicResult> sym(n);
  std::vector<bsm_matrix> shells(n, nullptr);
  std::vector<double *> cv(n, nullptr);
  std::vector<int32_t *> nz(n, nullptr);
  std::vector<void *> owned;
  unsigned *err = nullptr;
  bsm_status st = BSM_OK;
  SymbolicResult whole;  // the group's combined task list (owns seg / ta / tb)
  int64_t bound = 0;     // its length: the extent of ta / tb for every product
  bool views = false;    // sym[i].seg / ta / tb point into `whole`
  auto cleanup = [&](bool keep_results) {
    free_symbolic(&whole, s);
    for (int i = 0; i < n; i++) {
      if (views) sym[i].seg = sym[i].ta = sym[i].tb = nullptr;
      free_symbolic(&sym[i], s);
      if (!keep_results) {
        if (shells[i]) free_matrix_shell(shells[i], s);
        dev_free(cv[i], s);
      }
      dev_free(nz[i], s);
    }
    for (void *p : owned) dev_free(p, s);
    dev_free(err, s);
  };
  // one symbolic pass over the whole group; sym[i].seg / ta / tb are views
  // into `whole`, which owns them.  A group whose combined expansion exceeds
  // 32-bit pair indices at some level falls back to one pass per product.
  st = batched_symbolic(idx, A, B, sym, &whole, &bound, s);
  views = whole.seg != nullptr;  // the products' views exist (even if a later step failed)
  if (st == BSM_ERR_UNSUPPORTED && !views) {
    free_symbolic(&whole, s);
    for (int i = 0; i < n; i++) free_symbolic(&sym[i], s);
    st = parallel_products(n, s, [&](int i, cudaStream_t ws) {
      return symbolic_multiply(A[idx[i]], B[idx[i]], &sym[i], ws);
    });
  }
  for (int i = 0; i < n && st == BSM_OK; i++) {
    bsm_matrix a = A[idx[i]], b = B[idx[i]];
    if (sym[i].nc > 0xFFFFFFFFFFll) st = BSM_ERR_UNSUPPORTED;
    int64_t side = a->mb > b->nb ? a->mb : b->nb;
    shells[i] = new_matrix_shell(a->nrows, b->ncols, bs, ceil_log2_i64(side < 1 ? 1 : side));
    ls.triples += sym[i].nt;
    ls.nc_sym += sym[i].nc;
  }
  int64_t total = 0, total_nt = 0;
  for (int i = 0; i < n; i++) {
    total += sym[i].nc;
    total_nt += sym[i].nt;
  }
  if (st == BSM_OK) st = dev_alloc((void **)&err, sizeof(unsigned), s);
  if (st == BSM_OK) cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  for (int i = 0; i < n && st == BSM_OK; i++) {
    if (sym[i].nc == 0) continue;
    if ((st = dev_alloc((void **)&cv[i], sizeof(double) * bs * bs * sym[i].nc, s)) != BSM_OK) break;
    st = dev_alloc((void **)&nz[i], 4 * sym[i].nc, s);
  }
  // per-product descriptors; split mode: slices and exponents, and for long
  // lists sibling-pair items (merged lists, B pair slots)
  const int np = prec != BSM_FP64 && split_use_pairs(bs, slices, total_nt, total) ? 2 : 1;
  std::vector<ProdDesc> h(n);
  std::vector<int32_t *> bslot(n, nullptr);
  for (int i = 0; i < n && st == BSM_OK; i++) {
    h[i] = make_desc(A[idx[i]], B[idx[i]], sym[i], cv[i], nz[i]);
    if (views) h[i].nt = bound;  // seg entries index the combined ta / tb
    if (prec == BSM_FP64 || sym[i].nc == 0) continue;
    if (np == 2) {
      st = split_pairs_prepare(A[idx[i]], B[idx[i]], sym[i], slices, h[i], &bslot[i], owned, s);
      if (st == BSM_OK) st = split_compute(A[idx[i]], B[idx[i]], slices, h[i], err, s, bslot[i]);
    } else {
      st = split_prepare(A[idx[i]], B[idx[i]], slices, err, h[i], owned, s);
    }
  }
  const int64_t total_items = [&] {
    int64_t t = 0;
    for (int i = 0; i < n; i++) t += sym[i].nc ? h[i].nc : 0;
    return t;
  }();
  const int64_t total_item_nt = np == 2 ? [&] {
    int64_t t = 0;
    for (int i = 0; i < n; i++) t += sym[i].nc ? h[i].nt : 0;
    return t;
  }() : total_nt;
  // global work list, longest product lists first
  uint32_t *k0 = nullptr, *k1 = nullptr;
  uint64_t *v0 = nullptr, *v1 = nullptr;
  ProdDesc *table = nullptr;
  int *scr = nullptr;  // [0] longest list, [2..3] work counter
  if (st == BSM_OK && total > 0) {
    if ((st = dev_alloc((void **)&k0, 4 * total_items, s)) == BSM_OK) owned.push_back(k0);
    if (st == BSM_OK && (st = dev_alloc((void **)&k1, 4 * total_items, s)) == BSM_OK)
      owned.push_back(k1);
    if (st == BSM_OK && (st = dev_alloc((void **)&v0, 8 * total_items, s)) == BSM_OK)
      owned.push_back(v0);
    if (st == BSM_OK && (st = dev_alloc((void **)&v1, 8 * total_items, s)) == BSM_OK)
      owned.push_back(v1);
    if (st == BSM_OK &&
        (st = dev_alloc((void **)&table, sizeof(ProdDesc) * n, s)) == BSM_OK)
      owned.push_back(table);
    if (st == BSM_OK && (st = dev_alloc((void **)&scr, 16, s)) == BSM_OK) owned.push_back(scr);
  }
  const int t1 = timing_mark(s);
  if (st == BSM_OK && total > 0) {
    cudaMemsetAsync(scr, 0, 16, s);
    int64_t off = 0;
    for (int i = 0; i < n; i++) {  // items: C blocks, or pairs of them
      if (sym[i].nc == 0 || h[i].nc == 0) continue;
      count_launch();
      k_batch_items<<<grid_for(h[i].nc, 256), 256, 0, s>>>(h[i].seg, h[i].nc, (uint32_t)i,
                                                           k0 + off, v0 + off);
      off += h[i].nc;
    }
    st = sort_pairs_u32_u64(k0, k1, v0, v1, total_items, s);
    if (st == BSM_OK) {
      void *hp = host_scratch().get(sizeof(ProdDesc) * n + 16);
      if (!hp) st = BSM_ERR_OOM;
      if (st == BSM_OK) {
        memcpy(hp, h.data(), sizeof(ProdDesc) * n);
        cudaMemcpyAsync(table, hp, sizeof(ProdDesc) * n, cudaMemcpyHostToDevice, s);
        st = cuda_status(cudaStreamSynchronize(s));  // host table reused below
      }
    }
    int64_t *fold = nullptr;
    if (st == BSM_OK && prec != BSM_FP64 &&
        (st = dev_alloc((void **)&fold, split_fold_bytes(bs), s)) == BSM_OK)
      owned.push_back(fold);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(scr + 2);
    if (st == BSM_OK) {
      if (prec == BSM_FP64)
        st = numeric_fp64_batched(bs, table, v1, total, counter, err, 0, s);
      else {
        for (int i = 0; i < n; i++)  // the split kernel marks the nonzero C blocks
          if (sym[i].nc > 0) cudaMemsetAsync(nz[i], 0, 4 * sym[i].nc, s);
        st = split_launch(bs, slices, table, v1, total_items, counter, err, fold, s,
                          split_chunk_for(total_item_nt, total_items), np);
      }
    }
  }
  const int t2 = timing_mark(s);
  if (st == BSM_OK)
    st = parallel_products(n, s, [&](int i, cudaStream_t ws) {
      if (sym[i].nc == 0) return build_levels(shells[i], ws);
      double *c = cv[i];
      cv[i] = nullptr;
      return finish_product(shells[i], &sym[i], c, nz[i], err, ws);  // owns c
    });
  const int t3 = timing_mark(s);
  if (st != BSM_OK) {
    cleanup(false);
    return st;
  }
  for (int i = 0; i < n; i++) C[idx[i]] = shells[i];
  cleanup(true);
  timing_span(0, t0, t1);  // symbolic phases and the work list
  timing_span(1, t1, t2);  // the numeric launch
  timing_span(2, t2, t3);  // zero removal and C's levels
  return BSM_OK;
}

extern "C" bsm_status bsm_multiply_batched(int n, const bsm_matrix *A, const bsm_matrix *B,
                                           bsm_matrix *C, const bsm_mult_opts *opts,
                                           void *stream) {
  NvtxRange range("bsm_multiply_batched");
  if (n < 0 || (n > 0 && (!A || !B || !C))) return BSM_ERR_INVALID_ARG;
  for (int i = 0; i < n; i++) C[i] = nullptr;
  int prec, slices;
  BSM_TRY(check_opts(opts, &prec, &slices, 0));
  const int obs = opts ? opts->bs : 0;  // leaf size override (0: the operands')
  for (int i = 0; i < n; i++) {
    if (!A[i] || !B[i]) return BSM_ERR_INVALID_ARG;
    if (A[i]->ncols != B[i]->nrows) return BSM_ERR_DIM_MISMATCH;
    if (!obs && A[i]->bs != B[i]->bs) return BSM_ERR_BLOCKSIZE;
    if (A[i]->device != B[i]->device) return BSM_ERR_INVALID_ARG;
  }
  if (prec != BSM_FP64)
    for (int i = 0; i < n; i++)
      BSM_TRY(split_supported(split_width(prec, obs ? obs : A[i]->bs), slices));
  cudaStream_t s = (cudaStream_t)stream;
  LastStats &ls = last_stats();
  ls = LastStats();
  timing_begin();
  int64_t l0 = launch_counter();
  bsm_status st = BSM_OK;
  // Operands are re-cut (each distinct handle once) to the override size, and
  // split products at a width their kernels do not take to the kernel's
  // width; results are cut back to the override size or the operands' own,
  // exactly as bsm_multiply does (the split result does not depend on the
  // leaf size).
  std::vector<bsm_matrix> wa(A, A + n), wb(B, B + n), wc(n, nullptr), own;
  auto target = [&](bsm_matrix X) {
    const int b = obs ? obs : X->bs;
    return prec == BSM_FP64 ? b : split_width(prec, b);
  };
  auto recut = [&](bsm_matrix X, bsm_matrix *R) -> bsm_status {
    const int w = target(X);
    if (w == X->bs) {
      *R = X;
      return BSM_OK;
    }
    for (size_t k = 0; k < own.size(); k += 2)
      if (own[k] == X) {
        *R = own[k + 1];
        return BSM_OK;
      }
    BSM_TRY(reblock_impl(X, w, 0, R, nullptr, s));
    own.push_back(X);
    own.push_back(*R);
    return BSM_OK;
  };
  for (int i = 0; i < n && st == BSM_OK; i++) {
    st = recut(A[i], &wa[i]);
    if (st == BSM_OK) st = recut(B[i], &wb[i]);
  }
  for (int bs : {16, 32, 64}) {
    if (st != BSM_OK) break;
    std::vector<int> idx;
    for (int i = 0; i < n; i++)
      if (wa[i]->bs == bs) idx.push_back(i);
    if (idx.empty()) continue;
    st = batched_group(idx, wa.data(), wb.data(), wc.data(), prec, slices, s);
  }
  for (int i = 0; i < n; i++) {
    const int rbs = obs ? obs : A[i]->bs;  // the result's leaf size
    if (st == BSM_OK && wc[i] && wc[i]->bs != rbs) {
      st = reblock_impl(wc[i], rbs, 0, &C[i], nullptr, s);
      bsm_destroy(wc[i]);
    } else {
      C[i] = wc[i];
    }
    wc[i] = nullptr;
  }
  for (size_t k = 1; k < own.size(); k += 2) bsm_destroy(own[k]);
  ls.launches = launch_counter() - l0;
  if (st != BSM_OK) {
    for (int i = 0; i < n; i++) {
      bsm_destroy(C[i]);
      C[i] = nullptr;
    }
  }
  return st;
}
