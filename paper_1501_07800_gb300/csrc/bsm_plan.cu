// Plans: repeated batched products with fixed operand structures, replayed
// from a CUDA graph, with launch parameters picked by a measuring autotuner.
//
// bsm_plan_create does everything that depends only on the structures of the
// operands once: the symbolic phase of every product (Algorithm 1 over the
// quadtrees), C's structures, the global work list and every buffer.  It then
// captures the numeric phase -- for split precision the scaling and slicing
// kernels too, because they depend on the values -- into a CUDA graph.
// bsm_plan_execute replays the graph; after bsm_update_values changed the
// values of an operand (same blocks), a replay recomputes C from the new values
// with no symbolic work and no host round trips.
//
// Leaf size: with BSM_FLAG_AUTOTUNE_BS the plan also tries the block sides
// 16, 32 and 64 (split mode: 16 and 32) on re-blocked copies of the operands
// and keeps the fastest full execution (copy refresh included).
//
// Autotuning: for a product class (precision, block size, slice count, number
// of products, and the magnitudes of the C-block count and of the mean and
// largest product-list length) the tuner times each candidate launch
// configuration -- work order (longest product list first, or product by
// product in Morton order), work items claimed per atomic (split kernel), the
// FP64 kernel's thread tile (DFMA: bs/8, bs/16 or bs/4 consecutive output
// columns per thread, with the rows to fill a C block among 128 threads; every
// tile sums each output in the same order, so the choice never changes a
// result) -- and caches the fastest for the process.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "bsm_internal.cuh"

struct bsm_plan_s {
  int n = 0, prec = BSM_FP64, slices = 0, bs = 0, device = 0;
  std::vector<bsm_matrix> A, B;  // not owned; must outlive the plan
  std::vector<SymbolicResult> sym;
  std::vector<double *> cv;
  std::vector<int32_t *> nz;
  std::vector<ProdDesc> desc;
  int64_t nitems = 0;
  uint64_t *items_lpt = nullptr, *items_morton = nullptr;
  ProdDesc *table = nullptr;
  int *scr = nullptr;  // [0] longest product list, [2..3] work counter
  unsigned *err = nullptr;
  int64_t *fold = nullptr;  // split mode: scratch of the numeric kernel
  int np = 1;               // split mode: C blocks per item (2: sibling pairs)
  std::vector<int32_t *> bslot;  // pairs: B pair slot of every B block, per product
  std::vector<void *> owned;
  // chosen configuration
  int order = 0;  // 0: longest first, 1: product-major Morton
  int chunk = 32, ctas_per_sm = 0;
  // FP64 tile: 0 DMMA; 1, 2, 3 DFMA thread tiles.  Split item shape: 1 single
  // C blocks, 4 grouped C blocks (bs 16).  -1: the process default.
  int form = -1;
  bool tuned = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // Leaf-size choice (BSM_FLAG_AUTOTUNE_BS): the plan wraps an inner plan at
  // block size `bs` over re-blocked copies of the operands, refreshed from the
  // caller's handles at every execution; results are re-cut to user_bs.
  bsm_plan inner = nullptr;
  int user_bs = 0;
  std::vector<bsm_matrix> rsrc, rops;  // caller handle -> re-blocked copy (owned)
  std::vector<int32_t *> rmap;         // refresh maps (owned)
};

namespace {

__global__ void k_plan_items(const int32_t *__restrict__ seg, int64_t nc, uint32_t p,
                             uint32_t *__restrict__ keys, uint64_t *__restrict__ items) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  keys[c] = 0xFFFFFFFFu - (uint32_t)(seg[c + 1] - seg[c]);
  items[c] = make_item(p, (uint64_t)c);
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct TuneKey {
  int prec, bs, slices, np, n, lg_nc, lg_mean, lg_max;
  bool operator<(const TuneKey &o) const {
    return std::tie(prec, bs, slices, np, n, lg_nc, lg_mean, lg_max) <
           std::tie(o.prec, o.bs, o.slices, o.np, o.n, o.lg_nc, o.lg_mean, o.lg_max);
  }
};
struct TuneVal {
  int order, chunk, ctas, form;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

int ilog2(int64_t x) {
  int l = 0;
  while (x > 1) {
    x >>= 1;
    l++;
  }
  return l;
}

// The numeric phase of the plan with a given configuration (no allocation:
// it may be captured).
bsm_status enqueue_numeric(bsm_plan P, int order, int chunk, int ctas, int form,
                           cudaStream_t s) {
  cudaMemsetAsync(P->scr + 2, 0, 8, s);  // work counter
  cudaMemsetAsync(P->err, 0, sizeof(unsigned), s);
  const uint64_t *items = order == 0 ? P->items_lpt : P->items_morton;
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(P->scr + 2);
  if (P->prec == BSM_FP64)
    return numeric_fp64_batched(P->bs, P->table, items, P->nitems, counter, P->err, ctas, s,
                                form);
  for (int i = 0; i < P->n; i++)
    if (P->sym[i].nc > 0) {
      BSM_TRY(split_compute(P->A[i], P->B[i], P->slices, P->desc[i], P->err, s,
                            P->np == 2 ? P->bslot[i] : nullptr));
      cudaMemsetAsync(P->nz[i], 0, 4 * P->sym[i].nc, s);  // the kernel marks nonzero blocks
    }
  return split_launch(P->bs, P->slices, P->table, items, P->nitems, counter, P->err, P->fold, s,
                      chunk, P->np == 2 ? 2 : (form == 1 ? -1 : (form == 4 ? 4 : 1)));
}

void destroy_plan(bsm_plan P) {
  if (!P) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  if (P->inner) destroy_plan(P->inner);
  for (bsm_matrix M : P->rops) bsm_destroy(M);
  for (int32_t *m : P->rmap) dev_free(m, nullptr);
  cudaStream_t s = P->stream;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (auto &sy : P->sym) free_symbolic(&sy, s);
  for (double *p : P->cv) dev_free(p, s);
  for (int32_t *p : P->nz) dev_free(p, s);
  for (void *p : P->owned) dev_free(p, s);
  dev_free(P->err, s);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (cur != P->device) cudaSetDevice(cur);
  delete P;
}

// Times one configuration (best of `reps` runs), in ms.
float time_config(bsm_plan P, int order, int chunk, int ctas, int form, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(a, P->stream);
    if (enqueue_numeric(P, order, chunk, ctas, form, P->stream) != BSM_OK) break;
    cudaEventRecord(b, P->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

bsm_status autotune(bsm_plan P) {
  int64_t tot_nt = 0, max_nk = 0;
  for (int i = 0; i < P->n; i++) tot_nt += P->sym[i].nt;
  int *h = (int *)host_scratch().get(16);
  if (!h) return BSM_ERR_OOM;
  cudaMemsetAsync(P->scr, 0, 4, P->stream);
  for (int i = 0; i < P->n; i++) launch_max_seg(P->sym[i], P->scr, P->stream);
  readback(h, P->scr, 4, P->stream);
  BSM_CUDA(cudaStreamSynchronize(P->stream));
  max_nk = h[0];
  TuneKey key{P->prec, P->bs, P->slices, P->np, P->n, ilog2(P->nitems),
              ilog2(P->nitems ? tot_nt / P->nitems : 0), ilog2(max_nk)};
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      P->order = it->second.order;
      P->chunk = it->second.chunk;
      P->ctas_per_sm = it->second.ctas;
      P->form = it->second.form;
      P->tuned = true;
      return BSM_OK;
    }
  }
  // FP64 runs at the FP64 pipe's rate whatever the schedule, and one run of a
  // large batch takes seconds: the arithmetic tile is measured in the default
  // order, then the other order with the better tile.
  std::vector<TuneVal> cands;
  if (P->prec == BSM_FP64) {
    if (fp64_mode() == 0) {
      cands.push_back({0, 32, 0, 0});  // the tensor form has one tile
    } else {
      for (int form : {1, 2, 3}) cands.push_back({0, 32, 0, form});
    }
  } else if (P->np != 2 && split_groups_compiled(P->bs, P->slices)) {
    // the item shape first (grouped or single C blocks), then the schedule
    // with the better one
    cands.push_back({0, 32, 0, 4});
    cands.push_back({0, 32, 0, 1});
  } else {
    for (int order : {0, 1})
      for (int chunk : {32, 8, 1}) cands.push_back({order, chunk, 0, -1});
  }
  const int reps = P->prec == BSM_FP64 ? 1 : 2;
  enqueue_numeric(P, cands[0].order, cands[0].chunk, cands[0].ctas, cands[0].form,
                  P->stream);  // warm-up
  float best = 1e30f;
  TuneVal pick = cands[0];
  auto measure = [&](const TuneVal &c) {
    float ms = time_config(P, c.order, c.chunk, c.ctas, c.form, reps);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  };
  for (const TuneVal &c : cands) measure(c);
  if (P->prec == BSM_FP64) {
    measure({1, 32, 0, pick.form});
  } else if (cands.size() == 2) {
    const int f = pick.form;
    for (int order : {0, 1})
      for (int chunk : {32, 8, 1})
        if (order != 0 || chunk != 32) measure({order, chunk, 0, f});
  }
  P->order = pick.order;
  P->chunk = pick.chunk;
  P->ctas_per_sm = pick.ctas;
  P->form = pick.form;
  P->tuned = true;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_cache[key] = pick;
  return BSM_OK;
}

// Refreshes the re-blocked operands of a wrapper plan from the caller's
// handles, then runs the inner plan (stream-ordered on `cs`).
bsm_status execute_wrapped(bsm_plan W, cudaStream_t cs) {
  for (size_t r = 0; r < W->rops.size(); r++) reblock_refresh(W->rsrc[r], W->rops[r], W->rmap[r], cs);
  BSM_CUDA(cudaGetLastError());
  return bsm_plan_execute(W->inner, cs);
}

// A wrapper plan computing at block size cb on re-cut copies of the operands
// (operands already of size cb are used as they are); results at user_bs.
bsm_status create_at_bs(int n, const bsm_matrix *A, const bsm_matrix *B, const bsm_mult_opts &o,
                        int cb, int user_bs, cudaStream_t cs, bsm_plan *out) {
  *out = nullptr;
  bsm_plan W = new bsm_plan_s();
  cudaGetDevice(&W->device);
  W->n = n;
  W->prec = o.prec;
  W->bs = cb;
  W->user_bs = user_bs;
  W->A.assign(A, A + n);
  W->B.assign(B, B + n);
  std::vector<bsm_matrix> ia(n), ib(n);
  bsm_status st = BSM_OK;
  auto copy_of = [&](bsm_matrix X, bsm_matrix *R) -> bsm_status {
    if (X->bs == cb) {
      *R = X;
      return BSM_OK;
    }
    for (size_t r = 0; r < W->rsrc.size(); r++)
      if (W->rsrc[r] == X) {
        *R = W->rops[r];
        return BSM_OK;
      }
    int32_t *map = nullptr;
    BSM_TRY(reblock_impl(X, cb, 1, R, &map, cs));
    W->rsrc.push_back(X);
    W->rops.push_back(*R);
    W->rmap.push_back(map);
    return BSM_OK;
  };
  for (int i = 0; i < n && st == BSM_OK; i++) {
    st = copy_of(A[i], &ia[i]);
    if (st == BSM_OK) st = copy_of(B[i], &ib[i]);
  }
  if (st == BSM_OK) st = bsm_plan_create(n, ia.data(), ib.data(), &o, cs, &W->inner);
  if (st != BSM_OK) {
    destroy_plan(W);
    return st;
  }
  W->nitems = W->inner->nitems;
  *out = W;
  return BSM_OK;
}

// Leaf-size autotuning: a wrapper plan per candidate block size with the
// default launch schedule, each timed over one full execution (operand
// refresh included; the plan's creation ran it once already); the fastest
// size is then planned again with the launch-schedule autotuner, which thus
// runs at one size only.  FP64 products run at the FP64 pipe's rate at every
// leaf size, so a coarser size only adds the flops of the zero fill of its
// larger blocks: FP64 candidates are the operands' size and the finer ones.
// The split kernels take 16 and 32 (wider operands are re-cut to 32).
bsm_status create_tuned_bs(int n, const bsm_matrix *A, const bsm_matrix *B, bsm_mult_opts o,
                           cudaStream_t cs, bsm_plan *out) {
  *out = nullptr;
  o.flags = 0;
  std::vector<int> cands;
  for (int cb : {16, 32, 64})
    if (o.prec == BSM_FP64 ? cb <= A[0]->bs : cb <= 32) cands.push_back(cb);
  bsm_plan best = nullptr;
  float best_ms = 1e30f;
  bsm_status first_err = BSM_OK;
  cudaEvent_t a, b;
  BSM_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return BSM_ERR_CUDA;
  }
  for (int cb : cands) {
    bsm_plan W = nullptr;
    bsm_status st = create_at_bs(n, A, B, o, cb, A[0]->bs, cs, &W);
    float ms = 1e30f;
    if (st == BSM_OK && cands.size() > 1) {
      cudaEventRecord(a, cs);
      st = execute_wrapped(W, cs);
      cudaEventRecord(b, cs);
      if (st == BSM_OK) st = cuda_status(cudaEventSynchronize(b));
      float t = 0;
      if (st == BSM_OK && cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms = t;
    }
    if (st != BSM_OK) {
      if (first_err == BSM_OK) first_err = st;
      destroy_plan(W);
      cudaGetLastError();
      continue;
    }
    if (ms < best_ms) {
      destroy_plan(best);
      best = W;
      best_ms = ms;
    } else {
      destroy_plan(W);
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!best) return first_err != BSM_OK ? first_err : BSM_ERR_CUDA;
  const int cb = best->bs;
  destroy_plan(best);
  o.flags = BSM_FLAG_AUTOTUNE;  // the chosen size's plan tunes its launch schedule
  return create_at_bs(n, A, B, o, cb, A[0]->bs, cs, out);
}

}  // namespace

extern "C" bsm_status bsm_plan_create(int n, const bsm_matrix *A, const bsm_matrix *B,
                                      const bsm_mult_opts *opts, void *stream, bsm_plan *out) {
  NvtxRange range("bsm_plan_create");
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || !A || !B) return BSM_ERR_INVALID_ARG;
  int tune = opts ? (opts->flags & BSM_FLAG_AUTOTUNE) : 0;
  const int tune_bs = opts ? (opts->flags & BSM_FLAG_AUTOTUNE_BS) : 0;
  bsm_mult_opts o = opts ? *opts : bsm_mult_opts{BSM_FP64, 0, 0, 0};
  o.flags &= ~(BSM_FLAG_AUTOTUNE | BSM_FLAG_AUTOTUNE_BS);
  int prec, slices;
  BSM_TRY(check_opts(&o, &prec, &slices, 0));
  const int obs = o.bs;  // leaf size override: operands re-cut to it, results at it
  o.bs = 0;
  if (obs && tune_bs) return BSM_ERR_INVALID_ARG;
  for (int i = 0; i < n; i++) {
    if (!A[i] || !B[i]) return BSM_ERR_INVALID_ARG;
    if (A[i]->ncols != B[i]->nrows) return BSM_ERR_DIM_MISMATCH;
    if (A[i]->device != B[i]->device) return BSM_ERR_INVALID_ARG;
  }
  const int bs = A[0]->bs;
  if (obs) {
    bsm_mult_opts oi = o;
    oi.flags |= tune;
    return create_at_bs(n, A, B, oi, obs, obs, (cudaStream_t)stream, out);
  }
  for (int i = 0; i < n; i++)
    if (A[i]->bs != bs || B[i]->bs != bs) return BSM_ERR_BLOCKSIZE;  // one block size per plan
  if (tune_bs) return create_tuned_bs(n, A, B, o, (cudaStream_t)stream, out);
  if (prec != BSM_FP64 && split_width(prec, bs) != bs) {
    // split kernels of another width: a wrapper plan on re-cut operands,
    // results cut back (the split result does not depend on the leaf size)
    bsm_mult_opts oi = o;
    oi.flags |= tune;
    return create_at_bs(n, A, B, oi, split_width(prec, bs), bs, (cudaStream_t)stream, out);
  }
  if (prec != BSM_FP64) BSM_TRY(split_supported(bs, slices));

  bsm_plan P = new bsm_plan_s();
  cudaGetDevice(&P->device);
  P->n = n;
  P->prec = prec;
  P->slices = slices;
  P->bs = bs;
  P->A.assign(A, A + n);
  P->B.assign(B, B + n);
  P->sym.resize(n);
  P->cv.assign(n, nullptr);
  P->nz.assign(n, nullptr);
  P->desc.resize(n);
  bsm_status st = cuda_status(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
  if (st == BSM_OK) st = cuda_status(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  if (st == BSM_OK) st = cuda_status(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  cudaStream_t s = P->stream;
  // order the plan's stream after the caller's work on the operands
  if (st == BSM_OK) {
    cudaEventRecord(P->ev_in, (cudaStream_t)stream);
    cudaStreamWaitEvent(s, P->ev_in, 0);
  }
  int64_t all_nc = 0, all_nt = 0;
  for (int i = 0; i < n && st == BSM_OK; i++) {
    st = symbolic_multiply(A[i], B[i], &P->sym[i], s);
    all_nc += P->sym[i].nc;
    all_nt += P->sym[i].nt;
  }
  if (st == BSM_OK) st = dev_alloc((void **)&P->err, sizeof(unsigned), s);
  for (int i = 0; i < n && st == BSM_OK; i++) {
    const int64_t nc = P->sym[i].nc;
    if (nc == 0) continue;
    if ((st = dev_alloc((void **)&P->cv[i], sizeof(double) * bs * bs * nc, s)) != BSM_OK) break;
    st = dev_alloc((void **)&P->nz[i], 4 * nc, s);
  }
  // per-product descriptors; split mode: slices and exponents, and for long
  // lists the sibling-pair items (merged lists, B pair slots)
  P->np = prec != BSM_FP64 && split_use_pairs(bs, slices, all_nt, all_nc) ? 2 : 1;
  P->bslot.assign(n, nullptr);
  for (int i = 0; i < n && st == BSM_OK; i++) {
    P->desc[i] = make_desc(A[i], B[i], P->sym[i], P->cv[i], P->nz[i]);
    if (prec == BSM_FP64 || P->sym[i].nc == 0) continue;
    if (P->np == 2)
      st = split_pairs_prepare(A[i], B[i], P->sym[i], slices, P->desc[i], &P->bslot[i], P->owned, s);
    else
      st = split_alloc(A[i], B[i], slices, P->desc[i], P->owned, s);
  }
  for (int i = 0; i < n && st == BSM_OK; i++) P->nitems += P->sym[i].nc ? P->desc[i].nc : 0;
  if (st == BSM_OK && P->nitems > 0xFFFFFFFFFFll) st = BSM_ERR_UNSUPPORTED;
  uint32_t *k0 = nullptr, *k1 = nullptr;
  const int64_t tot = P->nitems > 0 ? P->nitems : 1;
  auto grab = [&](void **p, size_t bytes) {
    if (st != BSM_OK) return;
    st = dev_alloc(p, bytes, s);
    if (st == BSM_OK) P->owned.push_back(*p);
  };
  grab((void **)&k0, 4 * tot);
  grab((void **)&k1, 4 * tot);
  grab((void **)&P->items_morton, 8 * tot);
  grab((void **)&P->items_lpt, 8 * tot);
  grab((void **)&P->table, sizeof(ProdDesc) * n);
  grab((void **)&P->scr, 16);
  if (st == BSM_OK) {
    cudaMemsetAsync(P->scr, 0, 16, s);
    int64_t off = 0;
    for (int i = 0; i < n; i++) {  // items: C blocks, or pairs of them
      if (P->sym[i].nc == 0 || P->desc[i].nc == 0) continue;
      count_launch();
      k_plan_items<<<grid_for(P->desc[i].nc, 256), 256, 0, s>>>(P->desc[i].seg, P->desc[i].nc,
                                                                (uint32_t)i, k0 + off,
                                                                P->items_morton + off);
      off += P->desc[i].nc;
    }
    st = sort_pairs_u32_u64(k0, k1, P->items_morton, P->items_lpt, P->nitems, s);
  }
  if (st == BSM_OK && prec != BSM_FP64 &&
      (st = dev_alloc((void **)&P->fold, split_fold_bytes(bs), s)) == BSM_OK)
    P->owned.push_back(P->fold);
  if (st == BSM_OK) {
    void *hp = host_scratch().get(sizeof(ProdDesc) * n + 16);
    if (!hp) st = BSM_ERR_OOM;
    if (st == BSM_OK) {
      memcpy(hp, P->desc.data(), sizeof(ProdDesc) * n);
      cudaMemcpyAsync(P->table, hp, sizeof(ProdDesc) * n, cudaMemcpyHostToDevice, s);
      st = cuda_status(cudaStreamSynchronize(s));
    }
  }
  if (st == BSM_OK && tune && P->nitems > 0) st = autotune(P);
  // one eager run: kernel attributes are set up outside the capture, and the
  // chosen configuration is known to launch
  if (st == BSM_OK && P->nitems > 0) {
    st = enqueue_numeric(P, P->order, P->chunk, P->ctas_per_sm, P->form, s);
    if (st == BSM_OK) st = cuda_status(cudaStreamSynchronize(s));
  }
  // capture the numeric phase
  if (st == BSM_OK) {
    st = cuda_status(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    if (st == BSM_OK) {
      bsm_status st2 = P->nitems > 0 ? enqueue_numeric(P, P->order, P->chunk, P->ctas_per_sm,
                                                       P->form, s)
                                     : cuda_status(cudaMemsetAsync(P->err, 0, 4, s));
      cudaError_t e = cudaStreamEndCapture(s, &P->graph);
      st = st2 != BSM_OK ? st2 : cuda_status(e);
    }
    if (st == BSM_OK) st = cuda_status(cudaGraphInstantiate(&P->exec, P->graph, 0));
  }
  if (st != BSM_OK) {
    destroy_plan(P);
    return st;
  }
  *out = P;
  return BSM_OK;
}

extern "C" bsm_status bsm_plan_execute(bsm_plan P, void *stream) {
  if (!P) return BSM_ERR_INVALID_ARG;
  NvtxRange range("bsm_plan_execute");
  cudaStream_t cs = (cudaStream_t)stream;
  if (P->inner) return execute_wrapped(P, cs);
  BSM_CUDA(cudaEventRecord(P->ev_in, cs));
  BSM_CUDA(cudaStreamWaitEvent(P->stream, P->ev_in, 0));
  BSM_CUDA(cudaGraphLaunch(P->exec, P->stream));
  BSM_CUDA(cudaEventRecord(P->ev_out, P->stream));
  BSM_CUDA(cudaStreamWaitEvent(cs, P->ev_out, 0));
  return BSM_OK;
}

extern "C" bsm_status bsm_plan_results(bsm_plan P, bsm_matrix *C, void *stream) {
  if (!P || !C) return BSM_ERR_INVALID_ARG;
  for (int i = 0; i < P->n; i++) C[i] = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  bsm_status st = BSM_OK;
  if (P->inner) {
    BSM_TRY(bsm_plan_results(P->inner, C, stream));
    if (P->bs == P->user_bs) return BSM_OK;
    // re-cut to the operands' block size (all-zero blocks dropped)
    for (int i = 0; i < P->n && st == BSM_OK; i++) {
      bsm_matrix R = nullptr;
      st = reblock_impl(C[i], P->user_bs, 0, &R, nullptr, s);
      bsm_destroy(C[i]);
      C[i] = R;
    }
    if (st != BSM_OK)
      for (int i = 0; i < P->n; i++) {
        bsm_destroy(C[i]);
        C[i] = nullptr;
      }
    return st;
  }
  for (int i = 0; i < P->n && st == BSM_OK; i++) {
    bsm_matrix a = P->A[i], b = P->B[i];
    int64_t side = a->mb > b->nb ? a->mb : b->nb;
    bsm_matrix Ci = new_matrix_shell(a->nrows, b->ncols, P->bs, ceil_log2_i64(side < 1 ? 1 : side));
    st = finish_product_copy(Ci, P->sym[i], P->cv[i], P->nz[i], P->err, s);
    if (st != BSM_OK) {
      free_matrix_shell(Ci, s);
      break;
    }
    C[i] = Ci;
  }
  if (st != BSM_OK)
    for (int i = 0; i < P->n; i++) {
      bsm_destroy(C[i]);
      C[i] = nullptr;
    }
  return st;
}

extern "C" bsm_status bsm_plan_block_size(bsm_plan P, int *bs) {
  if (!P || !bs) return BSM_ERR_INVALID_ARG;
  *bs = P->bs;
  return BSM_OK;
}

extern "C" bsm_status bsm_plan_tile(bsm_plan P, int *form, int *tile_m, int *tile_n) {
  if (!P) return BSM_ERR_INVALID_ARG;
  if (P->inner) return bsm_plan_tile(P->inner, form, tile_m, tile_n);
  int f = 2, m = 128, nn = P->bs * P->np;
  if (P->prec != BSM_FP64 && P->np != 2 && split_groups_compiled(P->bs, P->slices) &&
      (P->form == 4 || (P->form < 0 && split_use_groups(P->bs, P->slices))))
    f = 3;  // grouped items: N = bs per MMA, up to four C blocks per item
  if (P->prec == BSM_FP64) {
    const int fm = P->form < 0 ? fp64_mode() : P->form;
    if (fm == 0) {  // a warp's 8 x 8 mma.sync tiles
      f = 0;
      m = nn = 8;
    } else {        // a thread's outputs
      f = 1;
      nn = fm == 2 ? P->bs / 16 : (fm == 3 ? std::min(P->bs / 4, P->bs * P->bs / 128) : P->bs / 8);
      m = P->bs * P->bs / (128 * nn);
    }
  }
  if (form) *form = f;
  if (tile_m) *tile_m = m;
  if (tile_n) *tile_n = nn;
  return BSM_OK;
}

extern "C" bsm_status bsm_plan_info(bsm_plan P, int *order, int *chunk, int *ctas_per_sm,
                                    int64_t *nitems) {
  if (!P) return BSM_ERR_INVALID_ARG;
  if (P->inner) return bsm_plan_info(P->inner, order, chunk, ctas_per_sm, nitems);
  if (order) *order = P->order;
  if (chunk) *chunk = P->chunk;
  if (ctas_per_sm) *ctas_per_sm = P->ctas_per_sm;
  if (nitems) *nitems = P->nitems;
  return BSM_OK;
}

extern "C" bsm_status bsm_plan_destroy(bsm_plan P) {
  destroy_plan(P);
  return BSM_OK;
}
