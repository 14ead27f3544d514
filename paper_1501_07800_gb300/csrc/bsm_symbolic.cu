// Symbolic multiply: level-by-level quadtree recursion over node pairs.
//
// Algorithm 1 registers, for every pair of non-NIL nodes (A node, B node), the
// eight child products A_mk * B_kn (m, k, n in {0,1}) and skips those with a
// NIL operand.  Here all pairs of one level are expanded at once.  A pair's
// non-NIL children are read from the 4-bit child masks, so the count of child
// pairs in C quadrant q = (m, n) is popc over k of maskA(m,k) & maskB(k,n).
//
// Ordering invariant: at every level the pair list is grouped into segments,
// one per C node, in increasing Morton order of the C node key; inside a
// segment the pairs are in increasing order of the inner index K.  Children
// are emitted in the order (segment, quadrant q, parent pair, k), which keeps
// the invariant at the next level.  At the leaf level the segments are
// therefore exactly the C blocks in Morton order, each with its (A block,
// B block) products in ascending K -- C's structure and the task list come out
// of the recursion without a sort.  The sums of Algorithm 2 (C_mn = Y1 + Y2)
// become the concatenation of the children of a segment's pairs.
//
// Per level: count (per pair, four quadrant counts; exact 64-bit level total)
// -> exclusive scan of the 4-vectors -> segment pass (quadrant totals, new
// segments) -> scan -> fill.
//
// Large products: when a level would exceed a pair budget, the expansion
// continues depth first on parts of it -- the two halves of its segment list
// (contiguous Morton ranges of C), or, for a single C node, its four C
// quadrants one at a time -- so the leaf task list arrives in chunks that are
// contiguous, consecutive ranges of C in Morton order.
#include <cstdlib>
#include <vector>

#include "bsm_internal.cuh"

namespace {

// Mask and first-child index of node `i` at height h of a matrix; heights
// above the matrix's own root are virtual nodes with a single child 0.
struct LevelView {
  const uint8_t *mask;
  const int32_t *cstart;
  int virt;
};

__device__ __forceinline__ void node_info(const LevelView &v, int32_t i, unsigned &mask,
                                          int32_t &cstart) {
  if (v.virt) {
    mask = 1u;
    cstart = 0;
  } else {
    mask = v.mask[i];
    cstart = v.cstart[i];
  }
}

__device__ __forceinline__ int quad_count(unsigned ma, unsigned mb, int m, int n) {
  // A child (m,k) is bit 2m+k; B child (k,n) is bit 2k+n.
  return (int)(((ma >> (2 * m + 0)) & (mb >> (0 + n)) & 1u) +
               ((ma >> (2 * m + 1)) & (mb >> (2 + n)) & 1u));
}

// Restrictions of C.  Upper-triangle products (symmetric square, SYRK) keep
// only C nodes on or above the diagonal: children of a node strictly above the
// diagonal all lie above it; a diagonal node drops its lower-left quadrant
// q = 2 (m=1, n=0).  A Morton range [lo, hi) of C's block keys keeps a child
// whose key range [k 4^h, (k+1) 4^h) at child height h meets it.
struct CView {
  const uint64_t *sck;  // segment C keys of the level part (NULL: no restriction)
  const int32_t *pseg;  // segment id of each pair, offset by soff
  int32_t soff;
  int upper;            // prune below the diagonal
  int ch;               // height of the children (for the range test)
  uint64_t lo, hi;      // block-key range; hi == 0: none
};

__device__ __forceinline__ unsigned pair_qmask(const CView &u, int64_t p, unsigned qmask) {
  if (!u.sck) return qmask;
  const uint64_t k = u.sck[u.pseg[p] - u.soff];
  if (u.upper) {
    const bool diag = ((k >> 1) & 0x5555555555555555ull) == (k & 0x5555555555555555ull);
    if (diag) qmask &= ~4u;
  }
  if (u.hi) {
    const int sh = 2 * u.ch;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint64_t first = (4 * k + q) << sh;
      const uint64_t last = first + ((1ull << sh) - 1);  // inclusive
      if (first >= u.hi || last < u.lo) qmask &= ~(1u << q);
    }
  }
  return qmask;
}

// The four per-quadrant counts of a pair are kept as two 64-bit words,
// quadrants (0, 1) in cxy and (2, 3) in czw, each count in a 32-bit half:
// prefix sums of the words are the halves' prefix sums, because no
// per-quadrant prefix reaches 2^32 (a level holds fewer than 2^31 pairs), so
// the scans are plain 64-bit sums.
__device__ __forceinline__ uint64_t pack2(int32_t lo, int32_t hi) {
  return (uint64_t)(uint32_t)lo | ((uint64_t)(uint32_t)hi << 32);
}
__device__ __forceinline__ int4 counts_at(const uint64_t *__restrict__ cxy,
                                          const uint64_t *__restrict__ czw, int64_t i) {
  const uint64_t a = cxy[i], b = czw[i];
  return make_int4((int32_t)(uint32_t)a, (int32_t)(a >> 32), (int32_t)(uint32_t)b,
                   (int32_t)(b >> 32));
}

// Per pair: child counts of the quadrants in qmask; the level's exact total
// is accumulated in 64 bits: per thread over a grid-stride loop, per block in
// shared memory, one atomic per block.
__global__ void k_sym_count(const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                            int64_t np, LevelView va, LevelView vb, unsigned qmask, CView up,
                            uint64_t *__restrict__ cxy, uint64_t *__restrict__ czw,
                            unsigned long long *__restrict__ total) {
  __shared__ unsigned long long wsum[32];
  unsigned long long mine = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= np; p += stride) {
    if (p == np) {
      cxy[p] = czw[p] = 0;  // sentinel: the exclusive scans then end with the totals
      continue;
    }
    unsigned ma, mb;
    int32_t ca, cb;
    node_info(va, pa[p], ma, ca);
    node_info(vb, pb[p], mb, cb);
    const unsigned qm = pair_qmask(up, p, qmask);
    int4 c = make_int4((qm & 1u) ? quad_count(ma, mb, 0, 0) : 0,
                       (qm & 2u) ? quad_count(ma, mb, 0, 1) : 0,
                       (qm & 4u) ? quad_count(ma, mb, 1, 0) : 0,
                       (qm & 8u) ? quad_count(ma, mb, 1, 1) : 0);
    cxy[p] = pack2(c.x, c.y);
    czw[p] = pack2(c.z, c.w);
    mine += (unsigned)(c.x + c.y + c.z + c.w);
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) b += wsum[w];
    if (b) atomicAdd(total, b);
  }
}

__device__ __forceinline__ int q_of(const int4 &v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// Segment starts sst[] are stored offset by poff (pair index of the first
// pair of this part of the level); P is indexed from that first pair.
__global__ void k_sym_seg_count(const int32_t *__restrict__ sst, int32_t poff, int64_t ns,
                                const uint64_t *__restrict__ Pxy,
                                const uint64_t *__restrict__ Pzw, int32_t *__restrict__ nnz) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > ns) return;
  if (s == ns) {
    nnz[s] = 0;
    return;
  }
  const int4 a = counts_at(Pxy, Pzw, sst[s] - poff), b = counts_at(Pxy, Pzw, sst[s + 1] - poff);
  nnz[s] = (b.x > a.x) + (b.y > a.y) + (b.z > a.z) + (b.w > a.w);
}

// New segments: key 4*ckey + q and start offset for each non-empty quadrant.
__global__ void k_sym_seg_write(const uint64_t *__restrict__ sck, const int32_t *__restrict__ sst,
                                int32_t poff, int64_t ns, const uint64_t *__restrict__ Pxy,
                                const uint64_t *__restrict__ Pzw,
                                const int32_t *__restrict__ nbase, uint64_t *__restrict__ nck,
                                int32_t *__restrict__ nst) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int4 a = counts_at(Pxy, Pzw, sst[s] - poff), b = counts_at(Pxy, Pzw, sst[s + 1] - poff);
  int32_t off = a.x + a.y + a.z + a.w;  // children of all earlier segments
  int32_t j = nbase[s];
  for (int q = 0; q < 4; q++) {
    int32_t t = q_of(b, q) - q_of(a, q);
    if (t > 0) {
      nck[j] = 4 * sck[s] + (uint64_t)q;
      nst[j] = off;
      j++;
    }
    off += t;
  }
  if (s == ns - 1) nst[j] = off;  // end sentinel = total child pairs
}

// Child pairs in (segment, quadrant, parent pair, k) order.  Segment ids in
// pseg are offset by soff.
__global__ void k_sym_fill(const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                           const int32_t *__restrict__ pseg, int32_t soff, int64_t np,
                           const int32_t *__restrict__ sst, int32_t poff,
                           const uint64_t *__restrict__ Pxy, const uint64_t *__restrict__ Pzw,
                           const int32_t *__restrict__ nbase,
                           LevelView va, LevelView vb, unsigned qmask, CView up,
                           int32_t *__restrict__ npa, int32_t *__restrict__ npb,
                           int32_t *__restrict__ npseg) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  qmask = pair_qmask(up, p, qmask);
  int32_t s = pseg[p] - soff;
  const int4 a = counts_at(Pxy, Pzw, sst[s] - poff), b = counts_at(Pxy, Pzw, sst[s + 1] - poff),
             me = counts_at(Pxy, Pzw, p);
  unsigned ma, mb;
  int32_t ca, cb;
  node_info(va, pa[p], ma, ca);
  node_info(vb, pb[p], mb, cb);
  int32_t off = a.x + a.y + a.z + a.w;
  int32_t segid = nbase[s];
  for (int q = 0; q < 4; q++) {
    int32_t t = q_of(b, q) - q_of(a, q);
    if (t == 0 || !((qmask >> q) & 1u)) continue;
    int m = q >> 1, n = q & 1;
    int32_t pos = off + (q_of(me, q) - q_of(a, q));
    for (int k = 0; k < 2; k++) {
      unsigned abit = 2 * m + k, bbit = 2 * k + n;
      if (((ma >> abit) & 1u) && ((mb >> bbit) & 1u)) {
        npa[pos] = ca + __popc(ma & ((1u << abit) - 1u));
        npb[pos] = cb + __popc(mb & ((1u << bbit) - 1u));
        if (npseg) npseg[pos] = segid;
        pos++;
      }
    }
    off += t;
    segid++;
  }
}

__global__ void k_sym_root(int32_t *pa, int32_t *pb, int32_t *pseg, uint64_t *sck, int32_t *sst) {
  pa[0] = 0;
  pb[0] = 0;
  pseg[0] = 0;
  sck[0] = 0;
  sst[0] = 0;
  sst[1] = 1;
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

LevelView view_of(bsm_matrix M, int h) {
  LevelView v;
  if (h > M->L) {
    v.mask = nullptr;
    v.cstart = nullptr;
    v.virt = 1;
  } else {
    v.mask = M->lmask[h];
    v.cstart = M->lcstart[h];
    v.virt = 0;
  }
  return v;
}

// One part of one level of the expansion.  Arrays may point into a larger
// level (then `owns` is false and the offsets are nonzero).
struct Level {
  int32_t *pa = nullptr, *pb = nullptr, *pseg = nullptr, *sst = nullptr;
  uint64_t *sck = nullptr;
  int64_t np = 0, ns = 0;
  int h = 0;
  int32_t soff = 0, poff = 0;
  bool owns = false;
};

void free_level(Level &L, cudaStream_t s) {
  if (!L.owns) return;
  dev_free(L.pa, s);
  dev_free(L.pb, s);
  dev_free(L.pseg, s);
  dev_free(L.sst, s);
  dev_free(L.sck, s);
  L = Level();
}

int64_t pair_budget() {
  const char *e = getenv("BSM_SYM_BUDGET");
  if (e) {
    long long v = atoll(e);
    if (v >= 1) return v;
  }
  return (int64_t)1 << 30;
}

struct Expander {
  bsm_matrix A, B;
  cudaStream_t s;
  int64_t budget;
  int64_t *tasks;  // per height
  const LeafSink &sink;
  int upper;  // 0: all of C; k >= 1: C nodes at height >= k - 1 on or above the diagonal
  uint64_t lo = 0, hi = 0;  // C block-key range [lo, hi); hi == 0: all
  int chunks = 0;

  // segment starts [0] and [idx] of a level part, read back
  bsm_status read_sst(const Level &L, int64_t idx, int32_t *out) {
    int32_t *h = (int32_t *)host_scratch().get(16);
    if (!h) return BSM_ERR_OOM;
    readback(h, L.sst + idx, 4, s);
    BSM_CUDA(cudaStreamSynchronize(s));
    *out = h[0];
    return BSM_OK;
  }

  Level sub(const Level &L, int64_t s0, int64_t s1, int32_t p0abs, int32_t p1abs) {
    Level S;
    const int32_t p0 = p0abs - L.poff;
    S.pa = L.pa + p0;
    S.pb = L.pb + p0;
    S.pseg = L.pseg + p0;
    S.sst = L.sst + s0;
    S.sck = L.sck + s0;
    S.np = p1abs - p0abs;
    S.ns = s1 - s0;
    S.h = L.h;
    S.soff = L.soff + (int32_t)s0;
    S.poff = p0abs;
    S.owns = false;
    return S;
  }

  bsm_status leaf(Level &L) {
    SymbolicResult r;
    r.nc = L.ns;
    r.nt = L.np;
    r.ckeys = L.sck;
    r.seg = L.sst;
    r.ta = L.pa;
    r.tb = L.pb;
    chunks++;
    // the sink may take ownership of the arrays (then it clears the pointers)
    bsm_status st = sink(r);
    if (L.owns) {
      if (r.ckeys == nullptr) L.sck = nullptr;
      if (r.seg == nullptr) L.sst = nullptr;
      if (r.ta == nullptr) L.pa = nullptr;
      if (r.tb == nullptr) L.pb = nullptr;
    }
    return st;
  }

  bsm_status process(Level &L, unsigned qmask) {
    if (L.h == 0) return leaf(L);
    LevelView va = view_of(A, L.h), vb = view_of(B, L.h);
    uint64_t *P = nullptr;  // per-pair counts: quadrants (0, 1) at P, (2, 3) at P + np + 1
    unsigned long long *tot = nullptr;
    bsm_status st;
    if ((st = dev_alloc((void **)&P, 2 * sizeof(uint64_t) * (L.np + 1), s)) != BSM_OK) return st;
    uint64_t *const Pzw = P + L.np + 1;
    if ((st = dev_alloc((void **)&tot, 8, s)) != BSM_OK) {
      dev_free(P, s);
      return st;
    }
    cudaMemsetAsync(tot, 0, 8, s);
    const bool up_on = upper && L.h - 1 >= upper - 1;
    const CView up{(up_on || hi) ? L.sck : nullptr, L.pseg, L.soff, up_on ? 1 : 0, L.h - 1, lo,
                   hi};
    count_launch();
    {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t want = (L.np + 1 + 255) / 256, cap = (int64_t)(sms > 0 ? sms : 1) * 16;
      k_sym_count<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(L.pa, L.pb, L.np, va, vb,
                                                                        qmask, up, P, Pzw, tot);
    }
    unsigned long long *ht = (unsigned long long *)host_scratch().get(16);
    if (!ht) st = BSM_ERR_OOM;
    if (st == BSM_OK) {
      readback(ht, tot, 8, s);
      st = cuda_status(cudaStreamSynchronize(s));
    }
    const int64_t total = st == BSM_OK ? (int64_t)ht[0] : 0;
    dev_free(tot, s);
    if (st != BSM_OK || total == 0) {
      dev_free(P, s);
      return st;
    }
    const int64_t hard = (int64_t)INT32_MAX - 1;
    if (total > budget) {
      // split: halves of the segment list, or the quadrants of a single node
      if (L.ns > 1) {
        dev_free(P, s);
        const int64_t mid = L.ns / 2;
        int32_t p0, pm, p1;
        BSM_TRY(read_sst(L, 0, &p0));
        BSM_TRY(read_sst(L, mid, &pm));
        BSM_TRY(read_sst(L, L.ns, &p1));
        Level lo = sub(L, 0, mid, p0, pm), hi = sub(L, mid, L.ns, pm, p1);
        BSM_TRY(process(lo, qmask));
        return process(hi, qmask);
      }
      if (__builtin_popcount(qmask) > 1) {
        dev_free(P, s);
        for (int q = 0; q < 4; q++)
          if ((qmask >> q) & 1u) BSM_TRY(process(L, 1u << q));
        return BSM_OK;
      }
      if (total > hard) {
        dev_free(P, s);
        return BSM_ERR_UNSUPPORTED;  // one quadrant of one node exceeds 2^31 pairs
      }
    }
    if (total > hard) {
      dev_free(P, s);
      return BSM_ERR_UNSUPPORTED;
    }
    tasks[L.h - 1] += total;
    // scan, segments, fill
    int32_t *nnz = nullptr, *nbase = nullptr;
    Level N;
    N.h = L.h - 1;
    N.np = total;
    N.owns = true;
    auto fail = [&](bsm_status e) {
      dev_free(P, s);
      dev_free(nnz, s);
      dev_free(nbase, s);
      free_level(N, s);
      return e;
    };
    if ((st = scan_exclusive_u64(P, P, L.np + 1, s)) != BSM_OK ||
        (st = scan_exclusive_u64(Pzw, Pzw, L.np + 1, s)) != BSM_OK)
      return fail(st);
    if ((st = dev_alloc((void **)&nnz, 4 * (L.ns + 1), s)) ||
        (st = dev_alloc((void **)&nbase, 4 * (L.ns + 1), s)))
      return fail(st);
    count_launch();
    k_sym_seg_count<<<grid_for(L.ns + 1, 256), 256, 0, s>>>(L.sst, L.poff, L.ns, P, Pzw, nnz);
    if ((st = scan_exclusive_i32(nnz, nbase, L.ns + 1, s)) != BSM_OK) return fail(st);
    int32_t *hn = (int32_t *)host_scratch().get(16);
    if (!hn) return fail(BSM_ERR_OOM);
    readback(hn, nbase + L.ns, 4, s);
    if ((st = cuda_status(cudaStreamSynchronize(s))) != BSM_OK) return fail(st);
    N.ns = hn[0];
    const bool last = (N.h == 0);
    if ((st = dev_alloc((void **)&N.pa, 4 * N.np, s)) ||
        (st = dev_alloc((void **)&N.pb, 4 * N.np, s)) ||
        (!last && (st = dev_alloc((void **)&N.pseg, 4 * N.np, s))) ||
        (st = dev_alloc((void **)&N.sck, 8 * N.ns, s)) ||
        (st = dev_alloc((void **)&N.sst, 4 * (N.ns + 1), s)))
      return fail(st);
    count_launch(2);
    k_sym_seg_write<<<grid_for(L.ns, 256), 256, 0, s>>>(L.sck, L.sst, L.poff, L.ns, P, Pzw,
                                                        nbase, N.sck, N.sst);
    k_sym_fill<<<grid_for(L.np, 256), 256, 0, s>>>(L.pa, L.pb, L.pseg, L.soff, L.np, L.sst, L.poff,
                                                   P, Pzw, nbase, va, vb, qmask, up, N.pa, N.pb,
                                                   N.pseg);
    st = cuda_status(cudaGetLastError());
    dev_free(P, s);
    dev_free(nnz, s);
    dev_free(nbase, s);
    if (st == BSM_OK) st = process(N, 0xFu);
    free_level(N, s);
    return st;
  }
};

}  // namespace

void free_symbolic(SymbolicResult *r, cudaStream_t s) {
  dev_free(r->ckeys, s);
  dev_free(r->seg, s);
  dev_free(r->ta, s);
  dev_free(r->tb, s);
  r->ckeys = nullptr;
  r->seg = nullptr;
  r->ta = r->tb = nullptr;
}

bsm_status symbolic_chunks(bsm_matrix A, bsm_matrix B, const LeafSink &sink, int64_t *tasks,
                           int *H, int *nchunks, cudaStream_t s, int64_t budget, int upper,
                           uint64_t key_lo, uint64_t key_hi) {
  const int h0 = A->L > B->L ? A->L : B->L;
  *H = h0;
  *nchunks = 0;
  for (int h = 0; h <= BSM_MAXH; h++) tasks[h] = 0;
  if (A->nblk == 0 || B->nblk == 0) return BSM_OK;
  Level R;
  R.np = 1;
  R.ns = 1;
  R.h = h0;
  R.owns = true;
  bsm_status st;
  if ((st = dev_alloc((void **)&R.pa, 4, s)) || (st = dev_alloc((void **)&R.pb, 4, s)) ||
      (st = dev_alloc((void **)&R.pseg, 4, s)) || (st = dev_alloc((void **)&R.sst, 8, s)) ||
      (st = dev_alloc((void **)&R.sck, 8, s))) {
    free_level(R, s);
    return st;
  }
  count_launch();
  k_sym_root<<<1, 1, 0, s>>>(R.pa, R.pb, R.pseg, R.sck, R.sst);
  tasks[h0] = 1;
  Expander ex{A, B, s, budget > 0 ? budget : pair_budget(), tasks, sink, upper};
  ex.lo = key_lo;
  ex.hi = key_hi;
  st = ex.process(R, 0xFu);
  free_level(R, s);
  *nchunks = ex.chunks;
  return st;
}

bsm_status symbolic_multiply(bsm_matrix A, bsm_matrix B, SymbolicResult *out, cudaStream_t s) {
  *out = SymbolicResult();
  int nch = 0, H = 0;
  int64_t tasks[BSM_MAXH + 1];
  bool got = false;
  // one task list for the whole product (no budget split): the sink keeps it
  LeafSink keep = [&](SymbolicResult &r) -> bsm_status {
    if (got) return BSM_ERR_UNSUPPORTED;
    got = true;
    *out = r;
    r.ckeys = nullptr;
    r.seg = nullptr;
    r.ta = r.tb = nullptr;
    return BSM_OK;
  };
  bsm_status st = symbolic_chunks(A, B, keep, tasks, &H, &nch, s, (int64_t)INT32_MAX - 1);
  out->H = H;
  for (int h = 0; h <= BSM_MAXH; h++) out->tasks[h] = tasks[h];
  if (st != BSM_OK) free_symbolic(out, s);
  return st;
}
