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
// Per level: count (per pair, four quadrant counts) -> exclusive scan of the
// 4-vectors -> segment pass (quadrant totals, new segments) -> scan -> fill.
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

__global__ void k_sym_count(const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                            int64_t np, LevelView va, LevelView vb, int4 *__restrict__ cnt) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > np) return;
  if (p == np) {  // sentinel so that the exclusive scan also yields the total
    cnt[p] = make_int4(0, 0, 0, 0);
    return;
  }
  unsigned ma, mb;
  int32_t ca, cb;
  node_info(va, pa[p], ma, ca);
  node_info(vb, pb[p], mb, cb);
  cnt[p] = make_int4(quad_count(ma, mb, 0, 0), quad_count(ma, mb, 0, 1), quad_count(ma, mb, 1, 0),
                     quad_count(ma, mb, 1, 1));
}

__device__ __forceinline__ int q_of(const int4 &v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// Per segment: quadrant totals and the number of non-empty quadrants.
__global__ void k_sym_seg_count(const int32_t *__restrict__ sst, int64_t ns,
                                const int4 *__restrict__ P, int32_t *__restrict__ nnz) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > ns) return;
  if (s == ns) {
    nnz[s] = 0;
    return;
  }
  int4 a = P[sst[s]], b = P[sst[s + 1]];
  nnz[s] = (b.x > a.x) + (b.y > a.y) + (b.z > a.z) + (b.w > a.w);
}

// New segments: key 4*ckey + q and start offset for each non-empty quadrant.
__global__ void k_sym_seg_write(const uint64_t *__restrict__ sck, const int32_t *__restrict__ sst,
                                int64_t ns, const int4 *__restrict__ P,
                                const int32_t *__restrict__ nbase, uint64_t *__restrict__ nck,
                                int32_t *__restrict__ nst) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  int4 a = P[sst[s]], b = P[sst[s + 1]];
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
  if (s == ns - 1) {
    nst[j] = off;  // end sentinel = total child pairs
  }
}

// Child pairs in (segment, quadrant, parent pair, k) order.
__global__ void k_sym_fill(const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                           const int32_t *__restrict__ pseg, int64_t np,
                           const int32_t *__restrict__ sst, const int4 *__restrict__ P,
                           const int32_t *__restrict__ nbase, LevelView va, LevelView vb,
                           int32_t *__restrict__ npa, int32_t *__restrict__ npb,
                           int32_t *__restrict__ npseg) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int32_t s = pseg[p];
  int4 a = P[sst[s]], b = P[sst[s + 1]], me = P[p];
  unsigned ma, mb;
  int32_t ca, cb;
  node_info(va, pa[p], ma, ca);
  node_info(vb, pb[p], mb, cb);
  int32_t off = a.x + a.y + a.z + a.w;
  int32_t segid = nbase[s];
  for (int q = 0; q < 4; q++) {
    int32_t t = q_of(b, q) - q_of(a, q);
    if (t == 0) continue;
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

bsm_status symbolic_multiply(bsm_matrix A, bsm_matrix B, SymbolicResult *out, cudaStream_t s) {
  *out = SymbolicResult();
  int H = A->L > B->L ? A->L : B->L;
  out->H = H;
  if (A->nblk == 0 || B->nblk == 0) return BSM_OK;
  bsm_status st = BSM_OK;
  // current level
  int32_t *pa = nullptr, *pb = nullptr, *pseg = nullptr, *sst = nullptr;
  uint64_t *sck = nullptr;
  int64_t np = 1, ns = 1;
  auto free_level = [&]() {
    dev_free(pa, s);
    dev_free(pb, s);
    dev_free(pseg, s);
    dev_free(sst, s);
    dev_free(sck, s);
    pa = pb = pseg = sst = nullptr;
    sck = nullptr;
  };
  if ((st = dev_alloc((void **)&pa, 4, s)) || (st = dev_alloc((void **)&pb, 4, s)) ||
      (st = dev_alloc((void **)&pseg, 4, s)) || (st = dev_alloc((void **)&sst, 8, s)) ||
      (st = dev_alloc((void **)&sck, 8, s))) {
    free_level();
    return st;
  }
  count_launch();
  k_sym_root<<<1, 1, 0, s>>>(pa, pb, pseg, sck, sst);
  out->tasks[H] = 1;
  int32_t *hbuf = (int32_t *)host_scratch().get(64);
  if (!hbuf) {
    free_level();
    return BSM_ERR_OOM;
  }
  for (int h = H; h >= 1; h--) {
    LevelView va = view_of(A, h), vb = view_of(B, h);
    int4 *P = nullptr;
    int32_t *nnz = nullptr, *nbase = nullptr;
    int32_t *npa = nullptr, *npb = nullptr, *npseg = nullptr, *nst = nullptr;
    uint64_t *nck = nullptr;
    auto free_tmp = [&]() {
      dev_free(P, s);
      dev_free(nnz, s);
      dev_free(nbase, s);
    };
    if ((st = dev_alloc((void **)&P, sizeof(int4) * (np + 1), s)) ||
        (st = dev_alloc((void **)&nnz, 4 * (ns + 1), s)) ||
        (st = dev_alloc((void **)&nbase, 4 * (ns + 1), s))) {
      free_tmp();
      free_level();
      return st;
    }
    count_launch();
    k_sym_count<<<grid_for(np + 1, 256), 256, 0, s>>>(pa, pb, np, va, vb, P);
    if ((st = scan_exclusive_int4(P, P, np + 1, s)) != BSM_OK) {
      free_tmp();
      free_level();
      return st;
    }
    count_launch();
    k_sym_seg_count<<<grid_for(ns + 1, 256), 256, 0, s>>>(sst, ns, P, nnz);
    if ((st = scan_exclusive_i32(nnz, nbase, ns + 1, s)) != BSM_OK) {
      free_tmp();
      free_level();
      return st;
    }
    // sizes of the next level
    cudaMemcpyAsync(hbuf, P + np, sizeof(int4), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hbuf + 4, nbase + ns, 4, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      free_tmp();
      free_level();
      return cuda_status(e);
    }
    int64_t tot = (int64_t)hbuf[0] + hbuf[1] + hbuf[2] + hbuf[3];
    int64_t nns = hbuf[4];
    if (tot > INT32_MAX - 1 || hbuf[0] < 0 || hbuf[1] < 0 || hbuf[2] < 0 || hbuf[3] < 0) {
      free_tmp();
      free_level();
      return BSM_ERR_UNSUPPORTED;  // more than 2^31 pairs in one level
    }
    out->tasks[h - 1] = tot;
    if (tot == 0) {
      free_tmp();
      free_level();
      for (int g = h - 2; g >= 0; g--) out->tasks[g] = 0;
      return BSM_OK;  // empty product
    }
    bool last = (h == 1);
    if ((st = dev_alloc((void **)&npa, 4 * tot, s)) || (st = dev_alloc((void **)&npb, 4 * tot, s)) ||
        (!last && (st = dev_alloc((void **)&npseg, 4 * tot, s))) ||
        (st = dev_alloc((void **)&nck, 8 * nns, s)) ||
        (st = dev_alloc((void **)&nst, 4 * (nns + 1), s))) {
      dev_free(npa, s);
      dev_free(npb, s);
      dev_free(npseg, s);
      dev_free(nck, s);
      dev_free(nst, s);
      free_tmp();
      free_level();
      return st;
    }
    count_launch();
    k_sym_seg_write<<<grid_for(ns, 256), 256, 0, s>>>(sck, sst, ns, P, nbase, nck, nst);
    count_launch();
    k_sym_fill<<<grid_for(np, 256), 256, 0, s>>>(pa, pb, pseg, np, sst, P, nbase, va, vb, npa, npb,
                                                 npseg);
    e = cudaGetLastError();
    free_tmp();
    free_level();
    pa = npa;
    pb = npb;
    pseg = npseg;
    sck = nck;
    sst = nst;
    np = tot;
    ns = nns;
    if (e != cudaSuccess) {
      free_level();
      return cuda_status(e);
    }
  }
  // leaf level: segments are the C blocks
  dev_free(pseg, s);
  out->nc = ns;
  out->nt = np;
  out->ckeys = sck;
  out->seg = sst;
  out->ta = pa;
  out->tb = pb;
  return BSM_OK;
}
