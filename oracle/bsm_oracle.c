/*
 * Plain CPU oracle for the block-sparse product C = A*B over a sparse quadtree.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use this file; the product library never links or calls it, and it
 * shares no code, header or table with the CUDA path.
 *
 * What it computes (Rubensson & Rudberg, arXiv 1501.07800):
 *   - A matrix is a quadtree of nodes, each holding four child pointers; a NULL
 *     child is a NIL chunk id, i.e. a zero submatrix, at any level (Sec. 3.1,
 *     "Matrix" chunk type).  Every level halves the submatrix side, starting
 *     from a power-of-two number of leaf blocks so that A and B submatrices
 *     always match (Sec. 3.1).  Child c = 2*rowhalf + colhalf.
 *   - The lowest level holds a block-sparse leaf matrix: a 2-D array of
 *     optional bs x bs blocks, only nonzero blocks allocated (Sec. 4.1).
 *   - multiply() is Algorithm 1: NIL if either input is NIL; the leaf multiply
 *     at the lowest level; otherwise C_mn = add(A_m1 B_1n, A_m2 B_2n) for
 *     m, n in {1, 2} and the four results assembled into a new node
 *     (createFromIds, Sec. 3.2).
 *   - add() is Algorithm 2: recurse (or leaf add) when both inputs are
 *     non-NIL, otherwise the non-NIL input or NIL.  orc_add() exposes it as
 *     the C = A + B task type (Sec. 3.2).
 *   - The transposed task types C = A^T B, A B^T, A^T B^T (Sec. 3.2) run the
 *     same recursion with the children of a transposed operand taken in
 *     transposed position and its leaf blocks read transposed.
 *   - The leaf multiply is a sum of outer products over the inner block index
 *     (Sec. 4.1, Fig. 3), each block product a naive triple loop.
 *   - Blocks whose entries are all exactly 0.0 are not stored: input blocks
 *     are dropped when the matrix is built, product blocks after the multiply
 *     (sparsity found during the computation, abstract; only nonzero submatrices
 *     stored, Sec. 4.1).  -0.0 counts as zero, NaN does not.
 *   - Multiply-task counts per level (tasks whose inputs are both non-NIL) are
 *     the quantities C_l of Sec. 5.1, Eq. 1 - Eq. 5.
 *
 * Single threaded and deliberately unoptimised.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = -1,
  ORC_ERR_DIM_MISMATCH = -2,
  ORC_ERR_BLOCKSIZE = -3,
  ORC_ERR_OUT_OF_RANGE = -4,
  ORC_ERR_DUPLICATE = -5,
  ORC_ERR_OOM = -6
};

typedef struct orc_node {
  struct orc_node *child[4]; /* NULL = NIL */
  double **blk;              /* leaf only: leaf_nb*leaf_nb optional blocks */
} orc_node;

typedef struct orc_matrix {
  int64_t nrows, ncols;
  int bs;
  int L;       /* the tree spans 2^L leaf blocks per side */
  int leaf_nb; /* leaf matrix side in blocks, 2^(L - depth) */
  int depth;   /* level index of the leaves; the root is level 0 */
  orc_node *root;
} orc_matrix;

typedef struct {
  int64_t *tasks; /* per level, or NULL */
  int64_t triples;
  int oom;
  int ta, tb; /* operands enter transposed (Sec. 3.2 transposed task types) */
} orc_ctx;

/* ------------------------------------------------------------ node helpers */
static orc_node *new_node(const orc_matrix *m, int leaf) {
  orc_node *n = (orc_node *)calloc(1, sizeof(orc_node));
  if (!n) return NULL;
  if (leaf) {
    n->blk = (double **)calloc((size_t)m->leaf_nb * m->leaf_nb, sizeof(double *));
    if (!n->blk) {
      free(n);
      return NULL;
    }
  }
  return n;
}

static void free_node(const orc_matrix *m, orc_node *n) {
  if (!n) return;
  if (n->blk) {
    for (int64_t t = 0; t < (int64_t)m->leaf_nb * m->leaf_nb; t++) free(n->blk[t]);
    free(n->blk);
  }
  for (int c = 0; c < 4; c++) free_node(m, n->child[c]);
  free(n);
}

static int leaf_is_empty(const orc_matrix *m, const orc_node *n) {
  for (int64_t t = 0; t < (int64_t)m->leaf_nb * m->leaf_nb; t++)
    if (n->blk[t]) return 0;
  return 1;
}

static int block_is_zero(const double *b, int bs) {
  for (int64_t t = 0; t < (int64_t)bs * bs; t++)
    if (!(b[t] == 0.0)) return 0;
  return 1;
}

/* --------------------------------------------------------------- building */
static int ceil_log2(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) l++;
  return l;
}

void orc_free(orc_matrix *m) {
  if (!m) return;
  free_node(m, m->root);
  free(m);
}

static orc_matrix *alloc_matrix(int64_t nrows, int64_t ncols, int bs, int L, int leaf_nb) {
  orc_matrix *m = (orc_matrix *)calloc(1, sizeof(orc_matrix));
  if (!m) return NULL;
  m->nrows = nrows;
  m->ncols = ncols;
  m->bs = bs;
  m->L = L;
  if (leaf_nb > (1 << L)) leaf_nb = 1 << L;
  m->leaf_nb = leaf_nb;
  m->depth = L - ceil_log2(leaf_nb);
  return m;
}

/* Build from a COO list of dense row-major blocks.  L is the common tree depth
 * in blocks (callers pass the same L for the operands of one product);
 * leaf_nb must be a power of two.  Exactly-zero blocks are dropped. */
orc_matrix *orc_build(int64_t nrows, int64_t ncols, int bs, int L, int leaf_nb, int64_t nblk,
                      const int32_t *brow, const int32_t *bcol, const double *vals,
                      int *status) {
  *status = ORC_OK;
  if (nrows < 0 || ncols < 0 || bs < 1 || nblk < 0 || L < 0 || L > 30 || leaf_nb < 1 ||
      (leaf_nb & (leaf_nb - 1))) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  int64_t mb = (nrows + bs - 1) / bs, nb = (ncols + bs - 1) / bs;
  if (mb > ((int64_t)1 << L) || nb > ((int64_t)1 << L)) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  orc_matrix *m = alloc_matrix(nrows, ncols, bs, L, leaf_nb);
  if (!m) {
    *status = ORC_ERR_OOM;
    return NULL;
  }
  int lbits = L - m->depth; /* log2(leaf_nb) */
  size_t bbytes = (size_t)bs * bs * sizeof(double);
  for (int64_t t = 0; t < nblk; t++) {
    int64_t I = brow[t], J = bcol[t];
    if (I < 0 || I >= mb || J < 0 || J >= nb) {
      *status = ORC_ERR_OUT_OF_RANGE;
      orc_free(m);
      return NULL;
    }
  }
  /* duplicate detection over all listed keys (zero or not) */
  {
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nblk > 0 ? nblk : 1));
    if (!keys) {
      *status = ORC_ERR_OOM;
      orc_free(m);
      return NULL;
    }
    for (int64_t t = 0; t < nblk; t++) keys[t] = ((int64_t)brow[t] << 32) | (uint32_t)bcol[t];
    /* insertion into the tree below catches duplicates among nonzero blocks;
     * a simple sort catches the rest */
    for (int64_t gap = nblk / 2; gap > 0; gap /= 2) /* shell sort */
      for (int64_t i = gap; i < nblk; i++) {
        int64_t v = keys[i], j = i;
        while (j >= gap && keys[j - gap] > v) {
          keys[j] = keys[j - gap];
          j -= gap;
        }
        keys[j] = v;
      }
    for (int64_t t = 1; t < nblk; t++)
      if (keys[t] == keys[t - 1]) {
        free(keys);
        *status = ORC_ERR_DUPLICATE;
        orc_free(m);
        return NULL;
      }
    free(keys);
  }
  for (int64_t t = 0; t < nblk; t++) {
    const double *src = vals + (size_t)t * bs * bs;
    if (block_is_zero(src, bs)) continue;
    int64_t I = brow[t], J = bcol[t];
    orc_node **slot = &m->root;
    for (int level = 0; level <= m->depth; level++) {
      int leaf = (level == m->depth);
      if (!*slot) {
        *slot = new_node(m, leaf);
        if (!*slot) {
          *status = ORC_ERR_OOM;
          orc_free(m);
          return NULL;
        }
      }
      if (leaf) break;
      int shift = L - level - 1; /* bit of I, J that selects the child */
      int c = (int)(2 * ((I >> shift) & 1) + ((J >> shift) & 1));
      slot = &(*slot)->child[c];
    }
    int64_t li = I & ((1 << lbits) - 1), lj = J & ((1 << lbits) - 1);
    double **b = &(*slot)->blk[li * m->leaf_nb + lj];
    *b = (double *)malloc(bbytes);
    if (!*b) {
      *status = ORC_ERR_OOM;
      orc_free(m);
      return NULL;
    }
    memcpy(*b, src, bbytes);
  }
  return m;
}

/* ------------------------------------------------------------ leaf library */
/* Sum of outer products over the inner block index k (Sec. 4.1, Fig. 3). */
static orc_node *leaf_multiply(const orc_matrix *m, const orc_node *a, const orc_node *b,
                               orc_ctx *cx) {
  int nb = m->leaf_nb, bs = m->bs;
  orc_node *x = new_node(m, 1);
  if (!x) {
    cx->oom = 1;
    return NULL;
  }
  /* op(A)_ik is A_ik, or A_ki read transposed; likewise op(B)_kj. */
  const int ta = cx->ta, tb = cx->tb;
  for (int k = 0; k < nb; k++)
    for (int i = 0; i < nb; i++) {
      const double *aik = ta ? a->blk[k * nb + i] : a->blk[i * nb + k];
      if (!aik) continue;
      for (int j = 0; j < nb; j++) {
        const double *bkj = tb ? b->blk[j * nb + k] : b->blk[k * nb + j];
        if (!bkj) continue;
        double **xij = &x->blk[i * nb + j];
        if (!*xij) {
          *xij = (double *)calloc((size_t)bs * bs, sizeof(double));
          if (!*xij) {
            cx->oom = 1;
            return x;
          }
        }
        cx->triples++;
        double *c = *xij;
        for (int r = 0; r < bs; r++)
          for (int kk = 0; kk < bs; kk++) {
            double av = ta ? aik[kk * bs + r] : aik[r * bs + kk];
            for (int q = 0; q < bs; q++)
              c[r * bs + q] += av * (tb ? bkj[q * bs + kk] : bkj[kk * bs + q]);
          }
      }
    }
  if (leaf_is_empty(m, x)) {
    free_node(m, x);
    return NULL;
  }
  return x;
}

/* Algorithm 2 on temporaries: consumes x and y, returns their sum. */
static orc_node *add(const orc_matrix *m, orc_node *x, orc_node *y, int level) {
  if (x && y) {
    if (level == m->depth) {
      int64_t nn = (int64_t)m->leaf_nb * m->leaf_nb, bb = (int64_t)m->bs * m->bs;
      for (int64_t t = 0; t < nn; t++) {
        if (!y->blk[t]) continue;
        if (!x->blk[t]) {
          x->blk[t] = y->blk[t];
        } else {
          for (int64_t e = 0; e < bb; e++) x->blk[t][e] += y->blk[t][e];
          free(y->blk[t]);
        }
        y->blk[t] = NULL;
      }
    } else {
      for (int c = 0; c < 4; c++) {
        x->child[c] = add(m, x->child[c], y->child[c], level + 1);
        y->child[c] = NULL;
      }
    }
    free_node(m, y);
    return x;
  }
  if (x) return x;
  if (y) return y;
  return NULL;
}

/* Algorithm 1. */
static orc_node *multiply(const orc_matrix *m, const orc_node *a, const orc_node *b, int level,
                          orc_ctx *cx) {
  if (!a || !b) return NULL; /* fallback: C = NIL */
  if (cx->tasks) cx->tasks[level]++;
  if (level == m->depth) return leaf_multiply(m, a, b, cx);
  orc_node *c = new_node(m, 0); /* createFromIds */
  if (!c) {
    cx->oom = 1;
    return NULL;
  }
  /* child (r, c) of op(X) is child (r, c) of X, or child (c, r) if X enters
   * transposed */
#define OPA(r, c) a->child[cx->ta ? 2 * (c) + (r) : 2 * (r) + (c)]
#define OPB(r, c) b->child[cx->tb ? 2 * (c) + (r) : 2 * (r) + (c)]
  int any = 0;
  for (int mm = 0; mm < 2; mm++)
    for (int n = 0; n < 2; n++) {
      orc_node *y1 = multiply(m, OPA(mm, 0), OPB(0, n), level + 1, cx);
      orc_node *y2 = multiply(m, OPA(mm, 1), OPB(1, n), level + 1, cx);
      c->child[2 * mm + n] = add(m, y1, y2, level + 1);
      any |= c->child[2 * mm + n] != NULL;
    }
#undef OPA
#undef OPB
  if (!any) {
    free_node(m, c);
    return NULL;
  }
  return c;
}

/* Remove exactly-zero product blocks, then empty leaves and nodes. */
static orc_node *drop_zero(const orc_matrix *m, orc_node *n, int level) {
  if (!n) return NULL;
  if (level == m->depth) {
    for (int64_t t = 0; t < (int64_t)m->leaf_nb * m->leaf_nb; t++)
      if (n->blk[t] && block_is_zero(n->blk[t], m->bs)) {
        free(n->blk[t]);
        n->blk[t] = NULL;
      }
    if (leaf_is_empty(m, n)) {
      free_node(m, n);
      return NULL;
    }
    return n;
  }
  int any = 0;
  for (int c = 0; c < 4; c++) {
    n->child[c] = drop_zero(m, n->child[c], level + 1);
    any |= n->child[c] != NULL;
  }
  if (!any) {
    free_node(m, n);
    return NULL;
  }
  return n;
}

/* C = op(A)*op(B), op(X) = X or X^T (ta, tb).  tasks (optional) receives the
 * multiply-task count of each level 0..depth; triples receives the number of
 * leaf block products. */
orc_matrix *orc_multiply_t(const orc_matrix *A, int ta, const orc_matrix *B, int tb,
                           int64_t *tasks, int64_t *triples, int *status) {
  *status = ORC_OK;
  if (!A || !B) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  int64_t ar = ta ? A->ncols : A->nrows, ac = ta ? A->nrows : A->ncols;
  int64_t br = tb ? B->ncols : B->nrows, bc = tb ? B->nrows : B->ncols;
  if (ac != br) {
    *status = ORC_ERR_DIM_MISMATCH;
    return NULL;
  }
  if (A->bs != B->bs) {
    *status = ORC_ERR_BLOCKSIZE;
    return NULL;
  }
  if (A->L != B->L || A->leaf_nb != B->leaf_nb) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  orc_matrix *C = alloc_matrix(ar, bc, A->bs, A->L, A->leaf_nb);
  if (!C) {
    *status = ORC_ERR_OOM;
    return NULL;
  }
  orc_ctx cx = {tasks, 0, 0, ta != 0, tb != 0};
  if (tasks) memset(tasks, 0, sizeof(int64_t) * (size_t)(A->depth + 1));
  C->root = multiply(C, A->root, B->root, 0, &cx);
  if (triples) *triples = cx.triples;
  if (cx.oom) {
    *status = ORC_ERR_OOM;
    orc_free(C);
    return NULL;
  }
  C->root = drop_zero(C, C->root, 0);
  return C;
}

orc_matrix *orc_multiply(const orc_matrix *A, const orc_matrix *B, int64_t *tasks,
                         int64_t *triples, int *status) {
  return orc_multiply_t(A, 0, B, 0, tasks, triples, status);
}

/* Deep copy of a subtree (the add below consumes its inputs). */
static orc_node *copy_node(const orc_matrix *m, const orc_node *n, int level, int *oom) {
  if (!n) return NULL;
  orc_node *x = new_node(m, level == m->depth);
  if (!x) {
    *oom = 1;
    return NULL;
  }
  if (level == m->depth) {
    size_t bb = (size_t)m->bs * m->bs * sizeof(double);
    for (int64_t t = 0; t < (int64_t)m->leaf_nb * m->leaf_nb; t++) {
      if (!n->blk[t]) continue;
      x->blk[t] = (double *)malloc(bb);
      if (!x->blk[t]) {
        *oom = 1;
        return x;
      }
      memcpy(x->blk[t], n->blk[t], bb);
    }
    return x;
  }
  for (int c = 0; c < 4; c++) x->child[c] = copy_node(m, n->child[c], level + 1, oom);
  return x;
}

/* C = A + B by Algorithm 2 (on copies of the operands), exactly-zero sums
 * removed. */
orc_matrix *orc_add(const orc_matrix *A, const orc_matrix *B, int *status) {
  *status = ORC_OK;
  if (!A || !B) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  if (A->nrows != B->nrows || A->ncols != B->ncols) {
    *status = ORC_ERR_DIM_MISMATCH;
    return NULL;
  }
  if (A->bs != B->bs) {
    *status = ORC_ERR_BLOCKSIZE;
    return NULL;
  }
  if (A->L != B->L || A->leaf_nb != B->leaf_nb) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  orc_matrix *C = alloc_matrix(A->nrows, A->ncols, A->bs, A->L, A->leaf_nb);
  if (!C) {
    *status = ORC_ERR_OOM;
    return NULL;
  }
  int oom = 0;
  orc_node *x = copy_node(C, A->root, 0, &oom);
  orc_node *y = copy_node(C, B->root, 0, &oom);
  C->root = add(C, x, y, 0);
  if (oom) {
    *status = ORC_ERR_OOM;
    orc_free(C);
    return NULL;
  }
  C->root = drop_zero(C, C->root, 0);
  return C;
}

/* ------------------------------------------------------ symmetric storage */
/* A symmetric matrix is given by its upper triangle of blocks (I <= J), the
 * diagonal blocks in full (Sec. 3.3, symmetric task types).  The symmetric
 * results are defined plainly: the full matrix S (each strictly-upper block
 * also placed, transposed, at its mirror position), the ordinary product by
 * Algorithm 1, and the blocks with I <= J of that product. */

/* Slot of leaf block (I, J), creating the path; NULL on OOM. */
static double **block_slot(orc_matrix *m, int64_t I, int64_t J) {
  orc_node **slot = &m->root;
  for (int level = 0; level <= m->depth; level++) {
    if (!*slot) {
      *slot = new_node(m, level == m->depth);
      if (!*slot) return NULL;
    }
    if (level == m->depth) break;
    int shift = m->L - level - 1;
    slot = &(*slot)->child[2 * ((I >> shift) & 1) + ((J >> shift) & 1)];
  }
  int64_t mask = m->leaf_nb - 1;
  return &(*slot)->blk[(I & mask) * m->leaf_nb + (J & mask)];
}

static int mirror_into(orc_matrix *F, const orc_matrix *U, const orc_node *n, int level,
                       int64_t I0, int64_t J0) {
  if (!n) return ORC_OK;
  int bs = U->bs;
  size_t bb = (size_t)bs * bs;
  if (level == U->depth) {
    for (int i = 0; i < U->leaf_nb; i++)
      for (int j = 0; j < U->leaf_nb; j++) {
        const double *b = n->blk[i * U->leaf_nb + j];
        if (!b) continue;
        int64_t I = I0 * U->leaf_nb + i, J = J0 * U->leaf_nb + j;
        if (I > J) return ORC_ERR_OUT_OF_RANGE; /* not upper-triangle storage */
        double **d = block_slot(F, I, J);
        if (!d || !(*d = (double *)malloc(bb * sizeof(double)))) return ORC_ERR_OOM;
        memcpy(*d, b, bb * sizeof(double));
        if (I < J) {
          double **t = block_slot(F, J, I);
          if (!t || !(*t = (double *)malloc(bb * sizeof(double)))) return ORC_ERR_OOM;
          for (int r = 0; r < bs; r++)
            for (int c = 0; c < bs; c++) (*t)[r * bs + c] = b[c * bs + r];
        }
      }
    return ORC_OK;
  }
  for (int c = 0; c < 4; c++) {
    int st = mirror_into(F, U, n->child[c], level + 1, 2 * I0 + (c >> 1), 2 * J0 + (c & 1));
    if (st) return st;
  }
  return ORC_OK;
}

/* The full symmetric matrix of an upper-triangle-stored one. */
orc_matrix *orc_sym_full(const orc_matrix *U, int *status) {
  *status = ORC_OK;
  if (!U) {
    *status = ORC_ERR_INVALID_ARG;
    return NULL;
  }
  if (U->nrows != U->ncols) {
    *status = ORC_ERR_DIM_MISMATCH;
    return NULL;
  }
  orc_matrix *F = alloc_matrix(U->nrows, U->ncols, U->bs, U->L, U->leaf_nb);
  if (!F) {
    *status = ORC_ERR_OOM;
    return NULL;
  }
  int st = mirror_into(F, U, U->root, 0, 0, 0);
  if (st) {
    *status = st;
    orc_free(F);
    return NULL;
  }
  return F;
}

/* Remove blocks with I > J (and nodes left empty). */
static orc_node *keep_upper(const orc_matrix *m, orc_node *n, int level, int64_t I0, int64_t J0) {
  if (!n) return NULL;
  if (level == m->depth) {
    for (int i = 0; i < m->leaf_nb; i++)
      for (int j = 0; j < m->leaf_nb; j++) {
        double **b = &n->blk[i * m->leaf_nb + j];
        if (*b && I0 * m->leaf_nb + i > J0 * m->leaf_nb + j) {
          free(*b);
          *b = NULL;
        }
      }
    if (leaf_is_empty(m, n)) {
      free_node(m, n);
      return NULL;
    }
    return n;
  }
  int any = 0;
  for (int c = 0; c < 4; c++) {
    n->child[c] = keep_upper(m, n->child[c], level + 1, 2 * I0 + (c >> 1), 2 * J0 + (c & 1));
    any |= n->child[c] != NULL;
  }
  if (!any) {
    free_node(m, n);
    return NULL;
  }
  return n;
}

/* C = A^2 for symmetric A (upper-triangle storage in and out). */
orc_matrix *orc_sym_square(const orc_matrix *U, int *status) {
  orc_matrix *F = orc_sym_full(U, status);
  if (!F) return NULL;
  orc_matrix *C = orc_multiply_t(F, 0, F, 0, NULL, NULL, status);
  orc_free(F);
  if (C) C->root = keep_upper(C, C->root, 0, 0, 0);
  return C;
}

/* Symmetric rank-k: C = A A^T (trans = 0) or A^T A (trans = 1), upper
 * triangle. */
orc_matrix *orc_syrk(const orc_matrix *A, int trans, int *status) {
  orc_matrix *C = orc_multiply_t(A, trans != 0, A, trans == 0, NULL, NULL, status);
  if (C) C->root = keep_upper(C, C->root, 0, 0, 0);
  return C;
}

/* C = S B (side 0, S = A symmetric) or C = A S (side 1, S = B symmetric). */
orc_matrix *orc_symm(const orc_matrix *A, const orc_matrix *B, int side, int *status) {
  orc_matrix *F = orc_sym_full(side == 0 ? A : B, status);
  if (!F) return NULL;
  orc_matrix *C = side == 0 ? orc_multiply_t(F, 0, B, 0, NULL, NULL, status)
                            : orc_multiply_t(A, 0, F, 0, NULL, NULL, status);
  orc_free(F);
  return C;
}

static const double *find_block(const orc_matrix *m, int64_t I, int64_t J);
int64_t orc_nblocks(const orc_matrix *m);

/* --------------------------------------------------- Frobenius norms */
/* Per-node Frobenius norms (Sec. 7 names them as extra quadtree information)
 * and truncation with a bound on the Frobenius norm of the error (Sec. 6.2
 * truncates the overlap matrix that way).  Squared norms are summed in one
 * fixed order so that both implementations round identically: a block's
 * squared norm is the sum over rows, in ascending order, of the row sums of
 * squares in ascending column order; a node's is the sum of its children's in
 * child order 0..3.  (The file is compiled without FMA contraction.) */
double orc_block_norm2(const double *b, int bs) {
  double t = 0.0;
  for (int r = 0; r < bs; r++) {
    double row = 0.0;
    for (int c = 0; c < bs; c++) {
      double sq = b[r * bs + c] * b[r * bs + c];
      row = row + sq;
    }
    t = t + row;
  }
  return t;
}

static double node_norm2(const orc_matrix *m, const orc_node *n, int level, int want_level,
                         int64_t I0, int64_t J0, int32_t *I, int32_t *J, double *v,
                         int64_t *pos) {
  double t;
  if (level == m->depth) {
    t = orc_block_norm2(n->blk[0], m->bs); /* leaf_nb == 1: one block per leaf */
  } else {
    t = 0.0;
    for (int c = 0; c < 4; c++)
      if (n->child[c])
        t = t + node_norm2(m, n->child[c], level + 1, want_level, 2 * I0 + (c >> 1),
                           2 * J0 + (c & 1), I, J, v, pos);
  }
  if (level == want_level) {
    if (I) {
      I[*pos] = (int32_t)I0;
      J[*pos] = (int32_t)J0;
      v[*pos] = t;
    }
    (*pos)++;
  }
  return t;
}

/* Squared norms of the nodes at `height` above the blocks (0 = the blocks)
 * of a tree built with one block per leaf, in depth-first child order, with
 * their coordinates at that height.  Returns the node count (arrays may be
 * NULL), or -1 if the tree has multi-block leaves or height is out of range. */
int64_t orc_node_norms2(const orc_matrix *m, int height, int32_t *I, int32_t *J, double *v) {
  if (m->leaf_nb != 1 || height < 0 || height > m->depth) return -1;
  int64_t pos = 0;
  if (m->root) node_norm2(m, m->root, 0, m->depth - height, 0, 0, I, J, v, &pos);
  return pos;
}

static uint64_t morton2(uint64_t I, uint64_t J) {
  uint64_t k = 0;
  for (int b = 0; b < 32; b++) k |= (((I >> b) & 1) << (2 * b + 1)) | (((J >> b) & 1) << (2 * b));
  return k;
}

typedef struct {
  double n2;
  uint64_t key;
  int64_t I, J;
} orc_nrm;

static int cmp_nrm(const void *a, const void *b) {
  const orc_nrm *x = (const orc_nrm *)a, *y = (const orc_nrm *)b;
  /* NaN sorts last */
  int xn = x->n2 != x->n2, yn = y->n2 != y->n2;
  if (xn != yn) return xn - yn;
  if (!xn && x->n2 != y->n2) return x->n2 < y->n2 ? -1 : 1;
  return (x->key > y->key) - (x->key < y->key);
}

static void collect_nrm(const orc_matrix *m, const orc_node *n, int level, int64_t I0, int64_t J0,
                        orc_nrm *out, int64_t *pos) {
  if (!n) return;
  if (level == m->depth) {
    for (int i = 0; i < m->leaf_nb; i++)
      for (int j = 0; j < m->leaf_nb; j++) {
        const double *b = n->blk[i * m->leaf_nb + j];
        if (!b) continue;
        int64_t I = I0 * m->leaf_nb + i, J = J0 * m->leaf_nb + j;
        out[*pos].n2 = orc_block_norm2(b, m->bs);
        out[*pos].key = morton2((uint64_t)I, (uint64_t)J);
        out[*pos].I = I;
        out[*pos].J = J;
        (*pos)++;
      }
    return;
  }
  for (int c = 0; c < 4; c++)
    collect_nrm(m, n->child[c], level + 1, 2 * I0 + (c >> 1), 2 * J0 + (c & 1), out, pos);
}

/* Truncation: remove the longest run of blocks, in ascending order of squared
 * norm (ties: ascending Morton key), whose squared norms sum to at most tau^2.
 * The sum is taken in integers so that the decision is exact: with
 * 2^e = 2^(floor(log2 tau^2) - 63), every squared norm s is rounded up to
 * Q = ceil(s / 2^e) (saturating at 2^64 - 1) and the run is the longest prefix
 * whose Q add up to at most T = floor(tau^2 / 2^e) in exact (saturating)
 * 64-bit arithmetic; so sum(s) <= sum(Q) 2^e <= tau^2 holds rigorously.
 * tau <= 0 (or tau^2 == 0) removes nothing; NaN norms are never removed.
 * *removed receives the count and *bound the value sum(Q) 2^e. */
orc_matrix *orc_truncate(const orc_matrix *A, double tau, int64_t *removed, double *bound,
                         int *status) {
  *status = ORC_OK;
  *removed = 0;
  *bound = 0.0;
  int64_t n = orc_nblocks(A), pos = 0;
  orc_nrm *it = (orc_nrm *)malloc(sizeof(orc_nrm) * (size_t)(n > 0 ? n : 1));
  if (!it) {
    *status = ORC_ERR_OOM;
    return NULL;
  }
  collect_nrm(A, A->root, 0, 0, 0, it, &pos);
  qsort(it, (size_t)n, sizeof(orc_nrm), cmp_nrm);
  double t2 = tau * tau;
  int64_t k = 0;
  if (tau > 0.0 && isinf(t2)) { /* everything but NaN-norm blocks */
    while (k < n && it[k].n2 == it[k].n2) k++;
    *bound = t2;
  } else if (tau > 0.0 && t2 > 0.0) {
    int ex;
    frexp(t2, &ex); /* t2 = f 2^ex, f in [0.5, 1): floor(log2 t2) = ex - 1 */
    const int e = ex - 1 - 63;
    const uint64_t T = (uint64_t)floor(ldexp(t2, -e)); /* in [2^63, 2^64) */
    uint64_t acc = 0;
    for (; k < n; k++) {
      if (it[k].n2 != it[k].n2) break; /* NaN */
      const double q = ceil(ldexp(it[k].n2, -e));
      const uint64_t Q = q >= 18446744073709551616.0 ? UINT64_MAX : (uint64_t)q;
      const uint64_t nxt = acc + Q < acc ? UINT64_MAX : acc + Q;
      if (nxt > T) break;
      acc = nxt;
    }
    *bound = ldexp((double)acc, e);
  }
  *removed = k;
  /* rebuild without the removed blocks */
  orc_matrix *C = alloc_matrix(A->nrows, A->ncols, A->bs, A->L, A->leaf_nb);
  if (!C) {
    free(it);
    *status = ORC_ERR_OOM;
    return NULL;
  }
  size_t bb = (size_t)A->bs * A->bs;
  for (int64_t t = k; t < n; t++) {
    const double *src = find_block(A, it[t].I, it[t].J);
    double **d = block_slot(C, it[t].I, it[t].J);
    if (!d || !(*d = (double *)malloc(bb * sizeof(double)))) {
      free(it);
      orc_free(C);
      *status = ORC_ERR_OOM;
      return NULL;
    }
    memcpy(*d, src, bb * sizeof(double));
  }
  free(it);
  return C;
}

/* ---------------------------------------------------------------- output */
static int64_t count_blocks(const orc_matrix *m, const orc_node *n, int level) {
  if (!n) return 0;
  int64_t s = 0;
  if (level == m->depth) {
    for (int64_t t = 0; t < (int64_t)m->leaf_nb * m->leaf_nb; t++) s += n->blk[t] != NULL;
    return s;
  }
  for (int c = 0; c < 4; c++) s += count_blocks(m, n->child[c], level + 1);
  return s;
}

int64_t orc_nblocks(const orc_matrix *m) { return m ? count_blocks(m, m->root, 0) : 0; }

int orc_depth(const orc_matrix *m) { return m->depth; }

typedef struct {
  int64_t key;
  const double *p;
} orc_item;

static void collect(const orc_matrix *m, const orc_node *n, int level, int64_t I0, int64_t J0,
                    orc_item *out, int64_t *pos) {
  if (!n) return;
  if (level == m->depth) {
    for (int i = 0; i < m->leaf_nb; i++)
      for (int j = 0; j < m->leaf_nb; j++) {
        const double *b = n->blk[i * m->leaf_nb + j];
        if (!b) continue;
        int64_t I = I0 * m->leaf_nb + i, J = J0 * m->leaf_nb + j;
        out[*pos].key = (I << 32) | J;
        out[*pos].p = b;
        (*pos)++;
      }
    return;
  }
  for (int c = 0; c < 4; c++)
    collect(m, n->child[c], level + 1, 2 * I0 + (c >> 1), 2 * J0 + (c & 1), out, pos);
}

static int cmp_item(const void *a, const void *b) {
  int64_t x = ((const orc_item *)a)->key, y = ((const orc_item *)b)->key;
  return (x > y) - (x < y);
}

/* Stored blocks in canonical row-major (I, J) order.  Buffers hold
 * orc_nblocks(m) entries. */
int orc_to_blocks(const orc_matrix *m, int32_t *brow, int32_t *bcol, double *vals) {
  int64_t n = orc_nblocks(m), pos = 0;
  orc_item *it = (orc_item *)malloc(sizeof(orc_item) * (size_t)(n > 0 ? n : 1));
  if (!it) return ORC_ERR_OOM;
  collect(m, m->root, 0, 0, 0, it, &pos);
  qsort(it, (size_t)n, sizeof(orc_item), cmp_item);
  size_t bb = (size_t)m->bs * m->bs;
  for (int64_t t = 0; t < n; t++) {
    brow[t] = (int32_t)(it[t].key >> 32);
    bcol[t] = (int32_t)(it[t].key & 0xFFFFFFFF);
    memcpy(vals + (size_t)t * bb, it[t].p, bb * sizeof(double));
  }
  free(it);
  return ORC_OK;
}

/* --------------------------------------------- single block, by definition */
static const double *find_block(const orc_matrix *m, int64_t I, int64_t J) {
  const orc_node *n = m->root;
  for (int level = 0; level < m->depth && n; level++) {
    int shift = m->L - level - 1;
    n = n->child[2 * ((I >> shift) & 1) + ((J >> shift) & 1)];
  }
  if (!n) return NULL;
  int64_t mask = m->leaf_nb - 1;
  return n->blk[(I & mask) * m->leaf_nb + (J & mask)];
}

/* C_IJ = sum_K A_IK B_KJ over the stored blocks (the plain definition of one
 * product block, for sampled checks of large products).  Returns 1 if some K
 * contributes, 0 if the block is structurally NIL. */
int orc_block_product(const orc_matrix *A, const orc_matrix *B, int64_t I, int64_t J,
                      double *out) {
  int bs = A->bs, any = 0;
  memset(out, 0, sizeof(double) * (size_t)bs * bs);
  int64_t kb = (A->ncols + bs - 1) / bs;
  for (int64_t K = 0; K < kb; K++) {
    const double *a = find_block(A, I, K);
    if (!a) continue;
    const double *b = find_block(B, K, J);
    if (!b) continue;
    any = 1;
    for (int r = 0; r < bs; r++)
      for (int kk = 0; kk < bs; kk++) {
        double av = a[r * bs + kk];
        for (int q = 0; q < bs; q++) out[r * bs + q] += av * b[kk * bs + q];
      }
  }
  return any;
}
