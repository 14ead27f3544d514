/*
 * bsm.h -- block-sparse matrix-matrix multiply C = A*B over a sparse quadtree,
 * single GB300 GPU (sm_103a).
 *
 * Method: Rubensson & Rudberg, "Locality-aware parallel block-sparse
 * matrix-matrix multiplication using the Chunks and Tasks programming model"
 * (arXiv 1501.07800).  A matrix is a quadtree whose zero submatrices are NIL at
 * any level (Sec. 3.1) and whose leaves hold dense bs x bs blocks (Sec. 4.1).
 * The product recurses over pairs of non-NIL children (Algorithm 1); sums of
 * partial products follow Algorithm 2.  Here the tree is stored on the device
 * as Morton-ordered block keys plus per-level child bitmasks, the recursion
 * runs level by level over all node pairs at once, and every C block is
 * computed by a single owner with no atomics.
 *
 * Conventions shared by every call
 *   - All calls return a bsm_status; no exception crosses this boundary.
 *   - Work is ordered on `stream` (a cudaStream_t passed as void*; NULL = the
 *     legacy default stream).  Calls that must size an output (build, multiply)
 *     synchronise `stream` before returning; the data of a returned handle is
 *     ready for any later work on the same stream.
 *   - Argument errors are detected before any device work is queued and leave
 *     outputs untouched (output handles set to NULL).  Errors found in the data
 *     on the device (a block coordinate out of range, a duplicate key) are
 *     reported by the same call after it synchronises.
 *   - Block payloads are row-major bs x bs float64.  Matrix sides need not be
 *     multiples of bs: edge blocks are stored full size and their entries
 *     outside the matrix must be zero (the quadtree pads the matrix to 2^L
 *     blocks per side: the uniform power-of-two blocking of Sec. 3.1).
 *   - A block is "zero" when every entry compares equal to 0.0 (so -0.0 is
 *     zero and NaN is not).  Zero blocks are never stored (Sec. 4.1).
 *   - A handle's block structure is fixed at creation (its values change only
 *     through bsm_update_values); handles are owned by the caller, freed with
 *     bsm_destroy, and bound to the device that was current at creation.
 */
#ifndef BSM_H
#define BSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsm_matrix_s *bsm_matrix;
typedef struct bsm_plan_s *bsm_plan;

typedef enum {
  BSM_OK = 0,
  BSM_ERR_INVALID_ARG = -1,      /* NULL pointer, negative size, bad option */
  BSM_ERR_DIM_MISMATCH = -2,     /* A.ncols != B.nrows */
  BSM_ERR_BLOCKSIZE = -3,        /* unsupported bs, or A.bs != B.bs */
  BSM_ERR_OUT_OF_RANGE = -4,     /* a block coordinate outside the matrix */
  BSM_ERR_DUPLICATE = -5,        /* the same (I, J) listed twice */
  BSM_ERR_OOM = -6,              /* device allocation failed */
  BSM_ERR_CUDA = -7,             /* a CUDA runtime error */
  BSM_ERR_TIMEOUT = -8,          /* a bounded device wait gave up */
  BSM_ERR_BUFFER_TOO_SMALL = -9, /* caller buffer smaller than the result */
  BSM_ERR_UNSUPPORTED = -10      /* a valid request the library does not support */
} bsm_status;

typedef enum {
  BSM_FP64 = 0,       /* FP64 tensor-core (DMMA) products, FP64 accumulation */
  BSM_SPLIT_BF16 = 1, /* FP64 blocks split into BF16 slices (7-bit digits) on tcgen05 */
  BSM_SPLIT_FP8 = 2   /* FP64 blocks split into FP8 E4M3 slices (4-bit digits) on tcgen05 */
} bsm_precision;

/* Options of one product (NULL = all defaults: FP64). */
typedef struct {
  int prec;   /* bsm_precision */
  int slices; /* split modes: digit slices per operand, 0 = default; BF16: 1..8
                 (default 7, 49-bit fixed point per row/column), FP8: 2, 3, 4,
                 6, 8 or 12 (default 6, 24 bits) */
  int flags;  /* 0, BSM_FLAG_AUTOTUNE (bsm_plan_create only), or
                 BSM_FLAG_TRANS_A / BSM_FLAG_TRANS_B (bsm_multiply only) */
  int bs;     /* leaf size to compute at (bsm_multiply, bsm_multiply_batched,
                 bsm_plan_create): 0 = the operands' own, which must then be
                 equal; 16, 32 or 64 = operands of another size are re-cut to
                 it exactly (bsm_reblock; plans refresh their re-cut copies
                 at every execution) and C has this size; the other calls
                 taking options require 0 (INVALID_ARG otherwise) */
} bsm_mult_opts;

/* bsm_plan_create: measure candidate launch configurations and keep the
 * fastest (cached per product class for the process). */
#define BSM_FLAG_AUTOTUNE 1
/* bsm_plan_create: also choose the leaf block size by timing the product on
 * re-blocked copies of the operands (FP64: the operands' size and the finer
 * ones -- coarser blocks only add zero-fill flops at the FP64 rate; split
 * modes: 16 and 32).  The plan then copies the operands' current values into
 * its re-blocked copies at every execution and returns C in the operands'
 * block size. */
#define BSM_FLAG_AUTOTUNE_BS 8
/* bsm_multiply: use A^T (resp. B^T) in place of A (resp. B), the transposed
 * multiplication task types C = A^T B, A B^T, A^T B^T of Sec. 3.2. */
#define BSM_FLAG_TRANS_A 2
#define BSM_FLAG_TRANS_B 4

/* Supported leaf block sides. */
#define BSM_BS_MIN 16
#define BSM_BS_MAX 64

/*
 * bsm_build -- create a matrix from a COO list of dense leaf blocks
 * (the "Matrix" chunk hierarchy of Sec. 3.1 built from the leaves up).
 *
 *   nrows, ncols  matrix size in elements (>= 0)
 *   bs            leaf block side: 16, 32 or 64
 *   nblk          number of listed blocks (>= 0)
 *   brow, bcol    int32[nblk] block coordinates, 0 <= brow < ceil(nrows/bs),
 *                 0 <= bcol < ceil(ncols/bs); any order; duplicates rejected
 *   vals          float64[nblk][bs][bs], block t row-major at vals + t*bs*bs
 *   on_device     0: the three arrays are host memory (copied in this call;
 *                 pinned, device-mapped arrays -- brow/bcol 4-byte and vals
 *                 16-byte aligned in the device's view -- are read in place
 *                 by the build kernels over the host link instead, with no
 *                 staging buffer and no copy-engine upload);
 *                 1: they are device memory of the current device (vals
 *                 16-byte aligned, brow/bcol 4-byte aligned)
 *   stream        cudaStream_t or NULL
 *   out           receives the new handle (NULL on error)
 *
 * Exactly-zero blocks are dropped.  The library copies the inputs; the caller
 * may reuse its buffers when the call returns.
 * Errors: INVALID_ARG (also: misaligned device arrays), BLOCKSIZE,
 * OUT_OF_RANGE, DUPLICATE, OOM, CUDA.
 */
bsm_status bsm_build(int64_t nrows, int64_t ncols, int bs, int64_t nblk, const int32_t *brow,
                     const int32_t *bcol, const double *vals, int on_device, void *stream,
                     bsm_matrix *out);

/*
 * bsm_multiply -- C = A*B (Algorithm 1 with the leaf product of Sec. 4.1).
 *
 * Symbolic phase: node pairs are expanded level by level from the roots down
 * to the leaf blocks, skipping NIL children, giving every C block its ordered
 * list of (A block, B block) products.  Numeric phase: each C block is summed
 * by one owner.  C blocks whose entries are all exactly zero are removed.
 * The depth of the product is the larger depth of A and B.
 *
 *   A, B   operands, op(A).ncols == op(B).nrows, same bs, where op(X) is X,
 *          or X^T when opts->flags holds BSM_FLAG_TRANS_A / _B
 *   C      receives the new handle (NULL on error); C.nrows = op(A).nrows,
 *          C.ncols = op(B).ncols, C.bs = A.bs
 *   opts   NULL or options (precision mode, slice count, transposition)
 * A transposed operand is materialised (bsm_transpose) for the duration of
 * the call.
 * Products too large for one pass of the symbolic phase are expanded and
 * computed in consecutive Morton ranges of C (see bsm_last_chunks).
 * Errors: INVALID_ARG, DIM_MISMATCH, BLOCKSIZE, OOM, CUDA, TIMEOUT,
 * UNSUPPORTED (one quadrant of one C node with more than 2^31 block pairs on
 * a level; split mode with bs 64).
 */
bsm_status bsm_multiply(bsm_matrix A, bsm_matrix B, bsm_matrix *C, const bsm_mult_opts *opts,
                        void *stream);

/*
 * bsm_multiply_range -- the C blocks of C = A*B whose Morton keys lie in
 * [key_lo, key_hi) (key of block (I, J): bit 2b+1 = bit b of I, bit 2b = bit
 * b of J).  Contiguous key ranges are quadtree subtrees and unions of them, so
 * disjoint ranges partition C with no block computed twice: the shards of a
 * product split over several GPUs.  The symbolic phase prunes every C node
 * outside the range.  Blocks are computed exactly as by bsm_multiply (same
 * values bit for bit); C has the full product's dimensions.
 * Errors: as bsm_multiply; INVALID_ARG if key_hi <= key_lo; UNSUPPORTED for a
 * split mode that re-cuts to wider blocks (E4M3 with bs 16).
 */
bsm_status bsm_multiply_range(bsm_matrix A, bsm_matrix B, uint64_t key_lo, uint64_t key_hi,
                              bsm_matrix *C, const bsm_mult_opts *opts, void *stream);

/*
 * bsm_transpose -- T = A^T as a new handle (keys with row and column swapped,
 * every block transposed; Sec. 3.2 transposed task types).
 *   A    input handle (unchanged)
 *   out  receives the new handle (NULL on error); out.nrows = A.ncols,
 *        out.ncols = A.nrows, same bs and depth
 * Stream-ordered; the caller owns the result (bsm_destroy).
 * Errors: INVALID_ARG, OOM, CUDA.
 */
bsm_status bsm_transpose(bsm_matrix A, bsm_matrix *out, void *stream);

/*
 * bsm_add -- C = A + B (Algorithm 2 with the leaf add): a block present in
 * both operands is the sum of the two, a block present in one is copied, and
 * a block present in neither is NIL.  Sums that are exactly zero in every
 * entry are removed, as for products.
 *   A, B  operands of equal dimensions and block size (unchanged)
 *   out   receives the new handle (NULL on error); depth = max of the two
 * Stream-ordered; the caller owns the result (bsm_destroy).
 * Errors: INVALID_ARG, DIM_MISMATCH, BLOCKSIZE, OOM, CUDA, UNSUPPORTED
 * (more than 2^31 - 1 blocks in A and B together).
 */
bsm_status bsm_add(bsm_matrix A, bsm_matrix B, bsm_matrix *out, void *stream);

/*
 * Symmetric matrices (Sec. 3.3, additional task types for the symmetric
 * matrix square) are stored as their upper triangle of blocks: only blocks
 * with I <= J, diagonal blocks in full.  Symmetric results are returned the
 * same way.  Operands in this storage must be square and hold no block below
 * the diagonal (else BSM_ERR_DIM_MISMATCH / BSM_ERR_OUT_OF_RANGE).  The
 * symmetric results are computed from the ordinary symbolic recursion with
 * the C nodes below the diagonal skipped, so roughly half of the block
 * products of the full product are formed.  All are stream-ordered and
 * return a new handle the caller owns; opts as for bsm_multiply (no flags).
 * Errors: as bsm_multiply, plus OUT_OF_RANGE as above.
 */
#define BSM_SYM_LEFT 0  /* bsm_sym_multiply: A is the symmetric operand */
#define BSM_SYM_RIGHT 1 /* bsm_sym_multiply: B is the symmetric operand */

/* bsm_sym_square -- C = A^2, A symmetric: upper triangle of A*A. */
bsm_status bsm_sym_square(bsm_matrix A, bsm_matrix *C, const bsm_mult_opts *opts, void *stream);

/* bsm_syrk -- symmetric rank-k product, upper triangle of C = A A^T
 * (trans = 0) or C = A^T A (trans = 1); A is a general matrix. */
bsm_status bsm_syrk(bsm_matrix A, int trans, bsm_matrix *C, const bsm_mult_opts *opts,
                    void *stream);

/* bsm_sym_multiply -- C = A B (general result) where A (side = BSM_SYM_LEFT)
 * or B (side = BSM_SYM_RIGHT) is symmetric in upper-triangle storage. */
bsm_status bsm_sym_multiply(bsm_matrix A, bsm_matrix B, int side, bsm_matrix *C,
                            const bsm_mult_opts *opts, void *stream);

/* bsm_sym_to_full -- the full matrix (both triangles) of a symmetric matrix
 * in upper-triangle storage: each strictly-upper block also appears,
 * transposed, at its mirror position. */
bsm_status bsm_sym_to_full(bsm_matrix A, bsm_matrix *out, void *stream);

/*
 * bsm_reblock -- the same matrix cut into leaf blocks of side bs (16, 32 or
 * 64).  Splitting drops sub-blocks that are exactly zero; merging fills
 * absent sub-blocks with zeros.  Values are copied bit for bit.
 *   A    input handle (unchanged)
 *   out  receives the new handle (NULL on error)
 * Stream-ordered; the caller owns the result.  Errors: INVALID_ARG,
 * BLOCKSIZE, OOM, CUDA, UNSUPPORTED (more than 2^31 - 1 sub-blocks).
 */
bsm_status bsm_reblock(bsm_matrix A, int bs, bsm_matrix *out, void *stream);

/*
 * bsm_node_norms2 -- squared Frobenius norms of the quadtree nodes at a
 * height above the leaf blocks (0 = the blocks themselves; the per-node norms
 * of Sec. 7), in Morton order of the nodes, with the nodes' coordinates at
 * that height.  Summation order is fixed (rows ascending, each row's squares
 * in column order; a node sums its children in child order), each operation
 * rounded separately, so results are reproducible bit for bit.
 *   height     0 .. depth of the matrix
 *   norm2      float64[capacity] or NULL
 *   I, J       int32[capacity] or NULL: node row / column at that height
 *   n_inout    in: capacity; out: number of nodes at that height
 *   on_device  0: host buffers (the call synchronises `stream`); 1: device
 *              buffers (norm2 8-byte, I/J 4-byte aligned)
 * With all three buffers NULL only the count is returned.
 * Errors: INVALID_ARG, OUT_OF_RANGE (height), BUFFER_TOO_SMALL, OOM, CUDA.
 */
bsm_status bsm_node_norms2(bsm_matrix M, int height, double *norm2, int32_t *I, int32_t *J,
                           int64_t *n_inout, int on_device, void *stream);

/*
 * bsm_truncate -- remove small blocks so that the Frobenius norm of the
 * removed part is at most tau (the truncation of Sec. 6.2): the longest run
 * of blocks in ascending order of squared norm (ties: Morton order) whose
 * squared norms sum to at most tau^2.  The sum is decided exactly in integer
 * units 2^e = 2^(floor(log2 tau^2) - 63): each squared norm is rounded up to a
 * whole unit and the run stops before the integer sum passes tau^2, so the
 * removed squared norm never exceeds tau^2.  tau <= 0 removes nothing; blocks
 * whose norm is NaN are never removed.
 *   out      receives the new handle (caller owns it)
 *   removed  NULL or receives the number of removed blocks
 *   bound    NULL or receives the rounded-up removed squared norm (<= tau^2)
 * Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED (more than 2^31 - 1 blocks).
 */
bsm_status bsm_truncate(bsm_matrix M, double tau, bsm_matrix *out, int64_t *removed,
                        double *bound, void *stream);

/*
 * bsm_multiply_batched -- C[i] = A[i]*B[i] for n independent products.
 * Symbolic phases run per product; the numeric phase of all products runs as
 * one persistent launch over a single work list ordered by decreasing work.
 * Results are identical to n calls of bsm_multiply with the same options
 * (split products at a leaf size their kernels do not take -- 64, or 16 with
 * E4M3 digits -- run on operands re-cut to 32 and are cut back, as there).
 *   n          number of products (>= 0)
 *   A, B       arrays of n handles
 *   C          array of n handle slots, filled on success (all NULL on error)
 * Errors: as bsm_multiply.
 */
bsm_status bsm_multiply_batched(int n, const bsm_matrix *A, const bsm_matrix *B, bsm_matrix *C,
                                const bsm_mult_opts *opts, void *stream);

/*
 * bsm_to_blocks -- copy the stored blocks out in canonical row-major (I, J)
 * order.
 *   nblk_inout  in: capacity of the caller buffers in blocks;
 *               out: number of stored blocks
 *   brow, bcol  int32[capacity] or NULL
 *   vals        float64[capacity][bs][bs] or NULL
 *   on_device   0: host buffers (the call synchronises `stream`);
 *               1: device buffers of the handle's device (vals 16-byte
 *               aligned, brow/bcol 4-byte aligned);
 *               2: page-locked, device-mapped host buffers (cudaHostAlloc /
 *               cudaHostRegister with mapping; vals 16-byte aligned), written
 *               asynchronously: the blocks are gathered in 512 MB chunks into
 *               a device staging buffer, each chunk moved by the copy engine,
 *               on a library-owned stream of the greatest priority (one
 *               per device, so concurrent downloads run one after another)
 *               that starts after the work queued on `stream` and that
 *               `stream` waits for; the call returns with the work queued,
 *               so the transfer overlaps later kernels on other streams.  The
 *               caller synchronises `stream` before reading the buffers and
 *               keeps M alive until then (INVALID_ARG if a buffer is not
 *               such memory)
 * With all three buffers NULL the call only reports the block count.
 * Errors: INVALID_ARG, BUFFER_TOO_SMALL (count still reported), OOM, CUDA.
 */
bsm_status bsm_to_blocks(bsm_matrix M, int64_t *nblk_inout, int32_t *brow, int32_t *bcol,
                         double *vals, int on_device, void *stream);

/* bsm_info -- sizes of a handle; any output pointer may be NULL. */
bsm_status bsm_info(bsm_matrix M, int64_t *nrows, int64_t *ncols, int *bs, int64_t *nblk);

/*
 * bsm_level_counts -- nodes per quadtree level of a handle, root level first
 * (the NIL-free node sets whose pairings are the multiply tasks of Sec. 5.1).
 *   counts  int64[cap] receives counts for levels 0..L (L+1 values)
 *   nlev    receives L+1
 * Errors: INVALID_ARG, BUFFER_TOO_SMALL.
 */
bsm_status bsm_level_counts(bsm_matrix M, int64_t *counts, int cap, int *nlev);

/*
 * bsm_last_stats -- statistics of the last bsm_multiply on this thread:
 *   tasks    int64[cap]: multiply tasks (non-NIL node pairs) per level of the
 *            product tree, root level first (Sec. 5.1, C_l); may be NULL
 *   nlev     receives the number of levels
 *   triples  receives the number of leaf block products
 *   nc_sym   receives the number of C blocks before zero-block removal
 */
bsm_status bsm_last_stats(int64_t *tasks, int cap, int *nlev, int64_t *triples, int64_t *nc_sym);

/*
 * bsm_last_chunks -- number of Morton-range chunks the symbolic phase of the
 * last bsm_multiply on this thread delivered its task list in.  A product
 * whose expansion exceeds the per-level pair budget (2^30 pairs by default;
 * the environment variable BSM_SYM_BUDGET overrides it) is computed chunk by
 * chunk: halves of a level's C-node list, or the four quadrants of one node.
 */
bsm_status bsm_last_chunks(int *nchunks);

/*
 * bsm_set_timing -- per-phase CUDA-event timing of bsm_multiply on the calling
 * thread: 1 = on, 0 = off (default off; the environment variable
 * BSM_TIMING=1 turns it on for every thread).  Timing records CUDA events on
 * the product's stream and never waits for them, so a timed product runs as
 * an untimed one does; bsm_last_phase_ms waits for the last product's events
 * when it is called.
 */
bsm_status bsm_set_timing(int on);

/*
 * bsm_release_memory -- return the device memory the library keeps cached to
 * the driver.  The library allocates stream-ordered from two memory pools of
 * the current device -- the device's default pool, and a pool of its own for
 * allocations of 1 GiB and more, so that a large block freed by one product
 * is reused whole by the next -- and keeps freed memory in them, so that
 * repeated products reuse it without new driver allocations; memory cached
 * there is not available to other allocators (cudaMalloc, PyTorch's
 * allocator).  This call synchronises the current device, then releases every
 * cached byte of both pools not backing a live allocation (handles, plans and
 * their buffers stay valid).
 * Errors: CUDA if the synchronisation or the release fails.
 */
bsm_status bsm_release_memory(void);

/*
 * bsm_set_memory_limit -- cap the device memory the library's allocations
 * may hold in the current device's two pools: an allocation that would take
 * their in-use bytes above `bytes` fails with OOM, and the call
 * that needed it returns OOM after freeing what it had allocated.  0 removes
 * the cap (the default).  Process-wide.  Meant for callers that share the
 * device and for fault injection in tests.
 * bsm_memory_in_use -- the pools' bytes in use by live allocations (handles,
 * plans, work in flight); synchronises the current device first.
 * Errors: INVALID_ARG (NULL bytes), CUDA.
 */
bsm_status bsm_set_memory_limit(uint64_t bytes);
bsm_status bsm_memory_in_use(uint64_t *bytes);

/*
 * bsm_last_phase_ms -- results of the last timed bsm_multiply (or
 * bsm_multiply_batched) on this thread; waits for that product's events.
 *   ms        double[cap]: ms[0] symbolic phase, ms[1] numeric phase (the
 *             numeric kernel plus, in split modes, the slicing kernels),
 *             ms[2] zero-block removal and level build of C; may be NULL
 *   nphase    receives 3
 *   launches  receives the number of kernel launches the product issued
 *             (timed or not); may be NULL
 * Errors: BUFFER_TOO_SMALL if cap < 3 with ms != NULL.
 */
bsm_status bsm_last_phase_ms(double *ms, int cap, int *nphase, int64_t *launches);

/*
 * bsm_update_values -- replace the block values of a handle, keeping its
 * structure.  The COO list must name exactly the handle's stored blocks (any
 * order; same count, same coordinates); blocks may become all-zero and stay
 * stored.  Arguments as in bsm_build.  The caller may reuse its buffers when
 * the call returns.
 * Errors: INVALID_ARG (also: a different block set, misaligned device
 * arrays), OUT_OF_RANGE, OOM, CUDA.
 */
bsm_status bsm_update_values(bsm_matrix M, int64_t nblk, const int32_t *brow, const int32_t *bcol,
                             const double *vals, int on_device, void *stream);

/*
 * bsm_plan_create -- prepare repeated products C[i] = A[i]*B[i], i < n, whose
 * operand structures stay fixed.  The symbolic phases (Algorithm 1), the C
 * structures, a longest-first work list over all (product, C block) items and
 * all buffers are set up once; the numeric phase (with, in split mode, the
 * scaling and slicing of the current operand values) is captured into a CUDA
 * graph that bsm_plan_execute replays as one persistent launch.  With
 * BSM_FLAG_AUTOTUNE in opts->flags the plan times candidate launch
 * configurations (work order, work items per claim, CTAs per SM) and keeps
 * the fastest.  All operands must share one block size; split plans at a
 * leaf size their kernels do not take (64, or 16 with E4M3 digits) compute on
 * re-cut copies of the operands, refreshed at every execution, and return
 * results at the operands' size.  The plan reads A[i],
 * B[i] at every execution: they must outlive it (use bsm_update_values to
 * change their values).  One eager run of the numeric phase is part of the
 * creation.
 * Errors: INVALID_ARG, DIM_MISMATCH, BLOCKSIZE, OOM, CUDA, UNSUPPORTED.
 */
bsm_status bsm_plan_create(int n, const bsm_matrix *A, const bsm_matrix *B,
                           const bsm_mult_opts *opts, void *stream, bsm_plan *plan);

/* bsm_plan_block_size -- the leaf block size the plan computes at. */
bsm_status bsm_plan_block_size(bsm_plan plan, int *bs);

/* bsm_plan_execute -- replay the plan's numeric phase, ordered after earlier
 * work on `stream` and before later work on it (asynchronous).  Errors:
 * INVALID_ARG, CUDA. */
bsm_status bsm_plan_execute(bsm_plan plan, void *stream);

/* bsm_plan_results -- new handles C[0..n-1] holding the products of the last
 * execution (exactly-zero blocks removed).  Synchronises `stream`.  Errors:
 * INVALID_ARG, OOM, CUDA, TIMEOUT (a bounded device wait gave up during the
 * execution). */
bsm_status bsm_plan_results(bsm_plan plan, bsm_matrix *C, void *stream);

/* bsm_plan_info -- the launch configuration in use: order (0 longest product
 * list first, 1 product by product in Morton order), work items per claim of
 * the split kernel, CTAs per SM of the FP64 kernel (0 = as many as fit), and
 * the number of (product, C block) work items.  Outputs may be NULL. */
bsm_status bsm_plan_info(bsm_plan plan, int *order, int *chunk, int *ctas_per_sm,
                         int64_t *nitems);

/* bsm_plan_tile -- the arithmetic tile of the plan's numeric phase (the FP64
 * thread tile is chosen by measurement with BSM_FLAG_AUTOTUNE):
 *   form           1: FP64 on scalar DFMA -- each of a C block's 128 threads
 *                  sums a tile_m x tile_n tile of outputs (tile_n consecutive
 *                  columns), one k at a time;
 *                  0: FP64 on the tensor path (BSM_FP64_MODE=dmma) -- 8 x 8
 *                  mma.sync m8n8k4 tiles, 2 x 2 warps per C block;
 *                  2: split modes -- tcgen05 MMAs of tile_m = 128 rows and
 *                  tile_n = N columns (bs: one C block per work item, 2 bs:
 *                  sibling pairs of C blocks sharing every A tile);
 *                  3: split modes at bs 16 with grouped items -- as 2 with
 *                  tile_n = bs, up to four C blocks of short product lists
 *                  per work item, each in accumulator columns of its own
 * With BSM_FLAG_AUTOTUNE the split item shape (grouped or single C blocks,
 * where both exist) is chosen by measurement as well.
 * Outputs may be NULL.  Errors: INVALID_ARG. */
bsm_status bsm_plan_tile(bsm_plan plan, int *form, int *tile_m, int *tile_n);

/* bsm_plan_destroy -- free a plan (NULL accepted). */
bsm_status bsm_plan_destroy(bsm_plan plan);

/*
 * bsm_selftest_wait_timeout -- failure-path check: runs one CTA that waits on
 * a device barrier that nothing completes, bounded by limit_ms (1..5000), the
 * same bounded-wait mechanism every kernel of this library uses.  Expected
 * result: BSM_ERR_TIMEOUT after about limit_ms, with the CUDA context intact.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
bsm_status bsm_selftest_wait_timeout(int limit_ms, void *stream);

/*
 * bsm_block_products_fp64_noalloc -- the FP64 numeric phase for a task list the
 * caller supplies, allocating nothing.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory on
 * their own path -- e.g. a process whose device memory is reserved in full by
 * another allocator (so any cudaMalloc fails), or a latency-critical loop that
 * cannot afford an allocation's implicit synchronisation.  It issues no
 * cudaMalloc, cudaMallocAsync, cudaMallocHost, cudaFree or allocating library
 * call; the caller passes every input and output.
 *
 *   bs            16, 32 or 64
 *   nc            number of C blocks, 0 <= nc <= BSM_NOALLOC_MAX_CBLOCKS
 *   seg           device int32[nc+1]: C block c is the sum of products
 *                 seg[c] .. seg[c+1]-1 (non-decreasing, seg[0] >= 0)
 *   ta, tb        device int32[seg[nc]]: A and B block index of each product
 *   a_vals, na    device float64[na][bs][bs], row-major blocks of A
 *   b_vals, nb    device float64[nb][bs][bs], row-major blocks of B
 *                 (a_vals, b_vals and c_vals 16-byte aligned)
 *   c_vals        device float64[nc][bs][bs], output: C block c = sum over its
 *                 products of A[ta] * B[tb], summed in list order
 *   nnz_out       device int64, output: number of C blocks with an entry
 *                 != 0.0, or -1 if an index was out of range or a bounded
 *                 device wait gave up (then c_vals is undefined)
 *   stream        cudaStream_t or NULL; the call is asynchronous on it
 *
 * Scratch: a static device array of BSM_NOALLOC_MAX_CBLOCKS + 64 int32 (about
 * 4 MiB) compiled into the library.  The first call on a device (any bs; a
 * call with nc = 0 is enough) sets the device up with that device current:
 * it looks up the array's device address and loads the module that holds
 * the array and these kernels, which under CUDA's lazy module loading is the
 * moment the array and the kernels' code take device memory.  Make that
 * first call on each device before the process reserves all device memory
 * and before any stream capture; from then on no call allocates, and the
 * device holds the array until the process exits.
 * All calls share the array and it keeps the last call's contents, so calls
 * whose work overlaps on the GPU race on it: serialise them (one stream, or
 * events between streams).
 * Errors: BLOCKSIZE, INVALID_ARG, UNSUPPORTED (nc above the maximum, or a
 * device ordinal >= 64), CUDA.
 */
#define BSM_NOALLOC_MAX_CBLOCKS (1 << 20)
bsm_status bsm_block_products_fp64_noalloc(int bs, int64_t nc, const int32_t *seg,
                                           const int32_t *ta, const int32_t *tb,
                                           const double *a_vals, int64_t na, const double *b_vals,
                                           int64_t nb, double *c_vals, int64_t *nnz_out,
                                           void *stream);

/* bsm_destroy -- free a handle (NULL is accepted).  Work queued on other
 * streams that still reads the handle must be complete. */
bsm_status bsm_destroy(bsm_matrix M);

/* bsm_status_string -- static description of a status code. */
const char *bsm_status_string(bsm_status s);

#ifdef __cplusplus
}
#endif

#endif /* BSM_H */
