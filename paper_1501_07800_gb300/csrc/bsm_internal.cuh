// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bsm.h"
#include "bsm_batch.cuh"

// Runs `set` (a kernel attribute setting, which is per device) the first
// time it is needed on the current device; thread-safe (setting an attribute
// twice is harmless).  `done` holds one bit per device ordinal below 64.
template <typename F>
bsm_status once_per_device(std::atomic<uint64_t> &done, F set) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set();
  const uint64_t bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return BSM_OK;
  const bsm_status st = set();
  if (st == BSM_OK) done.fetch_or(bit, std::memory_order_release);
  return st;
}

// NVTX range for the duration of a scope (visible to profilers; a no-op
// without one attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

#define BSM_MAXH 31  // tree heights 0..31: up to 2^31 blocks per side

// ------------------------------------------------------------- device errors
// Device code never traps: it records the first problem in an error word that
// the host reads after the kernel.
enum : unsigned {
  DERR_NONE = 0,
  DERR_OUT_OF_RANGE = 1,
  DERR_DUPLICATE = 2,
  DERR_TIMEOUT = 3,
  DERR_BOUNDS = 4,
};

// Spin limit of every mbarrier wait (each try_wait may itself suspend for a
// while); ~seconds at GB300 clocks, far beyond any legitimate wait.
#define BSM_SPIN_LIMIT (1u << 26)

struct bsm_matrix_s {
  int64_t nrows = 0, ncols = 0, mb = 0, nb = 0;
  int bs = 0;
  int L = 0;         // the tree spans 2^L blocks per side
  int device = 0;
  int64_t nblk = 0;  // stored (nonzero) blocks
  uint64_t *keys = nullptr;  // [nblk] Morton keys, ascending
  double *vals = nullptr;    // [nblk][bs][bs]
  // levels h = 1..L (height above the leaves); level L is the root
  int64_t nlev[BSM_MAXH + 1] = {};
  uint64_t *lkeys[BSM_MAXH + 1] = {};
  uint8_t *lmask[BSM_MAXH + 1] = {};
  int32_t *lcstart[BSM_MAXH + 1] = {};
  // every device allocation owned by the handle
  std::vector<void *> owned;
};

// v != 0.0 (so -0.0 is zero and NaN is not), from the bits: on GB300 a double
// compare would take the FP64 pipe, the scarcest unit of the chip.
__host__ __device__ inline bool nonzero_f64(double v) {
#ifdef __CUDA_ARCH__
  return ((uint64_t)__double_as_longlong(v) << 1) != 0;
#else
  return v != 0.0;
#endif
}

// Morton key: bit 2b+1 = bit b of the block row, bit 2b = bit b of the block
// column, so the two low bits of a key are the child index 2*rowbit + colbit.
__host__ __device__ inline uint64_t morton_spread(uint64_t x) {
  x &= 0xFFFFFFFFull;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
__host__ __device__ inline uint64_t morton_key(uint64_t I, uint64_t J) {
  return (morton_spread(I) << 1) | morton_spread(J);
}
__host__ __device__ inline uint32_t morton_compact(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

inline int ceil_log2_i64(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) l++;
  return l;
}

// ----------------------------------------------------------- host utilities
// Stream-ordered allocation from the device's default memory pool, or from
// the library's own pool for allocations of 1 GiB and more.
bsm_status dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
bsm_status cuda_status(cudaError_t e);

// Reusable pinned host scratch for small readbacks (per thread).
struct HostScratch {
  void *p = nullptr;
  size_t n = 0;
  void *get(size_t bytes);
  ~HostScratch();
};
HostScratch &host_scratch();
// Reads `bytes` (a multiple of 4, small: counts, flags, error words) from
// device memory into page-locked host memory, stream-ordered on s, with a
// one-block kernel writing the host memory's device-mapped address: a
// copy-engine transfer would queue behind any large device-to-host copy in
// flight on another stream (a download overlapping this work).  Other host
// memory falls back to cudaMemcpyAsync.  The host reads after synchronising s.
bsm_status readback(void *host, const void *dev, size_t bytes, cudaStream_t s);

// Exclusive prefix sums on the device (CUB), sized on first use.
bsm_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
bsm_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
bsm_status scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s);
// Inclusive prefix sums of uint64 values, saturating at 2^64 - 1.
bsm_status scan_inclusive_u64_sat(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s);
bsm_status sort_keys_u64(const uint64_t *kin, uint64_t *kout, const int32_t *vin, int32_t *vout,
                         int64_t n, int end_bit, cudaStream_t s);
bsm_status sort_pairs_u32_u64(const uint32_t *kin, uint32_t *kout, const uint64_t *vin,
                              uint64_t *vout, int64_t n, cudaStream_t s);

// Builds the level arrays of a handle whose keys are set (bsm_tree.cu).
bsm_status build_levels(bsm_matrix M, cudaStream_t s);
// Copies blocks: dst[t] = src[idx[t]] (bs*bs doubles each), on at most
// max_ctas CTAs (<= 0: a full-device grid).
void launch_gather_blocks(const double *src, const int32_t *idx, double *dst, int64_t n, int bs,
                          cudaStream_t s, int64_t max_ctas = 0);

// ---------------------------------------------------------- symbolic result
// Leaf-level task list of one product: C blocks in Morton order, each with the
// ordered (A block, B block) pairs that contribute to it (k ascending).
struct SymbolicResult {
  int64_t nc = 0;           // C blocks (before zero removal)
  int64_t nt = 0;           // triples
  uint64_t *ckeys = nullptr;  // [nc]
  int32_t *seg = nullptr;     // [nc+1] start of each C block's pairs
  int32_t *ta = nullptr;      // [nt] A leaf index
  int32_t *tb = nullptr;      // [nt] B leaf index
  int H = 0;                  // product tree height
  int64_t tasks[BSM_MAXH + 1] = {};  // pairs per height (index = height)
};
bsm_status symbolic_multiply(bsm_matrix A, bsm_matrix B, SymbolicResult *out, cudaStream_t s);

// Chunked symbolic phase: the leaf task list arrives as consecutive Morton
// ranges of C, each handed to `sink` (which may take ownership of the arrays
// by clearing the pointers).  budget: pairs per level part (0 = default, or
// the BSM_SYM_BUDGET environment variable).  tasks[h]: pairs per height.
// upper: 0, or k >= 1 to keep only C nodes on or above the diagonal at
// heights >= k - 1 (k = 1: C blocks with I <= J, for symmetric results; k = 2:
// blocks whose parent node is on or above the diagonal).
using LeafSink = std::function<bsm_status(SymbolicResult &)>;
// [key_lo, key_hi): only C blocks whose Morton keys lie in it (key_hi == 0: all).
bsm_status symbolic_chunks(bsm_matrix A, bsm_matrix B, const LeafSink &sink, int64_t *tasks,
                           int *H, int *nchunks, cudaStream_t s, int64_t budget, int upper = 0,
                           uint64_t key_lo = 0, uint64_t key_hi = 0);
void free_symbolic(SymbolicResult *r, cudaStream_t s);

// ----------------------------------------------------------- numeric phase
// Computes every C block of `sym` into cvals and sets nzflag[c] = 1 if the
// block has an entry != 0.0.  errword receives DERR_* codes.
bsm_status numeric_fp64(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, double *cvals,
                        int32_t *nzflag, unsigned *errword, cudaStream_t s);

// Split-precision numeric phase (BF16 or E4M3 digit slices on tcgen05, exact
// FP32 accumulation, integer recombination).  The split functions take a
// "spec": the slice count in the low byte and the digit format (0 BF16,
// 1 E4M3) above it, as check_opts makes it from the options.
inline int split_spec(int fmt, int slices) { return slices | (fmt << 8); }
inline int split_spec_fmt(int spec) { return spec >> 8; }
inline int split_spec_slices(int spec) { return spec & 0xFF; }
// Block width the split kernels run a single product at (operands of another
// width are re-cut exactly): E4M3 32; BF16 the operands' own, 64 as 32.
inline int split_width(int prec, int bs) {
  return prec == BSM_SPLIT_FP8 ? 32 : (bs == 64 ? 32 : bs);
}
bsm_status numeric_split(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, int slices,
                         double *cvals, int32_t *nzflag, unsigned *errword, cudaStream_t s);

// Batched numeric phases over a global (product, C block) work list.
ProdDesc make_desc(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, double *cvals,
                   int32_t *nz);
bsm_status numeric_fp64_batched(int bs, const ProdDesc *prods, const uint64_t *items,
                                int64_t nitems, unsigned long long *counter, unsigned *errword,
                                int ctas_per_sm, cudaStream_t s, int form = -1);
bsm_status split_supported(int bs, int slices);
int split_flush_group(int bs, int spec, int bound_log2);
bsm_status split_prepare(bsm_matrix A, bsm_matrix B, int slices, unsigned *errword, ProdDesc &d,
                         std::vector<void *> &owned, cudaStream_t s);
// fold: device scratch of split_fold_bytes(bs) bytes, private to the launch
// (C blocks with very long product lists park exact partial sums there).
// np = 2: items are pairs of sibling C blocks (ProdDesc.pairc, B slices in
// pair slots); np = 1: single C blocks, grouped where split_use_groups;
// np = -1: single C blocks, never grouped; np = 4: grouped where compiled.
bsm_status split_launch(int bs, int slices, const ProdDesc *prods_dev, const uint64_t *items,
                        int64_t nitems, unsigned long long *work, unsigned *errword,
                        int64_t *fold, cudaStream_t s, int chunk = 32, int np = 1);
size_t split_fold_bytes(int bs);
// Pair items (two sibling C blocks per item) for nt products over nc C blocks?
bool split_use_pairs(int bs, int spec, int64_t nt, int64_t nc);
// Grouped items (several short-list C blocks per item) for this format?
bool split_use_groups(int bs, int spec);
// Is there a grouped-item kernel for this leaf size and format?
bool split_groups_compiled(int bs, int spec);
// Pair-item structures of one product (task-list fields of d, A slices, B
// slices in pair slots, padded exponents); *bslot: B pair slot per B block.
bsm_status split_pairs_prepare(bsm_matrix A, bsm_matrix B, const SymbolicResult &sym, int spec,
                               ProdDesc &d, int32_t **bslot, std::vector<void *> &owned,
                               cudaStream_t s);
// Work items per claim for a list of nt block products over nc C blocks.
int split_chunk_for(int64_t nt, int64_t nc);
// Longest product list of a task list, atomically maxed into *dmax_dev.
void launch_max_seg(const SymbolicResult &sym, int *dmax_dev, cudaStream_t s);
bsm_status split_alloc(bsm_matrix A, bsm_matrix B, int slices, ProdDesc &d,
                       std::vector<void *> &owned, cudaStream_t s);
// bslot (pair items only): B pair slot of every B block, NULL otherwise.
bsm_status split_compute(bsm_matrix A, bsm_matrix B, int slices, const ProdDesc &d,
                         unsigned *errword, cudaStream_t s, const int32_t *bslot = nullptr);

// C assembly from a numeric result: zero removal and level build.
// finish_product takes ownership of sym->ckeys and cvals; finish_product_copy
// leaves both untouched and copies what it keeps.
bsm_status finish_product(bsm_matrix C, SymbolicResult *sym, double *cvals, int32_t *nz,
                          unsigned *err, cudaStream_t s);
bsm_status finish_product_copy(bsm_matrix C, const SymbolicResult &sym, const double *cvals,
                               const int32_t *nz, unsigned *err, cudaStream_t s);
bsm_status check_pair(bsm_matrix A, bsm_matrix B);
// One product through the chunked symbolic phase and the chosen numeric
// phase (bsm_multiply.cu); upper: only C blocks with I <= J.  Split modes
// at block size 64 run at 32 on re-cut operands (the split result does not
// depend on the leaf size) and merge C back.
bsm_status multiply_one(bsm_matrix A, bsm_matrix B, int prec, int slices, cudaStream_t s,
                        bsm_matrix *out, bool upper = false, uint64_t key_lo = 0,
                        uint64_t key_hi = 0);
// dst[t] = src[idx[t] & 0x7FFFFFFF], transposed when bit 31 of idx[t] is set
// (bsm_ops.cu).
void launch_gather_blocks_t(const double *src, const int32_t *idx, double *dst, int64_t n, int bs,
                            cudaStream_t s);
// Re-blocking (bsm_ops.cu).  keep_all, when splitting: 0 drops all-zero
// sub-blocks, 1 keeps every sub-block inside the matrix (the new structure
// then depends on A's structure only), 2 drops all-zero sub-blocks and those
// below the diagonal; map_out receives the index map reblock_refresh uses to
// copy new values of A into the re-blocked handle (caller frees it).
bsm_status reblock_impl(bsm_matrix A, int bs, int keep_all, bsm_matrix *out, int32_t **map_out,
                        cudaStream_t s);
void reblock_refresh(bsm_matrix src, bsm_matrix dst, const int32_t *map, cudaStream_t s);
bsm_status check_opts(const bsm_mult_opts *o, int *prec, int *slices, int allowed_flags);

// Handle shells for results (bsm_tree.cu).
bsm_matrix new_matrix_shell(int64_t nrows, int64_t ncols, int bs, int L);
void free_matrix_shell(bsm_matrix M, cudaStream_t s);

// Thread-local statistics of the last product.
struct LastStats {
  int nlev = 0;
  int64_t tasks[BSM_MAXH + 1] = {};
  int64_t triples = 0, nc_sym = 0;
  double phase_ms[3] = {0, 0, 0};
  int64_t launches = 0;
  int chunks = 0;  // symbolic chunks (Morton ranges of C) of the last product
};
LastStats &last_stats();

// Kernel-launch counter of the calling thread (every launch site adds to it).
int64_t &launch_counter();
inline void count_launch(int n = 1) { launch_counter() += n; }
bool timing_enabled();
// Arithmetic form of the FP64 numeric phase: 0 DMMA, 1 DFMA (bsm_numeric_fp64.cu).
int fp64_mode();
// Deferred per-phase timing of the last product on the calling thread (when
// timing is enabled): a product records CUDA events on its stream and never
// waits for them; bsm_last_phase_ms resolves them when it is called.
void timing_begin();                          // drops the previous product's events
int timing_mark(cudaStream_t s);              // records an event: its index, -1 if off
void timing_span(int phase, int e0, int e1);  // phase += elapsed(e0, e1)
void timing_rest(int phase, int e0, int e1);  // phase = elapsed(e0, e1) - the other phases

#define BSM_TRY(x)                       \
  do {                                   \
    bsm_status _st = (x);                \
    if (_st != BSM_OK) return _st;       \
  } while (0)
#define BSM_CUDA(x)                                   \
  do {                                                \
    cudaError_t _e = (x);                             \
    if (_e != cudaSuccess) return cuda_status(_e);    \
  } while (0)
