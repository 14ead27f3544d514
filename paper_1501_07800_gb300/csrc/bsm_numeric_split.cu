// Split-precision numeric phase (placeholder until the tcgen05 kernel lands).
#include "bsm_internal.cuh"

bsm_status numeric_split(bsm_matrix, bsm_matrix, const SymbolicResult &, int, double *, int32_t *,
                         unsigned *, cudaStream_t) {
  return BSM_ERR_UNSUPPORTED;
}
