// Batched products: per-product descriptors and the global work-list encoding.
#pragma once

#include <stdint.h>

// Everything one product's numeric phase needs, in device memory (a table of
// these is indexed by the work items).
struct ProdDesc {
  const int32_t *seg, *ta, *tb;  // task list: C block c sums products seg[c]..seg[c+1]-1
  const uint64_t *ckeys;         // C block Morton keys
  const double *av, *bv;         // A / B leaf blocks
  double *cv;                    // C blocks (output)
  int32_t *nz;                   // nonzero flag per C block (output)
  int64_t na, nb, nc, nt;        // A blocks, B blocks, C blocks, products
  // split mode only
  const uint8_t *asl, *bsl;      // digit slices of A / B (BF16 or E4M3 codes)
  const int *rowexp, *colexp;    // power-of-two scale exponents
  // pair items (split kernel with two C blocks per item): items are sibling
  // pairs (I, 2y), (I, 2y+1); seg / ta / tb / ckeys describe the pairs (merged
  // product lists, tb = B pair slot, key of the even sibling), pairc[2p],
  // pairc[2p+1] are the pair's C blocks (-1: absent), nb counts B pair slots
  const int32_t *pairc;
};

// Work item = (product index << 40) | C block index.
__host__ __device__ inline uint64_t make_item(uint32_t p, uint64_t c) {
  return ((uint64_t)p << 40) | c;
}
__host__ __device__ inline uint32_t item_product(uint64_t it) { return (uint32_t)(it >> 40); }
__host__ __device__ inline int64_t item_cblock(uint64_t it) {
  return (int64_t)(it & ((1ull << 40) - 1));
}
