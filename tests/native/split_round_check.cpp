// Host build of the split kernel's exact recombination and rounding helpers
// (paper_1501_07800_gb300/csrc/bsm_split_round.cuh), driven by
// tests/test_split_round.py.  Reads lines "S B X D_0 .. D_{S-1}" (diagonal
// sums D_d of one output) and prints "V ok bits": the recombined integer,
// whether the fast rounding applies, and the double's bit pattern.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cstdio>
#include <cstring>
#include "../../paper_1501_07800_gb300/csrc/bsm_split_round.cuh"

template <int S, int B>
static int64_t combine(const long long *D) {
  uint32_t p[S];
  for (int i = 0; i < S; i++) p[i] = 0x4B400000u + (uint32_t)(int32_t)D[i];
  return narrow_combine<S, B>(p);
}

int main() {
  // the fast-path sizes the kernel uses (block products per narrow flush)
  printf("%d %d %d %d %d %d\n", narrow_int64_products<7, 7, 32>(), narrow_int64_products<7, 7, 16>(),
         narrow_int64_products<6, 7, 32>(), narrow_int64_products<3, 7, 32>(),
         narrow_int64_products<12, 4, 32>(), narrow_int64_products<6, 4, 32>());
  int S, B, X;
  while (scanf("%d %d %d", &S, &B, &X) == 3) {
    long long D[16];
    for (int i = 0; i < S; i++)
      if (scanf("%lld", &D[i]) != 1) return 1;
    int64_t v = 0;
    if (S == 7 && B == 7) v = combine<7, 7>(D);
    else if (S == 6 && B == 7) v = combine<6, 7>(D);
    else if (S == 3 && B == 7) v = combine<3, 7>(D);
    else if (S == 6 && B == 4) v = combine<6, 4>(D);
    else if (S == 12 && B == 4) v = combine<12, 4>(D);
    else return 2;
    double out = 0;
    const bool ok = int64_scaled_to_double(v, X, out);
    unsigned long long b;
    memcpy(&b, &out, 8);
    printf("%lld %d %016llx\n", (long long)v, (int)ok, b);
  }
  return 0;
}
