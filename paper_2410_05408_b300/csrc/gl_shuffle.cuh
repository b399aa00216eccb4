// gl_shuffle.cuh -- counter-based random numbers and the per-epoch permutation
// of the surrogate's training samples (host and device, so that the host tests
// can check the permutation).
//
// SplitMix64 (Steele, Lea and Flood 2014, "Fast splittable pseudorandom number
// generators") maps a 64-bit counter to a 64-bit output; every draw is the
// generator at (seed, counter).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GL_SH_HD __host__ __device__ __forceinline__
#else
#define GL_SH_HD inline
#endif

namespace gl {

GL_SH_HD uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// The permutation of an epoch: a four-round Feistel network on 2h-bit indices
// (round keys from the generator at (seed, epoch, round)), walked until it lands
// below n; from j < n the walk stays on j's cycle, so it ends, and the map is a
// bijection of [0, n).  (The walk is capped far beyond any length it can
// reach with probability above 1e-30; at the cap j maps to itself.)
struct Shuffle {
  uint64_t key[4];
  int h;          // bits per half
  uint64_t mask;  // (1 << h) - 1
};

inline Shuffle make_shuffle(uint64_t seed, int64_t epoch, int64_t n) {
  Shuffle s;
  int bits = 2;
  while (bits < 62 && ((int64_t)1 << bits) < n) bits += 2;
  s.h = bits / 2;
  s.mask = ((uint64_t)1 << s.h) - 1;
  for (int r = 0; r < 4; ++r) s.key[r] = splitmix64(seed ^ splitmix64((uint64_t)epoch * 4 + r + 1));
  return s;
}

GL_SH_HD int64_t shuffle_index(const Shuffle& s, int64_t j, int64_t n) {
  uint64_t x = (uint64_t)j;
  for (int it = 0; it < 256; ++it) {
    uint64_t l = x >> s.h, r = x & s.mask;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint64_t f = splitmix64(r ^ s.key[k]) & s.mask;
      const uint64_t nl = r;
      r = l ^ f;
      l = nl;
    }
    x = (l << s.h) | r;
    if (x < (uint64_t)n) return (int64_t)x;
  }
  return j;
}


}  // namespace gl
