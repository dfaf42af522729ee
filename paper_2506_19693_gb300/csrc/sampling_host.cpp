// Host-side randomness (reading C4): counter-based SplitMix64 (Steele, Lea and
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
// draw(key, c) is output number c+1 of SplitMix64 started at state `key`;
// streams are keyed by (seed, tag, index) so every value is addressable.
//   secret : Fisher-Yates choice of h positions, one sign bit each
//   error  : rounded Gaussian by the Box-Muller cosine branch, tail cut at
//            |e| <= bound, up to 16 tries per sample, else 0
//   uniform: (hi * 2^64 + lo) mod q from two consecutive draws
//   mask   : public-key encryption's v in {0, +1, -1}, two bits of one draw
#include <cmath>

#include "ctx.h"

static inline u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

u64 sm_draw(u64 key, u64 ctr) { return mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL); }
u64 sm_stream(u64 seed, u64 tag, u64 idx) { return sm_draw(sm_draw(seed, tag), idx); }

void sample_secret(u64 seed, u32 n, int h, int8_t *s) {
  const u64 key = sm_stream(seed, TAG_SECRET, 0);
  std::vector<u32> slot(n);
  for (u32 i = 0; i < n; ++i) { slot[i] = i; s[i] = 0; }
  for (u32 i = 0; i < (u32)h; ++i) {
    u32 r = (u32)(sm_draw(key, i) % (u64)(n - i));
    std::swap(slot[i], slot[i + r]);
    s[slot[i]] = (sm_draw(key, (u64)h + i) & 1ULL) ? -1 : 1;
  }
}

void sample_gaussian(u64 key, u32 n, double sigma, i64 bound, i64 *e) {
  const double two_pi = 2.0 * M_PI;
  for (u32 j = 0; j < n; ++j) {
    i64 val = 0;
    for (u64 k = 0; k < 16; ++k) {
      const u64 c = 2 * ((u64)j * 16 + k);
      const double u1 = (double)((sm_draw(key, c) >> 11) + 1) * 0x1p-53;
      const double u2 = (double)(sm_draw(key, c + 1) >> 11) * 0x1p-53;
      const double g = sigma * std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
      const i64 r = (i64)std::llround(g);
      if (r >= -bound && r <= bound) { val = r; break; }
    }
    e[j] = val;
  }
}

// the low two bits of one draw per coefficient: 0, 1 -> 0; 2 -> +1; 3 -> -1
void sample_pk_mask(u64 key, u32 n, i64 *v) {
  for (u32 j = 0; j < n; ++j) {
    const u64 r = sm_draw(key, j) & 3;
    v[j] = r < 2 ? 0 : (r == 2 ? 1 : -1);
  }
}

u64 sample_uniform(u64 key, u64 idx, u64 q) {
  unsigned __int128 x = ((unsigned __int128)sm_draw(key, 2 * idx) << 64) | sm_draw(key, 2 * idx + 1);
  return (u64)(x % q);
}
