// Shared device/host definitions of the GB300 RNS-CKKS core.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ckks.h"

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;

#define MAX_MODS 80            // q's + p's
#define MAX_POLYS 256          // polynomials per launch (pointer arrays in kernel params)

// Per-modulus constants, read by every kernel through a device pointer.
struct ModInfo {
  u64 q;          // the prime (< 2^62)
  u64 twoq;       // 2q
  u64 r64;        // 2^64 mod q
  u64 r64_s;      // Shoup companion floor(r64 * 2^64 / q)
  u64 one_s;      // floor(2^64 / q): Shoup companion of 1
  u64 ninv;       // N^-1 mod q
  u64 ninv_s;
  u64 qinv_neg;   // -q^-1 mod 2^64 (Montgomery reduction)
};

#if defined(__CUDACC__)
// ---------------------------------------------------------------------------
// Modular arithmetic (q < 2^62).
// Shoup: for constant w < q with w_s = floor(w 2^64 / q), any x < 2^64:
//   w x - floor(w_s x / 2^64) q  lies in [0, 2q).
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 w_s, u64 q) {
  return w * x - __umul64hi(w_s, x) * q;
}
__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }
__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 w_s, u64 q) {
  return csub(shoup_lazy(x, w, w_s, q), q);
}
// Reduce the 128-bit value hi * 2^64 + lo mod q:
// hi * (2^64 mod q) via Shoup and lo * 1 via Shoup, each in [0, 2q); sum < 4q.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const ModInfo &m) {
  u64 a = shoup_lazy(hi, m.r64, m.r64_s, m.q);
  u64 b = lo - __umul64hi(m.one_s, lo) * m.q;
  u64 r = a + b;
  r = csub(r, m.twoq);
  return csub(r, m.q);
}
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const ModInfo &m) {
  return reduce128(__umul64hi(a, b), a * b, m);
}
// Montgomery reduction: (hi 2^64 + lo) 2^-64 mod q, for hi 2^64 + lo < 2^65 q.
// With m = lo (-q^-1) mod 2^64, lo + m q vanishes mod 2^64 (a carry out exactly
// when lo != 0), so (T + m q) / 2^64 = hi + floor(m q / 2^64) + [lo != 0] < 3q.
__device__ __forceinline__ u64 redc128(u64 hi, u64 lo, const ModInfo &m) {
  const u64 mm = lo * m.qinv_neg;
  u64 r = hi + __umul64hi(mm, m.q) + (lo != 0 ? 1 : 0);
  r = csub(r, m.twoq);
  return csub(r, m.q);
}
// 128-bit multiply-accumulate (hi:lo += a * b) as one carry chain
__device__ __forceinline__ void mac128(u64 &hi, u64 &lo, u64 a, u64 b) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
      "madc.hi.u64 %1, %2, %3, %1;"
      : "+l"(lo), "+l"(hi)
      : "l"(a), "l"(b));
}
__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) { return csub(a + b, q); }
// High word of a 64 x 64-bit product less e, e in {0, 1, 2}: the low x low
// partial product and the carries out of the cross products' low halves are
// dropped (each of the three dropped terms is below 2^32 after the shift, so
// together they carry at most 2 into the high word).  Three 32-bit multiplies
// instead of the exact high word's four and its carry chain.
__device__ __forceinline__ u64 umulhi_approx(u64 a, u64 b) {
  const u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
  return (u64)ah * bh + __umulhi(ah, bl) + __umulhi(al, bh);
}
// Shoup product with that quotient: w x - (floor(w_s x / 2^64) - e) q lies in
// [0, 4q) (the exact quotient gives [0, 2q)); q < 2^62.
__device__ __forceinline__ u64 shoup_approx(u64 x, u64 w, u64 w_s, u64 q) {
  return w * x - umulhi_approx(w_s, x) * q;
}
// The NTT's butterflies, one per call (the production sequences, also timed
// alone by the integer-pipe microbenchmark):
// forward, loose (65 q < 2^64): no correction, approximate quotient
__device__ __forceinline__ void bfly_fwd_loose(u64 &a, u64 &b, u64 w, u64 w_s, u64 q, u64 twoq) {
  const u64 t = shoup_approx(b, w, w_s, q);
  const u64 x = a;
  a = x + t;
  b = x + 2 * twoq - t;
}
// forward, strict (Harvey): inputs < 4q, x brought below 2q, outputs < 4q
__device__ __forceinline__ void bfly_fwd_strict(u64 &a, u64 &b, u64 w, u64 w_s, u64 q, u64 twoq) {
  u64 x = a;
  if (x >= twoq) x -= twoq;
  const u64 t = shoup_lazy(b, w, w_s, q);
  a = x + t;
  b = x + twoq - t;
}
// inverse (Gentleman-Sande): values in [0, r), r = 2q (exact quotient) or
// 4q (APPROX, q < 2^61)
template <bool APPROX>
__device__ __forceinline__ void bfly_inv(u64 &a, u64 &b, u64 w, u64 w_s, u64 q, u64 r) {
  const u64 x = a, y = b;
  u64 sum = x + y;
  if (sum >= r) sum -= r;
  a = sum;
  b = APPROX ? shoup_approx(x + r - y, w, w_s, q) : shoup_lazy(x + r - y, w, w_s, q);
}
// Counter-based uniform sampling (reading C4): draw(key, c) is output c + 1 of
// SplitMix64 (Steele, Lea and Flood 2014) started at state `key`, and a
// uniform residue is (draw(2 idx) 2^64 + draw(2 idx + 1)) mod q.
__device__ __forceinline__ u64 mix64_dev(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ u64 draw_dev(u64 key, u64 ctr) {
  return mix64_dev(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}
__device__ __forceinline__ u64 uniform_dev(u64 key, u64 idx, const ModInfo &m) {
  return reduce128(draw_dev(key, 2 * idx), draw_dev(key, 2 * idx + 1), m);
}
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
// Index read by the automorphism sigma_g (X -> X^g, g odd) at output position
// j of the canonical NTT order A[j] = a(psi^(2 brv(j) + 1)) (reading C11): the
// output at exponent 2 brv(j) + 1 takes the input at g (2 brv(j) + 1) mod 2N.
__device__ __forceinline__ u32 gal_src(u32 j, u32 g, u32 n, int log_n) {
  if (g == 1) return j;
  const u32 e = (u32)(((u64)g * (2 * (__brev(j) >> (32 - log_n)) + 1)) & (2 * n - 1));
  return __brev((e - 1) >> 1) >> (32 - log_n);
}
#endif  // __CUDACC__

// Host-side error helper
#define CK_CUDA(call)                                 \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) return CKKS_E_CUDA;        \
  } while (0)

struct PolyPtrs {
  u64 *p[MAX_POLYS];
};
struct CPolyPtrs {
  const u64 *p[MAX_POLYS];
};
