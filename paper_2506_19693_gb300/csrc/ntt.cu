// Negacyclic NTT / inverse NTT over uint64 RNS limbs (reading C2).
//
// Forward transform: merged-psi Cooley-Tukey, stages m = 1, 2, ..., N/2; at
// stage m the butterfly of group i pairs (j, j + N/2m) with twiddle
// psi^brv(m + i).  The output is in the canonical order
// A[j] = a(psi^(2 brv(j) + 1)).  The inverse runs the Gentleman-Sande mirror
// (stages m = N/2 .. 1, twiddles psi^-brv(m + i)) and multiplies by N^-1.
//
// GB300 layout: a limb (N = 2^16 words, 512 KiB) does not fit in one CTA's
// shared memory, so the transform is split in two passes over HBM.  View the
// limb as H x B (B = 256 contiguous words per row, H = N / B rows):
//   pass A -- the first log2 H stages pair words of the same column; a CTA
//             takes 16 adjacent columns (each row segment is one 128-byte
//             line), loads them straight into registers, runs radix-2^s
//             sub-transforms in registers, exchanges once through shared
//             memory and writes back coalesced;
//   pass B -- the last 8 stages stay inside one row; a CTA takes 16 rows.
// Each thread owns 2^s words and runs s butterfly stages in registers
// (Harvey's lazy butterflies: values stay in [0, 4q) forward, [0, 2q)
// inverse; q < 2^62).
#include "ctx.h"

namespace {

constexpr int LB = 8;            // log2 of the row length handled by pass B
constexpr int BROW = 1 << LB;    // 256
// columns per pass-A tile: 16 (128-byte row segments); 8 at 2^9 rows, so that
// the 2^LH x CA tile stays within the 48 KB of static shared memory
__host__ __device__ constexpr int ca_of(int lh) { return lh >= 9 ? 8 : 16; }
constexpr int THREADS = 256;     // pass A; pass B runs 16 threads per row of its tile
// pass B tiles: RBT rows per CTA (16 or 8, chosen per context by ckks_tune_ntt)
template <int RBT>
__host__ __device__ constexpr int threads_b() { return RBT * 16; }

struct NttParams {
  const ModInfo *mods;
  const ulonglong2 *tw;          // [modulus][N]
  const ulonglong2 *tw_row;      // [modulus][15 N / 16]: the row pass's second phase, regrouped
  u32 n;
  int n_limbs;
  unsigned char mod_of_limb[MAX_MODS];
  CPolyPtrs src;
  PolyPtrs dst;
};

// Pass-B shared-memory padding: one spare word per 16 keeps the 16-word
// strided accesses of the row stages conflict-free.
__device__ __forceinline__ int padb(int off) { return off + (off >> 4); }

// Cooley-Tukey stages of a 2^K-point block.  Strict (Harvey): inputs < 4q,
// x brought below 2q before each butterfly, outputs < 4q.  LOOSE, for
// 65 q < 2^64 only: no correction and the approximate Shoup product (t < 4q),
// every stage raises the bound by 4q, so inputs < q stay below
// (1 + 4 log2 N) q <= 65 q < 2^64 through all 16 stages.
// tw_of(s, i): the twiddle of local stage s, group i within the block.
template <int K, bool LOOSE, class TW>
__device__ __forceinline__ void fwd_step_t(u64 (&v)[1 << K], TW tw_of, u64 q, u64 twoq) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int half = 1 << (K - 1 - s);
#pragma unroll
    for (int e = 0; e < (1 << K); ++e) {
      if (e & half) continue;
      const ulonglong2 w = tw_of(s, e >> (K - s));
      if (LOOSE)
        bfly_fwd_loose(v[e], v[e + half], w.x, w.y, q, twoq);
      else
        bfly_fwd_strict(v[e], v[e + half], w.x, w.y, q, twoq);
    }
  }
}

// block mg of the merged-psi order: twiddle psi^brv((mg << s) + i)
template <int K, bool LOOSE>
__device__ __forceinline__ void fwd_step(u64 (&v)[1 << K], u32 mg, const ulonglong2 *__restrict__ tw,
                                         u64 q, u64 twoq) {
  fwd_step_t<K, LOOSE>(v, [&](int s, int i) { return __ldg(&tw[(mg << s) + i]); }, q, twoq);
}
// the row pass's second phase: block N/16 + m, twiddles from the regrouped
// table, where the 16 threads of a row read 16 consecutive entries
template <int K, bool LOOSE>
__device__ __forceinline__ void fwd_step_row(u64 (&v)[1 << K], u32 m, const ulonglong2 *__restrict__ twr,
                                             u32 n16, u64 q, u64 twoq) {
  static_assert(K <= 4, "the regrouped table holds four stages");
  fwd_step_t<K, LOOSE>(v, [&](int s, int i) { return __ldg(&twr[(size_t)((1 << s) - 1 + i) * n16 + m]); }, q,
                       twoq);
}

// Gentleman-Sande stages s = K-1 .. STOP of a 2^K-point block.  Values stay
// in [0, R) with R = 2q (exact Shoup products); APPROX, for q < 2^61 only,
// takes the approximate product and R = 4q (x + R - y < 8q < 2^64).
template <int K, bool APPROX, int STOP, class TW>
__device__ __forceinline__ void inv_step_t(u64 (&v)[1 << K], TW tw_of, u64 q, u64 twoq) {
  const u64 r = APPROX ? 2 * twoq : twoq;
#pragma unroll
  for (int s = K - 1; s >= STOP; --s) {
    const int half = 1 << (K - 1 - s);
#pragma unroll
    for (int e = 0; e < (1 << K); ++e) {
      if (e & half) continue;
      const ulonglong2 w = tw_of(s, e >> (K - s));
      bfly_inv<APPROX>(v[e], v[e + half], w.x, w.y, q, r);
    }
  }
}

template <int K, bool APPROX, int STOP = 0>
__device__ __forceinline__ void inv_step(u64 (&v)[1 << K], u32 mg, const ulonglong2 *__restrict__ tw,
                                         u64 q, u64 twoq) {
  inv_step_t<K, APPROX, STOP>(v, [&](int s, int i) { return __ldg(&tw[(mg << s) + i]); }, q, twoq);
}
template <int K, bool APPROX>
__device__ __forceinline__ void inv_step_row(u64 (&v)[1 << K], u32 m, const ulonglong2 *__restrict__ twr,
                                             u32 n16, u64 q, u64 twoq) {
  static_assert(K <= 4, "the regrouped table holds four stages");
  inv_step_t<K, APPROX, 0>(v, [&](int s, int i) { return __ldg(&twr[(size_t)((1 << s) - 1 + i) * n16 + m]); },
                           q, twoq);
}

// Primes below this bound take the forward transform without lazy corrections
// (65 q < 2^64), and primes below 2^61 the inverse with approximate products.
constexpr u64 LOOSE_BOUND = ~0ULL / 65;
constexpr u64 APPROX_INV_BOUND = 1ULL << 61;

// ---------------------------------------------------------------- forward
// One CTA's work of each pass, specialised on LOOSE; the kernels pick the body
// from the limb's modulus (uniform per CTA).
template <int LH, int S1, bool LOOSE>
__device__ __forceinline__ void fwd_a_body(const NttParams &prm, u64 *sm, int mi, const u64 *src, u64 *dst) {
  constexpr int H = 1 << LH, S2 = LH - S1, CA = ca_of(LH);
  const u64 q = prm.mods[mi].q, twoq = 2 * q;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int c0 = blockIdx.x * CA;
  for (int x = threadIdx.x; x < (H >> S1) * CA; x += THREADS) {
    const int c = x % CA, r0 = x / CA;
    u64 v[1 << S1];
#pragma unroll
    for (int e = 0; e < (1 << S1); ++e) v[e] = src[(size_t)(r0 + (e << S2)) * BROW + c0 + c];
    fwd_step<S1, LOOSE>(v, 1u, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S1); ++e) sm[(r0 + (e << S2)) * CA + c] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (1 << S1) * CA; x += THREADS) {
    const int c = x % CA, g = x / CA;
    u64 v[1 << S2];
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) v[e] = sm[((g << S2) + e) * CA + c];
    fwd_step<S2, LOOSE>(v, (1u << S1) + g, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) dst[(size_t)((g << S2) + e) * BROW + c0 + c] = v[e];
  }
}

// Pass A at 2^9 rows: three register phases of three stages each (8 values
// per thread), the first from global memory, the last to it, shared memory
// between.  Phase p starts at stage 3p, where the column splits into 2^(3p)
// blocks of 2^(9-3p) rows; block blk takes twiddle group 2^(3p) + blk.
template <bool LOOSE>
__device__ __forceinline__ void fwd_a3_body(const NttParams &prm, u64 *sm, int mi, const u64 *src, u64 *dst) {
  constexpr int H = 1 << 9, CA = ca_of(9);
  const u64 q = prm.mods[mi].q, twoq = 2 * q;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int c0 = blockIdx.x * CA;
  for (int x = threadIdx.x; x < (H >> 3) * CA; x += THREADS) {  // stages 0..2: rows r0 + 64 e
    const int c = x % CA, r0 = x / CA;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = src[(size_t)(r0 + (e << 6)) * BROW + c0 + c];
    fwd_step<3, LOOSE>(v, 1u, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[(r0 + (e << 6)) * CA + c] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (H >> 3) * CA; x += THREADS) {  // stages 3..5: rows 64 blk + r0 + 8 e
    const int c = x % CA, y = x / CA, blk = y >> 3, r0 = y & 7;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[((blk << 6) + r0 + (e << 3)) * CA + c];
    fwd_step<3, LOOSE>(v, 8u + blk, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[((blk << 6) + r0 + (e << 3)) * CA + c] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (H >> 3) * CA; x += THREADS) {  // stages 6..8: rows 8 blk + e
    const int c = x % CA, blk = x / CA;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[((blk << 3) + e) * CA + c];
    fwd_step<3, LOOSE>(v, 64u + blk, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < 8; ++e) dst[(size_t)((blk << 3) + e) * BROW + c0 + c] = v[e];
  }
}

template <int LH, int S1>
__global__ void __launch_bounds__(THREADS, 3) fwd_pass_a(const NttParams prm) {
  __shared__ u64 sm[(1 << LH) * ca_of(LH)];
  const int limb = blockIdx.y, poly = blockIdx.z;
  const int mi = prm.mod_of_limb[limb];
  const u64 *src = prm.src.p[poly] + (size_t)limb * prm.n;
  u64 *dst = prm.dst.p[poly] + (size_t)limb * prm.n;
  if constexpr (LH == 9) {
    if (prm.mods[mi].q < LOOSE_BOUND)
      fwd_a3_body<true>(prm, sm, mi, src, dst);
    else
      fwd_a3_body<false>(prm, sm, mi, src, dst);
  } else {
    if (prm.mods[mi].q < LOOSE_BOUND)
      fwd_a_body<LH, S1, true>(prm, sm, mi, src, dst);
    else
      fwd_a_body<LH, S1, false>(prm, sm, mi, src, dst);
  }
}

template <int LH, bool LOOSE, int RB>
__device__ __forceinline__ void fwd_b_body(const NttParams &prm, u64 *sm, int mi, const u64 *src, u64 *dst) {
  constexpr int H = 1 << LH, U1 = 4, U2 = LB - U1, THREADS = threads_b<RB>();
  const u64 q = prm.mods[mi].q, twoq = 2 * q;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int row0 = blockIdx.x * RB;
  for (int x = threadIdx.x; x < RB * (BROW >> U1); x += THREADS) {
    const int l0 = x % (BROW >> U1), rr = x / (BROW >> U1), b = row0 + rr;
    u64 v[1 << U1];
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) v[e] = src[(size_t)b * BROW + l0 + (e << U2)];
    fwd_step<U1, LOOSE>(v, (u32)(H + b), tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) sm[padb(rr * BROW + l0 + (e << U2))] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (RB << U1); x += THREADS) {
    const int g = x % (1 << U1), rr = x / (1 << U1), b = row0 + rr;
    u64 v[1 << U2];
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) v[e] = sm[padb(rr * BROW + (g << U2) + e)];
    fwd_step_row<U2, LOOSE>(v, ((u32)b << U1) + g, prm.tw_row + (size_t)mi * 15 * (prm.n / 16), prm.n / 16, q,
                            twoq);
    const u64 one_s = LOOSE ? prm.mods[mi].one_s : 0;
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) {
      u64 r = v[e];
      if (LOOSE) {  // r < 65 q: Barrett with floor(2^64 / q) to [0, 2q), then [0, q)
        r -= __umul64hi(r, one_s) * q;
      } else if (r >= twoq) {
        r -= twoq;
      }
      if (r >= q) r -= q;
      sm[padb(rr * BROW + (g << U2) + e)] = r;
    }
  }
  __syncthreads();
  ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(dst + (size_t)row0 * BROW);
#pragma unroll 4
  for (int x = threadIdx.x; x < RB * BROW / 2; x += THREADS) {
    const int o = padb(2 * x);
    d2[x] = make_ulonglong2(sm[o], sm[o + 1]);
  }
}

template <int LH, int RB>
__global__ void __launch_bounds__(threads_b<RB>(), RB == 16 ? 3 : 6) fwd_pass_b(const NttParams prm, int from_src) {
  __shared__ u64 sm[RB * BROW + (RB * BROW >> 4)];
  const int limb = blockIdx.y, poly = blockIdx.z;
  const int mi = prm.mod_of_limb[limb];
  const u64 *src = (from_src ? prm.src.p[poly] : prm.dst.p[poly]) + (size_t)limb * prm.n;
  u64 *dst = prm.dst.p[poly] + (size_t)limb * prm.n;
  if (prm.mods[mi].q < LOOSE_BOUND)
    fwd_b_body<LH, true, RB>(prm, sm, mi, src, dst);
  else
    fwd_b_body<LH, false, RB>(prm, sm, mi, src, dst);
}

// ---------------------------------------------------------------- inverse
// Specialised on APPROX (every modulus of the launch below 2^61: values in
// [0, 4q) between stages and passes), chosen by the host per launch.
template <int LH, bool APPROX, int RB>
__device__ __forceinline__ void inv_b_body(const NttParams &prm, u64 *sm, int mi, const u64 *src, u64 *dst) {
  constexpr int H = 1 << LH, U1 = 4, U2 = LB - U1, THREADS = threads_b<RB>();
  const u64 q = prm.mods[mi].q, twoq = 2 * q;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int row0 = blockIdx.x * RB;
  {  // the rows (contiguous) in 16-byte loads, all issued before the first store
    constexpr int PER = RB * BROW / 2 / THREADS;
    const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src + (size_t)row0 * BROW);
    ulonglong2 t[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) t[k] = s2[threadIdx.x + k * THREADS];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int o = padb(2 * (threadIdx.x + k * THREADS));  // an even word and its odd neighbour
      sm[o] = t[k].x;
      sm[o + 1] = t[k].y;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (RB << U1); x += THREADS) {
    const int g = x % (1 << U1), rr = x / (1 << U1), b = row0 + rr;
    u64 v[1 << U2];
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) v[e] = sm[padb(rr * BROW + (g << U2) + e)];
    inv_step_row<U2, APPROX>(v, ((u32)b << U1) + g, prm.tw_row + (size_t)mi * 15 * (prm.n / 16), prm.n / 16, q,
                             twoq);
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) sm[padb(rr * BROW + (g << U2) + e)] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < RB * (BROW >> U1); x += THREADS) {
    const int l0 = x % (BROW >> U1), rr = x / (BROW >> U1), b = row0 + rr;
    u64 v[1 << U1];
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) v[e] = sm[padb(rr * BROW + l0 + (e << U2))];
    inv_step<U1, APPROX>(v, (u32)(H + b), tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) dst[(size_t)b * BROW + l0 + (e << U2)] = v[e];
  }
}

template <int LH, int RB, bool APPROX>
__global__ void __launch_bounds__(threads_b<RB>(), RB == 16 ? 4 : 8) inv_pass_b(const NttParams prm) {
  __shared__ u64 sm[RB * BROW + (RB * BROW >> 4)];
  const int limb = blockIdx.y, poly = blockIdx.z;
  const int mi = prm.mod_of_limb[limb];
  const u64 *src = prm.src.p[poly] + (size_t)limb * prm.n;
  u64 *dst = prm.dst.p[poly] + (size_t)limb * prm.n;
  inv_b_body<LH, APPROX, RB>(prm, sm, mi, src, dst);
}

template <int LH, int S1, bool APPROX>
__device__ __forceinline__ void inv_a_body(const NttParams &prm, u64 *sm, int mi, u64 *dst) {
  constexpr int H = 1 << LH, S2 = LH - S1, CA = ca_of(LH);
  const ModInfo m = prm.mods[mi];
  const u64 q = m.q, twoq = 2 * q, ninv = m.ninv, ninv_s = m.ninv_s;
  const u64 r = APPROX ? 2 * twoq : twoq;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int c0 = blockIdx.x * CA;
  for (int x = threadIdx.x; x < (1 << S1) * CA; x += THREADS) {
    const int c = x % CA, g = x / CA;
    u64 v[1 << S2];
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) v[e] = dst[(size_t)((g << S2) + e) * BROW + c0 + c];
    inv_step<S2, APPROX>(v, (1u << S1) + g, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) sm[((g << S2) + e) * CA + c] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (H >> S1) * CA; x += THREADS) {
    const int c = x % CA, r0 = x / CA;
    u64 v[1 << S1];
#pragma unroll
    for (int e = 0; e < (1 << S1); ++e) v[e] = sm[(r0 + (e << S2)) * CA + c];
    inv_step<S1, APPROX, 1>(v, 1u, tw, q, twoq);
    // last stage (twiddle psi^-brv(1)) with N^-1 folded in: the sum is scaled
    // by N^-1, the difference by tw[0] = psi^-brv(1) N^-1; both fully reduced
    // by exact Shoup products
    constexpr int HALF = 1 << (S1 - 1);
    const ulonglong2 w0 = __ldg(&tw[0]);
#pragma unroll
    for (int e = 0; e < HALF; ++e) {
      const u64 x = v[e], y = v[e + HALF];
      dst[(size_t)(r0 + (e << S2)) * BROW + c0 + c] = shoup(x + y, ninv, ninv_s, q);
      dst[(size_t)(r0 + ((e + HALF) << S2)) * BROW + c0 + c] = shoup(x + r - y, w0.x, w0.y, q);
    }
  }
}

// The inverse of fwd_a3_body: stages 8..6 on blocks of 8 rows, 5..3 on
// blocks of 64, then 2..1 and the last stage with N^-1 folded in.
template <bool APPROX>
__device__ __forceinline__ void inv_a3_body(const NttParams &prm, u64 *sm, int mi, u64 *dst) {
  constexpr int H = 1 << 9, CA = ca_of(9);
  const ModInfo m = prm.mods[mi];
  const u64 q = m.q, twoq = 2 * q, ninv = m.ninv, ninv_s = m.ninv_s;
  const u64 r = APPROX ? 2 * twoq : twoq;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int c0 = blockIdx.x * CA;
  for (int x = threadIdx.x; x < (H >> 3) * CA; x += THREADS) {
    const int c = x % CA, blk = x / CA;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = dst[(size_t)((blk << 3) + e) * BROW + c0 + c];
    inv_step<3, APPROX>(v, 64u + blk, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[((blk << 3) + e) * CA + c] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (H >> 3) * CA; x += THREADS) {
    const int c = x % CA, y = x / CA, blk = y >> 3, r0 = y & 7;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[((blk << 6) + r0 + (e << 3)) * CA + c];
    inv_step<3, APPROX>(v, 8u + blk, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < 8; ++e) sm[((blk << 6) + r0 + (e << 3)) * CA + c] = v[e];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < (H >> 3) * CA; x += THREADS) {
    const int c = x % CA, r0 = x / CA;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = sm[(r0 + (e << 6)) * CA + c];
    inv_step<3, APPROX, 1>(v, 1u, tw, q, twoq);
    const ulonglong2 w0 = __ldg(&tw[0]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const u64 a = v[e], b = v[e + 4];
      dst[(size_t)(r0 + (e << 6)) * BROW + c0 + c] = shoup(a + b, ninv, ninv_s, q);
      dst[(size_t)(r0 + ((e + 4) << 6)) * BROW + c0 + c] = shoup(a + r - b, w0.x, w0.y, q);
    }
  }
}

template <int LH, int S1, bool APPROX>
__global__ void __launch_bounds__(THREADS, 4) inv_pass_a(const NttParams prm) {
  __shared__ u64 sm[(1 << LH) * ca_of(LH)];
  const int limb = blockIdx.y, poly = blockIdx.z;
  const int mi = prm.mod_of_limb[limb];
  u64 *dst = prm.dst.p[poly] + (size_t)limb * prm.n;
  if constexpr (LH == 9)
    inv_a3_body<APPROX>(prm, sm, mi, dst);
  else
    inv_a_body<LH, S1, APPROX>(prm, sm, mi, dst);
}

template <int LH, int RB, bool APPROX>
void launch_inv(ckks_ctx *c, const NttParams &prm, int npoly) {
  constexpr int S1 = (LH + 1) / 2;
  const unsigned long long units = (unsigned long long)prm.n_limbs * npoly;
  dim3 ga(BROW / ca_of(LH), prm.n_limbs, npoly), gb((1 << LH) / RB, prm.n_limbs, npoly);
  PROF_LAUNCH(c, PK_NTT_INV_B, units, (inv_pass_b<LH, RB, APPROX><<<gb, threads_b<RB>(), 0, c->stream>>>(prm)));
  PROF_LAUNCH(c, PK_NTT_INV_A, units, (inv_pass_a<LH, S1, APPROX><<<ga, THREADS, 0, c->stream>>>(prm)));
}

template <int LH>
void launch_lh(ckks_ctx *c, const NttParams &prm, int npoly, bool inverse, bool approx) {
  if (inverse) {
    if (c->ntt_rows == 8)
      approx ? launch_inv<LH, 8, true>(c, prm, npoly) : launch_inv<LH, 8, false>(c, prm, npoly);
    else
      approx ? launch_inv<LH, 16, true>(c, prm, npoly) : launch_inv<LH, 16, false>(c, prm, npoly);
    return;
  }
  constexpr int S1 = (LH + 1) / 2;
  const int H = 1 << LH;
  cudaStream_t st = c->stream;
  const unsigned long long units = (unsigned long long)prm.n_limbs * npoly;
  dim3 ga(BROW / ca_of(LH), prm.n_limbs, npoly);
  PROF_LAUNCH(c, PK_NTT_FWD_A, units, (fwd_pass_a<LH, S1><<<ga, THREADS, 0, st>>>(prm)));
  if (c->ntt_rows == 8) {
    dim3 gb(H / 8, prm.n_limbs, npoly);
    PROF_LAUNCH(c, PK_NTT_FWD_B, units, (fwd_pass_b<LH, 8><<<gb, threads_b<8>(), 0, st>>>(prm, 0)));
  } else {
    dim3 gb(H / 16, prm.n_limbs, npoly);
    PROF_LAUNCH(c, PK_NTT_FWD_B, units, (fwd_pass_b<LH, 16><<<gb, threads_b<16>(), 0, st>>>(prm, 0)));
  }
}

}  // namespace

int launch_ntt(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl, const int *mods,
               bool inverse) {
  if (npoly <= 0 || nl <= 0) return CKKS_OK;
  if (nl > MAX_MODS) return CKKS_E_PARAM;
  NttParams prm;
  prm.mods = c->d_mods;
  prm.tw = inverse ? c->d_tw_inv : c->d_tw_fwd;
  prm.tw_row = inverse ? c->d_tw_row_inv : c->d_tw_row_fwd;
  prm.n = c->n;
  prm.n_limbs = nl;
  bool approx = true;  // inverse: every modulus below 2^61
  int strict = 0;      // forward: limbs whose prime takes the strict butterfly
  for (int l = 0; l < nl; ++l) {
    prm.mod_of_limb[l] = (unsigned char)mods[l];
    approx = approx && c->mod[mods[l]] < APPROX_INV_BOUND;
    strict += c->mod[mods[l]] >= LOOSE_BOUND ? 1 : 0;
  }
  if (inverse && !approx) c->prof.count(PK_NTT_INV_EXACT, (unsigned long long)nl * npoly);
  if (!inverse) c->prof.count(PK_NTT_FWD_STRICT, (unsigned long long)strict * npoly);
  for (int i = 0; i < npoly; ++i)  // the row passes move 16-byte words
    if (((uintptr_t)src[i] | (uintptr_t)dst[i]) & 15) return CKKS_E_PARAM;
  for (int p0 = 0; p0 < npoly; p0 += MAX_POLYS) {
    const int cnt = npoly - p0 < MAX_POLYS ? npoly - p0 : MAX_POLYS;
    for (int i = 0; i < cnt; ++i) {
      prm.src.p[i] = src[p0 + i];
      prm.dst.p[i] = dst[p0 + i];
    }
    switch (c->log_n - LB) {
      case 2: launch_lh<2>(c, prm, cnt, inverse, approx); break;
      case 3: launch_lh<3>(c, prm, cnt, inverse, approx); break;
      case 4: launch_lh<4>(c, prm, cnt, inverse, approx); break;
      case 5: launch_lh<5>(c, prm, cnt, inverse, approx); break;
      case 6: launch_lh<6>(c, prm, cnt, inverse, approx); break;
      case 7: launch_lh<7>(c, prm, cnt, inverse, approx); break;
      case 8: launch_lh<8>(c, prm, cnt, inverse, approx); break;
      case 9: launch_lh<9>(c, prm, cnt, inverse, approx); break;
      default: return CKKS_E_PARAM;
    }
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}
