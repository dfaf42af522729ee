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
#include <cooperative_groups.h>

#include <algorithm>

#include "ops.cuh"

namespace cg = cooperative_groups;

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
  int skip_first;                // pass A: the first S1 column stages ran elsewhere
  unsigned char mod_of_limb[MAX_MODS];
  CPolyPtrs src;
  PolyPtrs dst;
};

// Final reduction of a loose forward output r < 65 q to [0, q), s = floor(2^64 / q).
// For q > 2^32 (s < 2^32) the quotient k = floor(r_hi s / 2^32), r_hi =
// floor(r / 2^32), satisfies floor(r/q) - 2 <= k <= r/q: the terms it drops
// are below r / 2^64 < 1 and 2^32 / q < 1.  So r - k q lies in [0, 3q), from
// one 32-bit high multiply and a 32 x 64 product instead of the 64 x 64 Barrett
// quotient (kept for q < 2^32, whose result lies in [0, 2q)).
__device__ __forceinline__ u64 reduce_loose_out(u64 r, u64 q, u64 one_s) {
  if (one_s >> 32) {
    r -= __umul64hi(r, one_s) * q;
  } else {
    r -= (u64)__umulhi((u32)(r >> 32), (u32)one_s) * q;
    if (r >= 2 * q) r -= 2 * q;
  }
  return r >= q ? r - q : r;
}

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
    if (!prm.skip_first) fwd_step<S1, LOOSE>(v, 1u, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S1); ++e) sm[(r0 + (e << S2)) * CA + c] = v[e];
  }
  if constexpr ((1 << S1) * CA == THREADS) {
    // one group per thread: its twiddles are loaded before the barrier
    const int c = threadIdx.x % CA, g = threadIdx.x / CA;
    ulonglong2 twv[(1 << S2) - 1];
#pragma unroll
    for (int s = 0; s < S2; ++s)
#pragma unroll
      for (int i = 0; i < (1 << s); ++i) twv[(1 << s) - 1 + i] = __ldg(&tw[(((1u << S1) + g) << s) + i]);
    __syncthreads();
    u64 v[1 << S2];
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) v[e] = sm[((g << S2) + e) * CA + c];
    fwd_step_t<S2, LOOSE>(v, [&](int s, int i) { return twv[(1 << s) - 1 + i]; }, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) dst[(size_t)((g << S2) + e) * BROW + c0 + c] = v[e];
  } else {
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

// One bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void l2_prefetch_bulk(const void *p, u32 bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The fused key-switch finish (RowFinish) of one row-pass tile: rows row0 ..
// row0 + RB - 1 of limb blockIdx.y, polynomial blockIdx.z, the transform's
// outputs in the padded tile `sm`.  Each thread finishes PER pairs (k, k + 1);
// UNR pairs' accumulator and base words are loaded before any is used.
template <int RB, int THREADS>
__device__ __forceinline__ void finish_tile(const RowFinish &f, const u64 *sm, int row0, u32 n, int log_n, u64 q) {
  constexpr int PER = RB * BROW / 2 / THREADS, UNR = 4;
  static_assert(PER % UNR == 0, "whole groups of pairs");
  const int poly = blockIdx.z, limb = blockIdx.y;
  const size_t lo = (size_t)limb * n + (size_t)row0 * BROW;
  const ulonglong2 *a2 = reinterpret_cast<const ulonglong2 *>(f.acc[poly] + lo);
  ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(f.out[poly] + lo);
  const u64 *base = f.base[poly];
  const u32 g = f.gal[poly];
  const u64 w = f.w[2 * limb], ws = f.w[2 * limb + 1];
  const bool scaled = f.wb != nullptr;
  const u64 wb = scaled ? f.wb[2 * limb] : 0, wbs = scaled ? f.wb[2 * limb + 1] : 0;
#pragma unroll 1
  for (int i0 = 0; i0 < PER; i0 += UNR) {
    ulonglong2 av[UNR], bv[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) av[j] = a2[threadIdx.x + (i0 + j) * THREADS];
    if (base) {
      if (g == 1) {
        const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(base + lo);
#pragma unroll
        for (int j = 0; j < UNR; ++j) bv[j] = b2[threadIdx.x + (i0 + j) * THREADS];
      } else {
        const u64 *bl = base + (size_t)limb * n;
#pragma unroll
        for (int j = 0; j < UNR; ++j) {
          const u32 k = (u32)(row0 * BROW + 2 * (threadIdx.x + (i0 + j) * THREADS));
          bv[j] = make_ulonglong2(bl[gal_src(k, g, n, log_n)], bl[gal_src(k + 1, g, n, log_n)]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int x = threadIdx.x + (i0 + j) * THREADS, o = padb(2 * x);
      u64 r0 = shoup(submod(av[j].x, sm[o], q), w, ws, q), r1 = shoup(submod(av[j].y, sm[o + 1], q), w, ws, q);
      if (base) {
        u64 b0 = bv[j].x, b1 = bv[j].y;
        if (scaled) {
          b0 = shoup(b0, wb, wbs, q);
          b1 = shoup(b1, wb, wbs, q);
        }
        r0 = addmod(r0, b0, q);
        r1 = addmod(r1, b1, q);
      }
      o2[x] = make_ulonglong2(r0, r1);
    }
  }
}

// FIN: the output stage applies the key-switch finish `fin` (fwd_pass_b_fin)
// and stores to fin.out instead of dst.
template <int LH, bool LOOSE, int RB, bool FIN = false>
__device__ __forceinline__ void fwd_b_body(const NttParams &prm, u64 *sm, int mi, const u64 *src, u64 *dst,
                                           const RowFinish *fin = nullptr) {
  constexpr int H = 1 << LH, U1 = 4, U2 = LB - U1, THREADS = threads_b<RB>();
  const u64 q = prm.mods[mi].q, twoq = 2 * q;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int row0 = blockIdx.x * RB;
  if constexpr (FIN) {
    // the finish's accumulator rows (and base rows read as they are) are
    // needed only after the butterflies: start bringing them to L2 now
    if (threadIdx.x == 0) {
      const int poly = blockIdx.z;
      const size_t lo = (size_t)blockIdx.y * prm.n + (size_t)row0 * BROW;
      l2_prefetch_bulk(fin->acc[poly] + lo, RB * BROW * 8);
      if (fin->base[poly] && fin->gal[poly] == 1) l2_prefetch_bulk(fin->base[poly] + lo, RB * BROW * 8);
    }
  }
  for (int x = threadIdx.x; x < RB * (BROW >> U1); x += THREADS) {
    const int l0 = x % (BROW >> U1), rr = x / (BROW >> U1), b = row0 + rr;
    u64 v[1 << U1];
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) v[e] = src[(size_t)b * BROW + l0 + (e << U2)];
    fwd_step<U1, LOOSE>(v, (u32)(H + b), tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) sm[padb(rr * BROW + l0 + (e << U2))] = v[e];
  }
  // one 16-value group per thread in the second phase: its 15 twiddles (one
  // per block of each of the last four stages, all distinct per thread, from
  // L2) are loaded before the barrier, so their latency overlaps it
  static_assert(THREADS == (RB << U1), "one group per thread");
  const int g = threadIdx.x % (1 << U1), rr = threadIdx.x / (1 << U1), b = row0 + rr;
  ulonglong2 twv[(1 << U2) - 1];
  {
    const u32 n16 = prm.n / 16, m = ((u32)b << U1) + g;
    const ulonglong2 *twr = prm.tw_row + (size_t)mi * 15 * n16;
#pragma unroll
    for (int k = 0; k < (1 << U2) - 1; ++k) twv[k] = __ldg(&twr[(size_t)k * n16 + m]);
  }
  __syncthreads();
  {
    u64 v[1 << U2];
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) v[e] = sm[padb(rr * BROW + (g << U2) + e)];
    fwd_step_t<U2, LOOSE>(v, [&](int s, int i) { return twv[(1 << s) - 1 + i]; }, q, twoq);
    const u64 one_s = LOOSE ? prm.mods[mi].one_s : 0;
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) {
      u64 r = v[e];
      if (LOOSE) {  // r < 65 q
        r = reduce_loose_out(r, q, one_s);
      } else {      // r < 4 q
        if (r >= twoq) r -= twoq;
        if (r >= q) r -= q;
      }
      sm[padb(rr * BROW + (g << U2) + e)] = r;
    }
  }
  __syncthreads();
  if constexpr (FIN) {
    finish_tile<RB, THREADS>(*fin, sm, row0, prm.n, LH + LB, q);
    return;
  }
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

// The row pass with the key-switch finish in its output stage (RowFinish).
template <int LH, int RB>
__global__ void __launch_bounds__(threads_b<RB>(), RB == 16 ? 3 : 6)
    fwd_pass_b_fin(const NttParams prm, int from_src, const RowFinish fin) {
  __shared__ u64 sm[RB * BROW + (RB * BROW >> 4)];
  const int limb = blockIdx.y, poly = blockIdx.z;
  const int mi = prm.mod_of_limb[limb];
  const u64 *src = (from_src ? prm.src.p[poly] : prm.dst.p[poly]) + (size_t)limb * prm.n;
  if (prm.mods[mi].q < LOOSE_BOUND)
    fwd_b_body<LH, true, RB, true>(prm, sm, mi, src, nullptr, &fin);
  else
    fwd_b_body<LH, false, RB, true>(prm, sm, mi, src, nullptr, &fin);
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
  // one 16-value group per thread in the row stages: its 15 distinct twiddles
  // (from L2) are loaded before the barrier, so their latency overlaps it
  static_assert(THREADS == (RB << U1), "one group per thread");
  {
    const int g = threadIdx.x % (1 << U1), rr = threadIdx.x / (1 << U1), b = row0 + rr;
    ulonglong2 twv[(1 << U2) - 1];
    const u32 n16 = prm.n / 16, m = ((u32)b << U1) + g;
    const ulonglong2 *twr = prm.tw_row + (size_t)mi * 15 * n16;
#pragma unroll
    for (int k = 0; k < (1 << U2) - 1; ++k) twv[k] = __ldg(&twr[(size_t)k * n16 + m]);
    __syncthreads();
    u64 v[1 << U2];
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) v[e] = sm[padb(rr * BROW + (g << U2) + e)];
    inv_step_t<U2, APPROX, 0>(v, [&](int s, int i) { return twv[(1 << s) - 1 + i]; }, q, twoq);
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

void launch_fwd_cluster(ckks_ctx *c, const NttParams &prm, int npoly);

// part: NTT_BOTH, or one pass alone -- the inverse's row pass (NTT_ROWS) or the
// forward's row pass (NTT_ROWS, reading src) around a fused column pass.
template <int LH, int RB, bool APPROX>
void launch_inv(ckks_ctx *c, const NttParams &prm, int npoly, int part) {
  constexpr int S1 = (LH + 1) / 2;
  const unsigned long long units = (unsigned long long)prm.n_limbs * npoly;
  dim3 ga(BROW / ca_of(LH), prm.n_limbs, npoly), gb((1 << LH) / RB, prm.n_limbs, npoly);
  if (part & NTT_ROWS)
    PROF_LAUNCH(c, PK_NTT_INV_B, units, (inv_pass_b<LH, RB, APPROX><<<gb, threads_b<RB>(), 0, c->stream>>>(prm)));
  if (part & NTT_COLS)
    PROF_LAUNCH(c, PK_NTT_INV_A, units, (inv_pass_a<LH, S1, APPROX><<<ga, THREADS, 0, c->stream>>>(prm)));
}

template <int LH>
void launch_lh(ckks_ctx *c, const NttParams &prm, int npoly, bool inverse, bool approx, int part,
               const RowFinish *fin = nullptr) {
  if (inverse) {
    if (c->ntt_rows == 8)
      approx ? launch_inv<LH, 8, true>(c, prm, npoly, part) : launch_inv<LH, 8, false>(c, prm, npoly, part);
    else
      approx ? launch_inv<LH, 16, true>(c, prm, npoly, part) : launch_inv<LH, 16, false>(c, prm, npoly, part);
    return;
  }
  constexpr int S1 = (LH + 1) / 2;
  const int H = 1 << LH;
  cudaStream_t st = c->stream;
  const unsigned long long units = (unsigned long long)prm.n_limbs * npoly;
  if (LH == 8 && part == NTT_BOTH && c->ntt_cluster && !prm.skip_first && !fin) {
    launch_fwd_cluster(c, prm, npoly);
    return;
  }
  dim3 ga(BROW / ca_of(LH), prm.n_limbs, npoly);
  if (part & NTT_COLS) PROF_LAUNCH(c, PK_NTT_FWD_A, units, (fwd_pass_a<LH, S1><<<ga, THREADS, 0, st>>>(prm)));
  if (!(part & NTT_ROWS)) return;
  const int from_src = (part & NTT_COLS) ? 0 : 1;
  if (fin) {
    if ((c->fin_rows ? c->fin_rows : c->ntt_rows) == 8) {
      dim3 gb(H / 8, prm.n_limbs, npoly);
      PROF_LAUNCH(c, PK_NTT_FWD_FINISH, units,
                  (fwd_pass_b_fin<LH, 8><<<gb, threads_b<8>(), 0, st>>>(prm, from_src, *fin)));
    } else {
      dim3 gb(H / 16, prm.n_limbs, npoly);
      PROF_LAUNCH(c, PK_NTT_FWD_FINISH, units,
                  (fwd_pass_b_fin<LH, 16><<<gb, threads_b<16>(), 0, st>>>(prm, from_src, *fin)));
    }
    return;
  }
  if (c->ntt_rows == 8) {
    dim3 gb(H / 8, prm.n_limbs, npoly);
    PROF_LAUNCH(c, PK_NTT_FWD_B, units, (fwd_pass_b<LH, 8><<<gb, threads_b<8>(), 0, st>>>(prm, from_src)));
  } else {
    dim3 gb(H / 16, prm.n_limbs, npoly);
    PROF_LAUNCH(c, PK_NTT_FWD_B, units, (fwd_pass_b<LH, 16><<<gb, threads_b<16>(), 0, st>>>(prm, from_src)));
  }
}

// ---------------------------------------------------------------- one-pass forward transform on a cluster
// N = 2^16: the limb (256 rows x 256 words, 512 KiB) is spread over a cluster of
// eight CTAs, 64 KiB of shared memory each, so it crosses HBM once (read once,
// written once) instead of twice.
//   phase 1: CTA r loads columns 32r .. 32r+31 (all rows) and runs the eight
//            column stages (pass A's two register phases, exchange in its tile);
//   cluster barrier;
//   phase 2: CTA r gathers rows 32r .. 32r+31 from the eight tiles through
//            distributed shared memory and runs the first four row stages in
//            registers; a second cluster barrier (every remote read done) frees
//            the tile for the row exchange; the last four row stages, the final
//            reduction and a contiguous store follow (pass B's steps).
// Every value goes through the same butterflies in the same order as
// fwd_pass_a then fwd_pass_b, so the output is bit-identical.  Both cluster
// barriers are reached by every thread: the only branch (loose or strict
// prime) is uniform over the cluster, which holds one limb.
constexpr int NC = 8;                    // CTAs per cluster
constexpr int NC_THREADS = 256;
constexpr int NC_IT = 512 / NC_THREADS;  // 16-value groups per thread in each phase
constexpr int NC_CA = BROW / NC;         // 32 columns per CTA in phase 1
constexpr int NC_RB = 256 / NC;          // 32 rows per CTA in phase 2
constexpr int NC_SMEM_WORDS = NC_RB * BROW + (NC_RB * BROW >> 4);  // the padded row buffer (>= 256 x 32)

template <bool LOOSE>
__device__ __forceinline__ void fwd_cluster_body(const NttParams &prm, u64 *sm, int mi, const u64 *src, u64 *dst,
                                                 cg::cluster_group &cl) {
  constexpr int H = 256, S1 = 4, S2 = 4, U1 = 4, U2 = 4;
  const u64 q = prm.mods[mi].q, twoq = 2 * q;
  const ulonglong2 *tw = prm.tw + (size_t)mi * prm.n;
  const int rank = (int)cl.block_rank();
  const int c0 = rank * NC_CA;
  {  // column stages 0..3: rows r0 + 16 e of column c0 + c, every load issued first
    u64 v[NC_IT][1 << S1];
#pragma unroll
    for (int it = 0; it < NC_IT; ++it) {
      const int x = threadIdx.x + it * NC_THREADS, c = x % NC_CA, r0 = x / NC_CA;
#pragma unroll
      for (int e = 0; e < (1 << S1); ++e) v[it][e] = src[(size_t)(r0 + (e << S2)) * BROW + c0 + c];
    }
#pragma unroll
    for (int it = 0; it < NC_IT; ++it) {
      const int x = threadIdx.x + it * NC_THREADS, c = x % NC_CA, r0 = x / NC_CA;
      fwd_step<S1, LOOSE>(v[it], 1u, tw, q, twoq);
#pragma unroll
      for (int e = 0; e < (1 << S1); ++e) sm[(r0 + (e << S2)) * NC_CA + c] = v[it][e];
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < NC_IT; ++it) {  // column stages 4..7: rows 16 g + e
    const int x = threadIdx.x + it * NC_THREADS, c = x % NC_CA, g = x / NC_CA;
    u64 v[1 << S2];
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) v[e] = sm[((g << S2) + e) * NC_CA + c];
    fwd_step<S2, LOOSE>(v, (1u << S1) + g, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) sm[((g << S2) + e) * NC_CA + c] = v[e];
  }
  cl.sync();  // every CTA's columns are transformed
  u64 v[NC_IT][1 << U1];
#pragma unroll
  for (int it = 0; it < NC_IT; ++it) {
    const int x = threadIdx.x + it * NC_THREADS, l0 = x % (BROW >> U1), rr = x / (BROW >> U1);
    const int b = rank * NC_RB + rr;
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) {  // word l0 + 16 e of row b lives in CTA (l0 + 16 e) / 32
      const int col = l0 + (e << U2);
      const u64 *rem = cl.map_shared_rank(sm, col / NC_CA);
      v[it][e] = rem[b * NC_CA + col % NC_CA];
    }
  }
#pragma unroll
  for (int it = 0; it < NC_IT; ++it) {
    const int x = threadIdx.x + it * NC_THREADS, rr = x / (BROW >> U1);
    fwd_step<U1, LOOSE>(v[it], (u32)(H + rank * NC_RB + rr), tw, q, twoq);
  }
  cl.sync();  // every remote read is done: the tile becomes the row buffer
#pragma unroll
  for (int it = 0; it < NC_IT; ++it) {
    const int x = threadIdx.x + it * NC_THREADS, l0 = x % (BROW >> U1), rr = x / (BROW >> U1);
#pragma unroll
    for (int e = 0; e < (1 << U1); ++e) sm[padb(rr * BROW + l0 + (e << U2))] = v[it][e];
  }
  __syncthreads();
  const u64 one_s = LOOSE ? prm.mods[mi].one_s : 0;
#pragma unroll 1
  for (int it = 0; it < NC_IT; ++it) {
    const int x = threadIdx.x + it * NC_THREADS, g = x % (1 << U1), r2 = x / (1 << U1);
    const int b2 = rank * NC_RB + r2;
    u64 w[1 << U2];
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) w[e] = sm[padb(r2 * BROW + (g << U2) + e)];
    fwd_step_row<U2, LOOSE>(w, ((u32)b2 << U1) + g, prm.tw_row + (size_t)mi * 15 * (prm.n / 16), prm.n / 16, q,
                            twoq);
#pragma unroll
    for (int e = 0; e < (1 << U2); ++e) {
      u64 r = w[e];
      if (LOOSE) {
        r = reduce_loose_out(r, q, one_s);
      } else {
        if (r >= twoq) r -= twoq;
        if (r >= q) r -= q;
      }
      sm[padb(r2 * BROW + (g << U2) + e)] = r;
    }
  }
  __syncthreads();
  ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(dst + (size_t)rank * NC_RB * BROW);
#pragma unroll 4
  for (int y = threadIdx.x; y < NC_RB * BROW / 2; y += NC_THREADS) {
    const int o = padb(2 * y);
    d2[y] = make_ulonglong2(sm[o], sm[o + 1]);
  }
}

__global__ void __cluster_dims__(NC, 1, 1) __launch_bounds__(NC_THREADS, 2) fwd_cluster(const NttParams prm) {
  extern __shared__ u64 csm[];
  cg::cluster_group cl = cg::this_cluster();
  const int limb = blockIdx.y, poly = blockIdx.z;
  const int mi = prm.mod_of_limb[limb];
  const u64 *src = prm.src.p[poly] + (size_t)limb * prm.n;
  u64 *dst = prm.dst.p[poly] + (size_t)limb * prm.n;
  if (prm.mods[mi].q < LOOSE_BOUND)
    fwd_cluster_body<true>(prm, csm, mi, src, dst, cl);
  else
    fwd_cluster_body<false>(prm, csm, mi, src, dst, cl);
}

constexpr size_t NC_SMEM_BYTES = NC_SMEM_WORDS * sizeof(u64);

// Launch errors stay pending for the caller's cudaGetLastError.
void launch_fwd_cluster(ckks_ctx *c, const NttParams &prm, int npoly) {
  const unsigned long long units = (unsigned long long)prm.n_limbs * npoly;
  dim3 g(NC, prm.n_limbs, npoly);
  PROF_LAUNCH(c, PK_NTT_FWD_CLUSTER, units, (fwd_cluster<<<g, NC_THREADS, NC_SMEM_BYTES, c->stream>>>(prm)));
}

// Opt the kernel into its dynamic shared memory and check that the device can
// hold at least one cluster of it: CKKS_E_PARAM off N = 2^16, CKKS_E_CUDA when
// the attribute or the occupancy query fails or no cluster fits.
int prepare_fwd_cluster(const ckks_ctx *c, int *max_clusters) {
  if (c->log_n != 16) return CKKS_E_PARAM;
  if (cudaFuncSetAttribute(fwd_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NC_SMEM_BYTES) !=
      cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_CUDA;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC, 1, 1);
  cfg.blockDim = dim3(NC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = NC_SMEM_BYTES;
  int nclu = 0;
  if (cudaOccupancyMaxActiveClusters(&nclu, fwd_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_CUDA;
  }
  if (max_clusters) *max_clusters = nclu;
  return nclu > 0 ? CKKS_OK : CKKS_E_CUDA;
}

// ---------------------------------------------------------------- fused conversion column pass
// The middle of the key-switch pipeline in one kernel (readings C8, C9, C21):
// a CTA takes one tile of FCA columns x H rows of one polynomial and one digit,
//   A. runs the inverse transform's column stages on each of the digit's
//      source limbs (their row stages ran before, NTT_ROWS), with N^-1, and
//      multiplies by [Bhat_i^-1]_{b_i}: y_i in shared memory;
//   B. for each target t: y_t = sum_i y_i (Bhat_i mod t) mod t at every
//      position of the tile (128-bit sums, one reduction), then the forward
//      transform's column stages, and stores the tile (its row stages run
//      after, NTT_ROWS).
// So the digit's coefficient-domain limbs and the conversion's targets never
// reach HBM: the sources are read once after their row pass, the targets
// written once before theirs.  The arithmetic per value is the unfused
// path's (same lazy butterflies per modulus, same conversion), so the limbs
// are identical.  MERGED adds reading C21's terms: [H]_{s_i} on the sources,
// the overflow estimate v (32.32 fixed point) times -S mod t, and -[H]_t.
constexpr int FCA = 4;          // columns per tile: 32-byte row segments
constexpr int F_THREADS = 256;
constexpr int F_MAXS = 16;      // sources of one conversion
constexpr int F_MAXD = 8;       // digits per launch
// shared-memory word index of (row, column) in a padded tile: four spare words
// per 16 rows keep the 16-row strided accesses free of bank conflicts
__host__ __device__ constexpr int fpad(int r, int c) { return FCA * (r + (r >> 4)) + c; }
__host__ __device__ constexpr int ftile(int lh) { return FCA * ((1 << lh) + ((1 << lh) >> 4)); }

struct FusedArgs {
  const ModInfo *mods;
  const ulonglong2 *tw_inv, *tw_fwd;   // [modulus][N]
  u32 n;
  // per digit (blockIdx.y): sources = limbs src_off .. +ns of the polynomial's
  // source buffer (moduli src_mod); targets tt < nt go to limb pos(tt) of the
  // digit's target buffer (dst_off), pos(tt) = tt below gap_lo and
  // tt + gap_hi - gap_lo from there (the digit's own limbs are skipped)
  int ns[F_MAXD], nt[F_MAXD], gap_lo[F_MAXD], gap_hi[F_MAXD];
  size_t src_off[F_MAXD], dst_off[F_MAXD];
  unsigned char src_mod[F_MAXD][F_MAXS];
  unsigned char pos_mod[MAX_MODS];     // modulus of target limb position
  const u64 *inv[F_MAXD];              // [ns] Shoup pairs: [Bhat_i^-1]_{b_i}
  const u64 *tab[F_MAXD];              // [nt][ns]: Bhat_i mod t
  const u64 *src_add, *dst_sub, *rdiv, *negs;  // MERGED: [ns], [nt], [2][ns] (low, high words), [nt]
  const u64 *src[MAX_CTS];
  u64 *dst[MAX_CTS];
};

template <int LH, bool MERGED>
__global__ void __launch_bounds__(F_THREADS, 2) k_conv_fused(const FusedArgs a) {
  constexpr int H = 1 << LH, S1 = (LH + 1) / 2, S2 = LH - S1, T = ftile(LH);
  constexpr int PER_T = (H >> S1) * FCA;    // threads per target in phase B
  constexpr int TCON = F_THREADS / PER_T;   // targets in flight
  static_assert(F_THREADS % PER_T == 0, "phase B groups");
  extern __shared__ u64 fsm[];
  const int j = blockIdx.y, p = blockIdx.z;
  const int ns = a.ns[j], nt = a.nt[j];
  u64 *sy = fsm;                          // [ns][T]: the sources, then y
  u64 *sx = sy + (size_t)ns * T;          // [TCON][T]: phase B exchange tiles
  u64 *stab = sx + (size_t)TCON * T;      // [nt][ns] conversion constants
  const int c0 = blockIdx.x * FCA;
  const u64 *src = a.src[p] + a.src_off[j];
  u64 *dst = a.dst[p] + a.dst_off[j];
  for (int x = threadIdx.x; x < nt * ns; x += F_THREADS) stab[x] = __ldg(a.tab[j] + x);

  // A.1 inverse column stages S1 .. LH-1 (rows (g << S2) + e), from global
  for (int x = threadIdx.x; x < ns * (1 << S1) * FCA; x += F_THREADS) {
    const int i = x / ((1 << S1) * FCA), r = x % ((1 << S1) * FCA);
    const int c = r % FCA, g = r / FCA;
    const int mi = a.src_mod[j][i];
    const u64 q = a.mods[mi].q, twoq = 2 * q;
    const ulonglong2 *tw = a.tw_inv + (size_t)mi * a.n;
    const u64 *sl = src + (size_t)i * a.n;
    u64 v[1 << S2];
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) v[e] = sl[(size_t)((g << S2) + e) * BROW + c0 + c];
    if (q < APPROX_INV_BOUND)
      inv_step<S2, true>(v, (1u << S1) + g, tw, q, twoq);
    else
      inv_step<S2, false>(v, (1u << S1) + g, tw, q, twoq);
#pragma unroll
    for (int e = 0; e < (1 << S2); ++e) sy[i * T + fpad((g << S2) + e, c)] = v[e];
  }
  __syncthreads();
  // A.2 the remaining stages with N^-1, then y = x [Bhat_i^-1]_{b_i} (+ [H]_{b_i})
  for (int x = threadIdx.x; x < ns * (H >> S1) * FCA; x += F_THREADS) {
    const int i = x / ((H >> S1) * FCA), r = x % ((H >> S1) * FCA);
    const int c = r % FCA, r0 = r / FCA;
    const int mi = a.src_mod[j][i];
    const ModInfo m = a.mods[mi];
    const u64 q = m.q, twoq = 2 * q;
    const bool approx = q < APPROX_INV_BOUND;
    const ulonglong2 *tw = a.tw_inv + (size_t)mi * a.n;
    u64 v[1 << S1];
#pragma unroll
    for (int e = 0; e < (1 << S1); ++e) v[e] = sy[i * T + fpad(r0 + (e << S2), c)];
    if (approx)
      inv_step<S1, true, 1>(v, 1u, tw, q, twoq);
    else
      inv_step<S1, false, 1>(v, 1u, tw, q, twoq);
    const u64 rr = approx ? 2 * twoq : twoq;
    const ulonglong2 w0 = __ldg(&tw[0]);
    const u64 iw = __ldg(a.inv[j] + 2 * i), iws = __ldg(a.inv[j] + 2 * i + 1);
    const u64 add = MERGED ? __ldg(a.src_add + i) : 0;
    constexpr int HALF = 1 << (S1 - 1);
#pragma unroll
    for (int e = 0; e < HALF; ++e) {
      const u64 xa = v[e], xb = v[e + HALF];
      u64 ya = shoup(shoup(xa + xb, m.ninv, m.ninv_s, q), iw, iws, q);
      u64 yb = shoup(shoup(xa + rr - xb, w0.x, w0.y, q), iw, iws, q);
      if (MERGED) {
        ya = addmod(ya, add, q);
        yb = addmod(yb, add, q);
      }
      sy[i * T + fpad(r0 + (e << S2), c)] = ya;
      sy[i * T + fpad(r0 + ((e + HALF) << S2), c)] = yb;
    }
  }
  __syncthreads();

  // B. per target: conversion at the tile's positions, forward column stages
  const int grp = threadIdx.x / PER_T, lt = threadIdx.x % PER_T;
  const int gl = a.gap_lo[j], gh = a.gap_hi[j];
  u64 *xt = sx + grp * T;
  for (int t0 = 0; t0 < nt; t0 += TCON) {
    const int tt = t0 + grp;
    const bool act = tt < nt;
    const int pos = tt < gl ? tt : tt + (gh - gl);
    const int mi = act ? a.pos_mod[pos] : 0;
    const ModInfo m = a.mods[mi];
    const u64 q = m.q, twoq = 2 * q;
    const bool loose = q < LOOSE_BOUND;
    const ulonglong2 *tw = a.tw_fwd + (size_t)mi * a.n;
    if (act) {
      const int c = lt % FCA, r0 = lt / FCA;
      const u64 *crow = stab + tt * ns;
      const u64 ng = MERGED ? __ldg(a.negs + tt) : 0, ds = MERGED ? __ldg(a.dst_sub + tt) : 0;
      u64 v[1 << S1];
      // sources outer, positions inner, in halves: FH independent 128-bit sums
      // per thread at a time (the other half's results wait in v)
      constexpr int FH = (1 << S1) > 8 ? 8 : (1 << S1);
#pragma unroll
      for (int h = 0; h < (1 << S1); h += FH) {
        u64 hi[FH], lo[FH], fix[FH];
#pragma unroll
        for (int e = 0; e < FH; ++e) hi[e] = lo[e] = fix[e] = 0;
        for (int i = 0; i < ns; ++i) {
          const u64 cf = crow[i];
          const u64 rd = MERGED ? __ldg(a.rdiv + i) : 0, rd_hi = MERGED ? __ldg(a.rdiv + ns + i) : 0;
          const u64 *yi = sy + i * T;
#pragma unroll
          for (int e = 0; e < FH; ++e) {
            const u64 y = yi[fpad(r0 + ((h + e) << S2), c)];
            mac128(hi[e], lo[e], y, cf);
            if (MERGED) fix[e] += __umul64hi(y, rd) + y * rd_hi;
          }
        }
#pragma unroll
        for (int e = 0; e < FH; ++e) {
          if (MERGED) mac128(hi[e], lo[e], fix[e] >> 32, ng);
          u64 r = reduce128(hi[e], lo[e], m);
          if (MERGED) r = submod(r, ds, q);
          v[h + e] = r;
        }
      }
      if (loose)
        fwd_step<S1, true>(v, 1u, tw, q, twoq);
      else
        fwd_step<S1, false>(v, 1u, tw, q, twoq);
#pragma unroll
      for (int e = 0; e < (1 << S1); ++e) xt[fpad(r0 + (e << S2), c)] = v[e];
    }
    __syncthreads();
    if (act) {
      u64 *dl = dst + (size_t)pos * a.n;
      for (int x = lt; x < (1 << S1) * FCA; x += PER_T) {
        const int c = x % FCA, g = x / FCA;
        u64 v[1 << S2];
#pragma unroll
        for (int e = 0; e < (1 << S2); ++e) v[e] = xt[fpad((g << S2) + e, c)];
        if (loose)
          fwd_step<S2, true>(v, (1u << S1) + g, tw, q, twoq);
        else
          fwd_step<S2, false>(v, (1u << S1) + g, tw, q, twoq);
#pragma unroll
        for (int e = 0; e < (1 << S2); ++e) dl[(size_t)((g << S2) + e) * BROW + c0 + c] = v[e];
      }
    }
    __syncthreads();  // xt is rewritten by the next target
  }
}

template <int LH>
int launch_fused_lh(ckks_ctx *c, const FusedArgs &a, int ndig, int np, size_t smem, bool merged) {
  dim3 g(BROW / FCA, ndig, np);
  u64 pairs = 0, srcs = 0, dsts = 0, strict = 0;
  for (int j = 0; j < ndig; ++j) {
    pairs += (u64)a.ns[j] * a.nt[j];
    srcs += (u64)a.ns[j];
    dsts += (u64)a.nt[j];
    for (int tt = 0; tt < a.nt[j]; ++tt) {
      const int pos = tt < a.gap_lo[j] ? tt : tt + (a.gap_hi[j] - a.gap_lo[j]);
      strict += c->mod[a.pos_mod[pos]] >= LOOSE_BOUND ? 1 : 0;
    }
  }
  c->prof.count(PK_FUSED_SRC_LIMBS, srcs * np);
  c->prof.count(PK_FUSED_DST_LIMBS, dsts * np);
  c->prof.count(PK_FUSED_DST_STRICT, strict * np);
  if (merged) {
    CK_CUDA(cudaFuncSetAttribute(k_conv_fused<LH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PROF_LAUNCH(c, PK_CONV_FUSED, pairs * np, (k_conv_fused<LH, true><<<g, F_THREADS, smem, c->stream>>>(a)));
  } else {
    CK_CUDA(cudaFuncSetAttribute(k_conv_fused<LH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PROF_LAUNCH(c, PK_CONV_FUSED, pairs * np, (k_conv_fused<LH, false><<<g, F_THREADS, smem, c->stream>>>(a)));
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

}  // namespace

int ntt_cluster_prepare(const ckks_ctx *c, int *max_clusters) { return prepare_fwd_cluster(c, max_clusters); }

static int launch_ntt_impl(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl, const int *mods,
                           bool inverse, int part, const RowFinish *fin) {
  if (npoly <= 0 || nl <= 0) return CKKS_OK;
  if (part != NTT_BOTH && part != NTT_ROWS) return CKKS_E_PARAM;
  if (nl > MAX_MODS) return CKKS_E_PARAM;
  if (fin) {  // one launch set, the 16-byte words of the output stage
    if (inverse || npoly > MAX_POLYS || !fin->w) return CKKS_E_PARAM;
    unsigned long long with_base = 0;
    for (int i = 0; i < npoly; ++i) {
      uintptr_t a = (uintptr_t)fin->acc[i] | (uintptr_t)fin->out[i];
      if (fin->base[i] && fin->gal[i] == 1) a |= (uintptr_t)fin->base[i];
      if (!fin->acc[i] || !fin->out[i] || (a & 15)) return CKKS_E_PARAM;
      if (fin->base[i] && fin->gal[i] != 1 && (fin->wb || !(fin->gal[i] & 1))) return CKKS_E_PARAM;
      with_base += fin->base[i] ? 1 : 0;
    }
    c->prof.count(PK_FINISH_BASE_LIMBS, with_base * nl);
  }
  NttParams prm;
  prm.skip_first = 0;
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
  if (!inverse && (part & NTT_COLS)) c->prof.count(PK_NTT_FWD_STRICT, (unsigned long long)strict * npoly);
  for (int i = 0; i < npoly; ++i)  // the row passes move 16-byte words
    if (((uintptr_t)src[i] | (uintptr_t)dst[i]) & 15) return CKKS_E_PARAM;
  for (int p0 = 0; p0 < npoly; p0 += MAX_POLYS) {
    const int cnt = npoly - p0 < MAX_POLYS ? npoly - p0 : MAX_POLYS;
    for (int i = 0; i < cnt; ++i) {
      prm.src.p[i] = src[p0 + i];
      prm.dst.p[i] = dst[p0 + i];
    }
    switch (c->log_n - LB) {
      case 2: launch_lh<2>(c, prm, cnt, inverse, approx, part, fin); break;
      case 3: launch_lh<3>(c, prm, cnt, inverse, approx, part, fin); break;
      case 4: launch_lh<4>(c, prm, cnt, inverse, approx, part, fin); break;
      case 5: launch_lh<5>(c, prm, cnt, inverse, approx, part, fin); break;
      case 6: launch_lh<6>(c, prm, cnt, inverse, approx, part, fin); break;
      case 7: launch_lh<7>(c, prm, cnt, inverse, approx, part, fin); break;
      case 8: launch_lh<8>(c, prm, cnt, inverse, approx, part, fin); break;
      case 9: launch_lh<9>(c, prm, cnt, inverse, approx, part, fin); break;
      default: return CKKS_E_PARAM;
    }
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

int launch_ntt_part(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl, const int *mods,
                    bool inverse, int part) {
  return launch_ntt_impl(c, src, dst, npoly, nl, mods, inverse, part, nullptr);
}

int launch_ntt_fwd_finish(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl, const int *mods,
                          int part, const RowFinish &f) {
  return launch_ntt_impl(c, src, dst, npoly, nl, mods, false, part, &f);
}

int launch_ntt(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl, const int *mods,
               bool inverse) {
  return launch_ntt_part(c, src, dst, npoly, nl, mods, inverse, NTT_BOTH);
}

// Host side of the fused column pass (see k_conv_fused).  Rings of 2^12..2^16
// (the 2^17 ring's pass A runs three register phases and is not fused).
bool conv_fused_supported(const ckks_ctx *c) { return c->log_n >= 12 && c->log_n <= 16; }

int launch_conv_fused(ckks_ctx *c, const FusedConv &f, const u64 *const *src, u64 *const *dst, int np) {
  if (!conv_fused_supported(c) || f.ndig < 1 || f.ndig > F_MAXD || np < 1 || np > MAX_CTS) return CKKS_E_PARAM;
  FusedArgs a;
  a.mods = c->d_mods;
  a.tw_inv = c->d_tw_inv;
  a.tw_fwd = c->d_tw_fwd;
  a.n = c->n;
  int max_ns = 0, max_tab = 0;
  for (int j = 0; j < f.ndig; ++j) {
    const FusedConv::Digit &d = f.dig[j];
    if (d.ns < 1 || d.ns > F_MAXS || d.nt < 1 || d.nt > MAX_MODS) return CKKS_E_PARAM;
    a.ns[j] = d.ns;
    a.nt[j] = d.nt;
    a.gap_lo[j] = d.gap_lo;
    a.gap_hi[j] = d.gap_hi;
    a.src_off[j] = d.src_off;
    a.dst_off[j] = d.dst_off;
    for (int i = 0; i < d.ns; ++i) a.src_mod[j][i] = (unsigned char)d.src_mod[i];
    a.inv[j] = d.inv;
    a.tab[j] = d.tab;
    max_ns = std::max(max_ns, d.ns);
    max_tab = std::max(max_tab, d.ns * d.nt);
  }
  for (int t = 0; t < MAX_MODS; ++t) a.pos_mod[t] = (unsigned char)f.pos_mod[t];
  a.src_add = f.src_add;
  a.dst_sub = f.dst_sub;
  a.rdiv = f.rdiv;
  a.negs = f.negs;
  const bool merged = f.src_add != nullptr;
  if (merged && f.ndig != 1) return CKKS_E_PARAM;
  for (int i = 0; i < np; ++i) {
    a.src[i] = src[i];
    a.dst[i] = dst[i];
  }
  const int lh = c->log_n - LB;
  const int per_t = ((1 << lh) >> ((lh + 1) / 2)) * FCA;
  const size_t smem = sizeof(u64) * ((size_t)(max_ns + F_THREADS / per_t) * ftile(lh) + max_tab);
  if (smem > 227 * 1024) return CKKS_E_PARAM;
  switch (lh) {
    case 4: return launch_fused_lh<4>(c, a, f.ndig, np, smem, merged);
    case 5: return launch_fused_lh<5>(c, a, f.ndig, np, smem, merged);
    case 6: return launch_fused_lh<6>(c, a, f.ndig, np, smem, merged);
    case 7: return launch_fused_lh<7>(c, a, f.ndig, np, smem, merged);
    case 8: return launch_fused_lh<8>(c, a, f.ndig, np, smem, merged);
    default: return CKKS_E_PARAM;
  }
}

// ---------------------------------------------------------------- tensor-core NTT stage prototype
// The forward transform's first S1 = 4 column stages act on 16-point blocks
// (rows r0 + 16 e of one column) with the same twiddles for every block: the
// block transform is one 16 x 16 matrix M over Z_q, and applying it to a limb
// is the product M V with V the limb's 16-row slabs as 16 "sources" of N/16
// coefficients.  That product runs as the exact byte-split GEMM of the
// tensor-core conversion (fp16 bytes, fp32 accumulation in tensor memory,
// modular recombination, fully reduced residues); the remaining 12 stages run
// on the CUDA cores.  The result equals launch_ntt's bit for bit.
static void stage_matrix(const ckks_ctx *c, int mi, u64 *M) {  // M[16][16], row = output
  const u64 q = c->mod[mi];
  for (int j = 0; j < 16; ++j) {
    u64 v[16] = {0};
    v[j] = 1;
    for (int st = 0; st < 4; ++st) {  // Cooley-Tukey stages of the block, group mg = 1
      const int half = 8 >> st;
      for (int e = 0; e < 16; ++e) {
        if (e & half) continue;
        const u64 idx = (1u << st) + (u64)(e >> (4 - st));
        const u64 w = host_powmod(c->psi[mi], host_bitrev(idx, c->log_n), q);
        const u64 t = host_mulmod(w, v[e + half], q);
        const u64 a = v[e];
        v[e] = (a + t) % q;
        v[e + half] = (a + q - t) % q;
      }
    }
    for (int k = 0; k < 16; ++k) M[k * 16 + j] = v[k];
  }
}

extern "C" int ckks_ntt_tc(ckks_ctx *c, uint64_t *data, uint32_t n_polys, uint32_t n_limbs) {
  if (!c || !data || n_polys < 1 || n_polys > MAX_CTS || n_limbs < 1 || (int)n_limbs > c->n_q + c->n_p)
    return CKKS_E_PARAM;
  const int lh = c->log_n - LB;
  if (lh != 7 && lh != 8) return CKKS_E_PARAM;  // 16-point first phase: N = 2^15, 2^16
  if (c->capturing) return CKKS_E_STATE;
  const u32 n = c->n, nv = n / 16;
  int rc = ensure_scratch(c, (size_t)n_polys * n);
  if (rc) return rc;
  for (u32 t = 0; t < n_limbs; ++t) {
    const int mi = (int)t;
    u64 M[256], inv[32];
    stage_matrix(c, mi, M);
    for (int i = 0; i < 16; ++i) inv[2 * i] = 1, inv[2 * i + 1] = host_shoup(1, c->mod[mi]);
    int sm[16], dm[16], dp[16];
    for (int i = 0; i < 16; ++i) sm[i] = mi, dm[i] = mi, dp[i] = i;
    std::vector<const u64 *> src(n_polys);
    std::vector<u64 *> dst(n_polys);
    for (u32 p = 0; p < n_polys; ++p) {
      src[p] = data + ((size_t)p * n_limbs + t) * n;
      dst[p] = c->scratch + (size_t)p * n;
    }
    rc = launch_bconv_tc_view(c, ((size_t)1 << 62) | (size_t)mi, inv, M, 16, 16, sm, dm, dp, src.data(), dst.data(),
                              (int)n_polys, nv);
    if (rc) return rc;
    NttParams prm;
    prm.skip_first = 1;
    prm.mods = c->d_mods;
    prm.tw = c->d_tw_fwd;
    prm.tw_row = c->d_tw_row_fwd;
    prm.n = n;
    prm.n_limbs = 1;
    prm.mod_of_limb[0] = (unsigned char)mi;
    for (u32 p = 0; p < n_polys; ++p) {
      prm.src.p[p] = dst[p];
      prm.dst.p[p] = const_cast<u64 *>(src[p]);
    }
    if (lh == 8)
      launch_lh<8>(c, prm, (int)n_polys, false, true, NTT_BOTH);
    else
      launch_lh<7>(c, prm, (int)n_polys, false, true, NTT_BOTH);
    if (cudaGetLastError() != cudaSuccess) return CKKS_E_CUDA;
  }
  return CKKS_OK;
}
