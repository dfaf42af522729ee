// Fast basis conversion (reading C8) on the 5th-generation tensor cores,
// exact, as a byte-split GEMM.
//
//   y_t = sum_i y_i * c_(i,t)  mod t,   y_i = [x_i Bhat_i^-1]_(b_i) < 2^62,
//   c_(i,t) = Bhat_i mod t.
// Split y_i into bytes y_(i,a) (y_i = sum_a y_(i,a) 2^(8a)) and fold 2^(8a) into
// the constant: c'_(i,a,t) = 2^(8a) c_(i,t) mod t; split c' into bytes
// c'_(i,a,t,b).  Then
//   y_t = sum_b 2^(8b) sum_(i,a) y_(i,a) c'_(i,a,t,b)   mod t,
// where the inner sum is a GEMM  D[n][(t,b)] = sum_(i,a) A[n][(i,a)] B[(t,b)][(i,a)]
// with 8-bit operands (exact in fp16) and K = 8 * sources <= 128 terms, so every
// accumulator is an integer below 128 * 255 * 255 < 2^23, exact in fp32.
//
// Epilogue per target: adding 2^23 to an accumulator puts its integer in the low
// 23 mantissa bits (one FADD, no conversion unit); bytes 0..3 and 4..7 of the
// target are summed into S_lo, S_hi < 2^47.01, and y_t = S_lo + S_hi 2^32 is
// reduced by two Shoup products and two conditional subtractions.  The result is
// the fully reduced residue, bit-identical to the uint64 kernel.
//
// GB300 mapping: one persistent CTA of 16 warps per SM owns all 512 TMEM
// columns as two 128 x (8 targets, <= 256) fp32 accumulators and two A tiles in
// shared memory, so the MMAs of tile j+1 run on the tensor pipe while the 16
// warps recombine tile j:
//   build A(j+1) | sync | one thread issues MMA(j+1) -> mbar | wait mbar(j) | epilogue(j)
// A rows are written with 16-byte stores in the canonical K-major, no-swizzle
// layout; bytes become fp16 through PRMT (0x64bb = 1024 + b) and one HSUB2.
// Warp w reads TMEM lanes 32 (w mod 4) .. +31 (its coefficients) for the
// targets of column group w / 4.  B (the constants) is loaded into shared
// memory once per CTA.  Every wait is bounded: on expiry the kernel records an
// error flag, waits (bounded) for its MMAs in flight, frees its TMEM and returns.
// Flag values: 1 = a wait expired and no MMA was outstanding when the TMEM was
// freed; 2 = MMAs committed to the freed TMEM had still not completed after a
// second, longer bounded wait (the tensor memory was released under them).
#include <cuda_fp16.h>

#include <algorithm>

#include "ops.cuh"

namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 512;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_COL_GROUPS = TC_WARPS / 4;   // warps sharing one TMEM lane quarter
constexpr int TC_ACC_COLS = 256;              // columns per accumulator
constexpr int TC_TMEM_COLS = 2 * TC_ACC_COLS; // the whole TMEM of the SM
constexpr int TC_MAX_S = 16, TC_MAX_T = 32;
constexpr u64 TC_WAIT_NS = 1000000000ULL;     // bounded waits give up after about 1 s
constexpr u64 TC_DRAIN_NS = 4 * TC_WAIT_NS;   // the failure path's wait for MMAs in flight

__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u64 global_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin on an mbarrier phase for at most limit_ns; 1 when the phase completed.
__device__ __forceinline__ u32 wait_parity(u32 mbar_addr, u32 phase, u64 limit_ns) {
  const u64 t0 = global_ns();
  u32 done = 0;
  while (!done) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(mbar_addr), "r"(phase));
    if (!done && global_ns() - t0 > limit_ns) break;
  }
  return done;
}

// Canonical K-major, no-swizzle layout of an R x K fp16 operand: core matrices of
// 8 rows x 8 elements (16 bytes per row, 128 bytes each); adjacent along K at
// LBO = 128 bytes, adjacent along R at SBO = K/8 * 128 bytes.
__device__ __forceinline__ u32 canon_offset(int row, int k, int kpad) {
  return (u32)((row >> 3) * (kpad / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ u64 make_desc(u32 saddr, u32 lbo, u32 sbo) {
  return (u64)((saddr >> 4) & 0x3FFF) | ((u64)((lbo >> 4) & 0x3FFF) << 16) | ((u64)((sbo >> 4) & 0x3FFF) << 32) |
         (1ULL << 46);  // descriptor version 1; base offset 0; no swizzle
}

// Two bytes of w (selected by sel) as exact fp16 integers: PRMT builds the
// half-words 0x64bb = 1024 + b, HSUB2 removes the 1024.
__device__ __forceinline__ u32 bytes_to_half2(u32 w, u32 sel) {
  const u32 h = __byte_perm(w, 0x64646464u, sel);
  __half2 v = *reinterpret_cast<const __half2 *>(&h);
  v = __hsub2(v, __half2half2(__ushort_as_half((unsigned short)0x6400)));
  return *reinterpret_cast<const u32 *>(&v);
}

// Integer value of an exact fp32 accumulator below 2^23.
__device__ __forceinline__ u32 acc_int(u32 bits) {
  return __float_as_uint(__uint_as_float(bits) + 8388608.0f) & 0x7FFFFFu;
}

__device__ __forceinline__ u64 mad_wide(u32 x, u32 y, u64 z) {
  u64 d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(x), "r"(y), "l"(z));
  return d;
}

// s * w mod 2^64 for a 32-bit s
__device__ __forceinline__ u64 mul_lo_32x64(u32 s, u64 w) {
  return mad_wide(s, (u32)w, (u64)(s * (u32)(w >> 32)) << 32);
}

// Per-target constants of the recombination.
struct TcTarget {
  u64 q, one_s;    // t, floor(2^64 / t)
  u64 r64, r64_s;  // 2^64 mod t and its Shoup companion
  u32 m80;         // floor(2^80 / t) when t > 2^48 (the quotient estimate of recombine_wide)
  u64 sub;         // subtracted from the result mod t when TcArgs::has_sub
  int wide;        // t > 2^48: the low half L < 2^47.01 is already reduced
};

// y_t = sum_b 2^(8b) v_b mod t from the 8 fp32 accumulators of one target.
__device__ __forceinline__ u64 recombine(const u32 *v, const TcTarget &tg) {
  const u32 c0 = acc_int(v[0]), c1 = acc_int(v[1]), c2 = acc_int(v[2]), c3 = acc_int(v[3]);
  const u32 c4 = acc_int(v[4]), c5 = acc_int(v[5]), c6 = acc_int(v[6]), c7 = acc_int(v[7]);
  // bytes 0..3 and 4..7: L, H < 2^47.01
  const u64 L = mad_wide(c3, 1u << 24, mad_wide(c2, 1u << 16, (u64)(c0 + (c1 << 8))));
  const u64 H = mad_wide(c7, 1u << 24, mad_wide(c6, 1u << 16, (u64)(c4 + (c5 << 8))));
  // y = L + H 2^32 = y_hi 2^64 + y_lo with y_hi < 2^16
  const u64 y_lo = L + (H << 32);
  const u32 y_hi = (u32)(H >> 32) + (y_lo < L ? 1u : 0u);
  // y_lo mod t in [0, 2t): quotient estimate floor(y_lo floor(2^64/t) / 2^64)
  const u64 r_lo = y_lo - __umul64hi(tg.one_s, y_lo) * tg.q;
  // y_hi (2^64 mod t) mod t in [0, 2t): Shoup with a 16-bit multiplicand
  const u64 qt = mad_wide(y_hi, (u32)(tg.r64_s >> 32), (u64)__umulhi(y_hi, (u32)tg.r64_s)) >> 32;
  const u64 r_hi = mul_lo_32x64(y_hi, tg.r64) - mul_lo_32x64((u32)qt, tg.q);
  return csub(csub(r_lo + r_hi, tg.q << 1), tg.q);
}

// The same for t > 2^48: y = L + H 2^32 < 2^80 has a quotient below 2^32.  With
// H' = floor(H / 2^16), y lies in [H' 2^48, H' 2^48 + 2^49); with m = floor(2^80 / t)
// < 2^32, k = floor(H' m / 2^32) satisfies floor(y / t) - 3 <= k <= y / t (the
// dropped parts are below 2^49 / t < 2 and H' / 2^32 < 1).  So y - k t lies in
// [0, 4t) and is formed exactly from the low words: one 32-bit high multiply and
// a 32 x 64 product.
__device__ __forceinline__ u64 recombine_wide(const u32 *v, const TcTarget &tg) {
  const u32 c0 = acc_int(v[0]), c1 = acc_int(v[1]), c2 = acc_int(v[2]), c3 = acc_int(v[3]);
  const u32 c4 = acc_int(v[4]), c5 = acc_int(v[5]), c6 = acc_int(v[6]), c7 = acc_int(v[7]);
  const u64 L = mad_wide(c3, 1u << 24, mad_wide(c2, 1u << 16, (u64)(c0 + (c1 << 8))));
  const u64 H = mad_wide(c7, 1u << 24, mad_wide(c6, 1u << 16, (u64)(c4 + (c5 << 8))));
  const u32 k = __umulhi((u32)(H >> 16), tg.m80);
  const u64 r = L + (H << 32) - (u64)k * tg.q;  // [0, 4t)
  return csub(csub(r, tg.q << 1), tg.q);
}

// ALL_WIDE: every target of the launch is above 2^48 (checked on the host), so
// only the one-product path is compiled in.
// The launch's options (TcArgs::has_add, has_sub, has_v) at compile time: FL = 0
// none, 7 all three (the merged ModDown-rescale), -1 read at run time.
template <int FL>
__device__ __forceinline__ bool tc_flag(int runtime, int bit) {
  return FL < 0 ? runtime != 0 : ((FL >> bit) & 1) != 0;
}

template <bool ALL_WIDE = false>
__device__ __forceinline__ u64 recombine_target(const u32 *v, const TcTarget &tg, bool has_sub) {
  u64 r = (ALL_WIDE || tg.wide) ? recombine_wide(v, tg) : recombine(v, tg);
  if (has_sub) r = submod(r, tg.sub, tg.q);
  return r;
}

// Two adjacent targets' 16 accumulators of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(u32 (&v)[16], u32 addr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
}
__device__ __forceinline__ void tmem_ld8(u32 *v, u32 addr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(addr));
}

constexpr int TC_SRC_GROUPS = TC_THREADS / TC_M;        // threads sharing one A row
constexpr int TC_SRC_PER = TC_MAX_S / TC_SRC_GROUPS;    // sources per thread at most

struct TcArgs {
  u32 n;
  int ns, nt, kpad, npad;
  const __half *bmat;                         // [npad][kpad] row-major constants (bytes)
  u64 sq[TC_MAX_S], inv[TC_MAX_S], inv_s[TC_MAX_S];  // b_i, [Bhat_i^-1]_(b_i), Shoup companion
  u64 src_add[TC_MAX_S];                      // added to y_i mod b_i when has_add
  u64 rdiv[TC_MAX_S], rdiv_hi[TC_MAX_S];      // floor(2^96 / b_i), low and high words, when has_v
  int has_add, has_sub;
  int has_v;                                  // overflow removal: A column 8 ns holds v, B row holds -B mod t
  TcTarget tg[TC_MAX_T];
  unsigned char dst_pos[TC_MAX_T];
  const u64 *src[MAX_CTS];
  u64 *dst[MAX_CTS];
  int np;
  int *err;                                   // set to 1 (or 2) when a bounded wait expires
  u64 wait_ns;                                // the bound of every wait for an MMA group
  // test only: before any MMA is issued, every CTA waits (bounded by wait_ns)
  // on barrier 0, which nothing arrives on, so the wait expires with no MMA
  // outstanding and the failure path runs
  int test_expire;
};

// Sources of one 128-coefficient block for this thread: row tid mod 128,
// sources i = tid / 128 + 4 k.
// tiles_per_poly is a power of two (n / 128): tpp_log2 its log
__device__ __forceinline__ void load_sources(const TcArgs &a, int tile, int tpp_log2, int tid,
                                             u64 (&x)[TC_SRC_PER]) {
  const u64 *src = a.src[tile >> tpp_log2];
  const u32 kc = (u32)(tile & ((1 << tpp_log2) - 1)) * TC_M + (u32)(tid & (TC_M - 1));
#pragma unroll
  for (int k = 0; k < TC_SRC_PER; ++k) {
    const int i = tid / TC_M + k * TC_SRC_GROUPS;
    if (i < a.ns) x[k] = __ldg(src + (size_t)i * a.n + kc);
  }
}

// y_i = [x_i Bhat_i^-1]_(b_i) as 8 fp16 bytes into row tid mod 128 of an A tile;
// with overflow removal, this thread's part of sum_i floor(y_i R_i / 2^64)
// goes to part[group][row].
template <int FL>
__device__ __forceinline__ void store_sources(const TcArgs &a, unsigned char *sA, int tid,
                                              const u64 (&x)[TC_SRC_PER], u64 *part) {
  const int row = tid & (TC_M - 1);
  u64 fix = 0;
#pragma unroll
  for (int k = 0; k < TC_SRC_PER; ++k) {
    const int i = tid / TC_M + k * TC_SRC_GROUPS;
    if (i < a.ns) {
      u64 y = shoup(x[k], a.inv[i], a.inv_s[i], a.sq[i]);
      if (tc_flag<FL>(a.has_add, 0)) y = addmod(y, a.src_add[i], a.sq[i]);
      if (tc_flag<FL>(a.has_v, 2)) fix += __umul64hi(y, a.rdiv[i]) + y * a.rdiv_hi[i];  // high word: b_i < 2^32 only
      const u32 lo = (u32)y, hi = (u32)(y >> 32);
      uint4 v;
      v.x = bytes_to_half2(lo, 0x4140);
      v.y = bytes_to_half2(lo, 0x4342);
      v.z = bytes_to_half2(hi, 0x4140);
      v.w = bytes_to_half2(hi, 0x4342);
      *reinterpret_cast<uint4 *>(sA + canon_offset(row, i * 8, a.kpad)) = v;
    }
  }
  if (tc_flag<FL>(a.has_v, 2)) part[(tid / TC_M) * TC_M + row] = fix;
}

// v = floor(sum of the four parts / 2^32) into column 8 ns of row tid (tid < 128).
__device__ __forceinline__ void store_overflow(const TcArgs &a, unsigned char *sA, int tid, const u64 *part) {
  const u64 f = part[tid] + part[TC_M + tid] + part[2 * TC_M + tid] + part[3 * TC_M + tid];
  *reinterpret_cast<__half *>(sA + canon_offset(tid, 8 * a.ns, a.kpad)) = __uint2half_rn((unsigned)(f >> 32));
}

template <bool ALL_WIDE, int FL>
__global__ void __launch_bounds__(TC_THREADS, 1) k_bconv_tc(const TcArgs a) {
  const bool has_v = tc_flag<FL>(a.has_v, 2), has_sub = tc_flag<FL>(a.has_sub, 1);
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a_bytes = TC_M * a.kpad * 2;
  unsigned char *sB = smem + 2 * a_bytes;  // A tiles 0 and 1 precede it
  u64 *mbar = reinterpret_cast<u64 *>(sB + a.npad * a.kpad * 2);  // two barriers
  u32 *tmem_slot = reinterpret_cast<u32 *>(mbar + 2);
  u64 *part = mbar + 4;  // [4][128] overflow parts (after the barriers and the TMEM slot)

  // constants into the canonical layout; zero padding columns of both A tiles
  for (int idx = tid; idx < a.npad * a.kpad; idx += TC_THREADS) {
    const int r = idx / a.kpad, k = idx % a.kpad;
    *reinterpret_cast<__half *>(sB + canon_offset(r, k, a.kpad)) = a.bmat[idx];
  }
  for (int idx = tid; idx < 2 * TC_M * (a.kpad / 8 - a.ns); idx += TC_THREADS) {
    const int b = idx / (TC_M * (a.kpad / 8 - a.ns)), rem = idx % (TC_M * (a.kpad / 8 - a.ns));
    const int r = rem % TC_M, i = a.ns + rem / TC_M;
    *reinterpret_cast<uint4 *>(smem + b * a_bytes + canon_offset(r, i * 8, a.kpad)) = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }

  const int tpp_log2 = 31 - __clz((int)(a.n / TC_M));  // n / 128 is a power of two
  const int total = (1 << tpp_log2) * a.np;
  const int grid = (int)gridDim.x;
  int tile = blockIdx.x;
  u64 x[TC_SRC_PER];  // sources of the next block to be written into an A tile
  if (tile < total) {
    load_sources(a, tile, tpp_log2, tid, x);
    store_sources<FL>(a, smem, tid, x, part);
  }
  if (tile + grid < total) load_sources(a, tile + grid, tpp_log2, tid, x);
  if (has_v && tile < total) {
    __syncthreads();
    if (tid < TC_M) store_overflow(a, smem, tid, part);
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const u32 tmem = *tmem_slot;

  // instruction descriptor: D fp32, A and B fp16, both K-major, M = 128, N = npad
  const u32 idesc = (1u << 4) | ((u32)(a.npad >> 3) << 17) | ((u32)(TC_M >> 4) << 24);
  const u32 sB_addr = smem_u32(sB);
  const u32 sbo = (u32)(a.kpad / 8) * 128;
  u32 phase = 0;    // bit b: parity of the next completion of mbar[b]
  u32 pending = 0;  // bit b: an MMA group committed to mbar[b] and not yet waited for

  auto issue = [&](int b) {
    if (tid == 0) {
      const u32 sa = smem_u32(smem + b * a_bytes);
      for (int kk = 0; kk < a.kpad / 16; ++kk) {
        const u64 ad = make_desc(sa + kk * 256, 128, sbo);
        const u64 bd = make_desc(sB_addr + kk * 256, 128, sbo);
        const u32 acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (u32)(b * TC_ACC_COLS)),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar + b)));
    }
    pending |= 1u << b;
  };

  bool failed = false;
  if (a.test_expire) {  // nothing arrives on barrier 0: the wait runs out
    wait_parity(smem_u32(mbar), 0u, a.wait_ns);
    failed = true;
  }
  if (!failed && tile < total) issue(0);
  const int lq = warp & 3, cg = warp >> 2;
  const int per_group = (a.nt + TC_COL_GROUPS - 1) / TC_COL_GROUPS;
  const int t_lo = cg * per_group, t_hi = min(a.nt, t_lo + per_group);
  for (int j = 0; !failed && tile < total; ++j, tile += grid) {
    const int cur = j & 1, nxt = cur ^ 1;
    const int next = tile + grid;
    // A tile of the next block from the prefetched sources (its buffer's MMAs
    // completed before epilogue j - 1), then prefetch the block after it
    if (next < total) store_sources<FL>(a, smem + nxt * a_bytes, tid, x, part);
    if (next + grid < total) load_sources(a, next + grid, tpp_log2, tid, x);
    if (has_v && next < total) {  // the parts are complete after this barrier
      __syncthreads();
      if (tid < TC_M) store_overflow(a, smem + nxt * a_bytes, tid, part);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (next < total) issue(nxt);
    // bounded wait for the MMAs of this block; the outcome is agreed by the whole CTA
    const u32 done = wait_parity(smem_u32(mbar + cur), (phase >> cur) & 1u, a.wait_ns);
    if (__syncthreads_or(done == 0)) {
      failed = true;
      break;
    }
    phase ^= 1u << cur;
    pending &= ~(1u << cur);
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: lanes 32 lq .. +31 = coefficients k0 + 32 lq + lane, targets t_lo .. t_hi - 1
    u64 *dst = a.dst[tile >> tpp_log2];
    const u32 kc = (u32)(tile & ((1 << tpp_log2) - 1)) * TC_M + (u32)(lq * 32 + lane);
    const u32 tbase = tmem + ((u32)(lq * 32) << 16) + (u32)(cur * TC_ACC_COLS);
    // four targets per wait where possible, then a pair, then a single one
    int t = t_lo;
    for (; t + 4 <= t_hi; t += 4) {
      u32 v[16], u[16];
      tmem_ld16(v, tbase + (u32)(t * 8));
      tmem_ld16(u, tbase + (u32)((t + 2) * 8));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      dst[(size_t)a.dst_pos[t] * a.n + kc] = recombine_target<ALL_WIDE>(v, a.tg[t], has_sub);
      dst[(size_t)a.dst_pos[t + 1] * a.n + kc] = recombine_target<ALL_WIDE>(v + 8, a.tg[t + 1], has_sub);
      dst[(size_t)a.dst_pos[t + 2] * a.n + kc] = recombine_target<ALL_WIDE>(u, a.tg[t + 2], has_sub);
      dst[(size_t)a.dst_pos[t + 3] * a.n + kc] = recombine_target<ALL_WIDE>(u + 8, a.tg[t + 3], has_sub);
    }
    if (t + 2 <= t_hi) {
      u32 v[16];
      tmem_ld16(v, tbase + (u32)(t * 8));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      dst[(size_t)a.dst_pos[t] * a.n + kc] = recombine_target<ALL_WIDE>(v, a.tg[t], has_sub);
      dst[(size_t)a.dst_pos[t + 1] * a.n + kc] = recombine_target<ALL_WIDE>(v + 8, a.tg[t + 1], has_sub);
      t += 2;
    }
    if (t < t_hi) {
      u32 v[8];
      tmem_ld8(v, tbase + (u32)(t * 8));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      dst[(size_t)a.dst_pos[t] * a.n + kc] = recombine_target<ALL_WIDE>(v, a.tg[t], has_sub);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  if (failed) {
    // give the MMAs in flight one more (longer) bounded wait, then record the
    // error: 1 when none is outstanding any more, 2 when some still are (the
    // TMEM is freed all the same: a CTA that exits holding it would stall the
    // next allocation on its SM without bound)
    u32 drained = 1;
    for (int b = 0; b < 2; ++b)
      if ((pending >> b) & 1u) drained &= wait_parity(smem_u32(mbar + b), (phase >> b) & 1u, TC_DRAIN_NS);
    const int stuck = __syncthreads_or(drained == 0);
    if (tid == 0) atomicMax(a.err, stuck ? 2 : 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}


// ---------------------------------------------------------------- key inner product as a GEMM
// The key-switch inner product out_o = sum_j d_j key_(j,o) mod q (o = 0, 1;
// reading C7) for P = 128 ciphertexts sharing one key: at one coefficient k
// of limb t it is a [P x ndig] x [ndig x 2] product whose right operand (the
// key words) is shared by the 128 rows.  Byte-split as the conversion above:
//   A[p][(j, a)]     = byte a of d_j[p]                       (K = 8 ndig <= 32)
//   B[(o, b)][(j, a)] = byte b of 2^(8a) key_(j,o) mod q       (N = 16)
//   out_o[p] = sum_b 2^(8b) D[p][(o, b)] mod q, every D entry below 32 255^2 < 2^23.
// One M = 128, N = 16 MMA (K in steps of 16) per coefficient; a unit is 8
// consecutive coefficients of one limb, built into one of two shared-memory
// buffers while the other's MMAs run; 8 x 16 TMEM columns per buffer.
// Layouts: digits [P][ndig][L][N], keys [ndig][2][L][N] (plain residues),
// out [P][2][L][N]; limb t is taken mod the context's modulus t.
constexpr int IP_P = 128;         // ciphertexts (MMA rows)
constexpr int IP_G = 8;           // coefficients per unit
constexpr int IP_MAX_L = 40;
constexpr int IP_TMEM_COLS = 2 * IP_G * 16;

struct IpTcArgs {
  u32 n;
  int L, ndig, kpad, upl_log2;    // units per limb = n / IP_G = 2^upl_log2
  const u64 *d, *key;
  u64 *out;
  const ModInfo *mods;
  u64 pw[IP_MAX_L][8];            // 2^(8a) mod q_t
  TcTarget tg[IP_MAX_L];
  int *err;
  u64 wait_ns;
};

__device__ __forceinline__ int ip_a_item(int kpad) { return IP_P * kpad * 2; }
__device__ __forceinline__ int ip_b_item(int kpad) { return 16 * kpad * 2; }
__device__ __forceinline__ int ip_buf(int kpad) { return IP_G * (ip_a_item(kpad) + ip_b_item(kpad)); }

// A and B tiles of one unit (limb t, coefficients k0 .. k0 + 7) into buffer sbuf.
__device__ __forceinline__ void ip_build(const IpTcArgs &a, unsigned char *sbuf, int unit, int tid) {
  const int t = unit >> a.upl_log2;
  const u32 k0 = (u32)(unit & ((1 << a.upl_log2) - 1)) * IP_G;
  const int a_item = ip_a_item(a.kpad), b_item = ip_b_item(a.kpad);
  unsigned char *sB = sbuf + IP_G * a_item;
  const size_t limb = (size_t)a.L * a.n;
  for (int idx = tid; idx < IP_P * IP_G; idx += TC_THREADS) {  // (ciphertext, coefficient)
    const int p = idx / IP_G, kk = idx % IP_G;
    const u64 *dp = a.d + (size_t)p * a.ndig * limb + (size_t)t * a.n + k0 + kk;
    for (int j = 0; j < a.ndig; ++j) {
      const u64 y = __ldg(dp + (size_t)j * limb);
      const u32 lo = (u32)y, hi = (u32)(y >> 32);
      uint4 v;
      v.x = bytes_to_half2(lo, 0x4140);
      v.y = bytes_to_half2(lo, 0x4342);
      v.z = bytes_to_half2(hi, 0x4140);
      v.w = bytes_to_half2(hi, 0x4342);
      *reinterpret_cast<uint4 *>(sbuf + kk * a_item + canon_offset(p, j * 8, a.kpad)) = v;
    }
  }
  const ModInfo m = a.mods[t];
  for (int idx = tid; idx < IP_G * 2 * a.ndig * 8; idx += TC_THREADS) {  // (coefficient, output, digit, a)
    const int a8 = idx & 7;
    int r = idx >> 3;
    const int j = r % a.ndig;
    r /= a.ndig;
    const int o = r & 1, kk = r >> 1;
    const u64 w = __ldg(a.key + ((size_t)(j * 2 + o) * a.L + t) * a.n + k0 + kk);
    const u64 c = mulmod(w, a.pw[t][a8], m);
    unsigned char *b0 = sB + kk * b_item;
#pragma unroll
    for (int b = 0; b < 8; ++b)
      *reinterpret_cast<__half *>(b0 + canon_offset(o * 8 + b, j * 8 + a8, a.kpad)) =
          __uint2half_rn((unsigned)((c >> (8 * b)) & 255u));
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_inner_tc(const IpTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a_item = ip_a_item(a.kpad), b_item = ip_b_item(a.kpad), buf_bytes = ip_buf(a.kpad);
  u64 *mbar = reinterpret_cast<u64 *>(smem + 2 * buf_bytes);
  u32 *tmem_slot = reinterpret_cast<u32 *>(mbar + 2);
  // zero the padding columns 8 ndig .. kpad - 1 of every tile of both buffers
  const int padc = a.kpad / 8 - a.ndig;
  for (int idx = tid; idx < 2 * IP_G * (IP_P + 16) * padc; idx += TC_THREADS) {
    int r = idx;
    const int cblk = a.ndig + r % padc;
    r /= padc;
    const int row = r % (IP_P + 16);
    r /= IP_P + 16;
    const int kk = r % IP_G, b = r / IP_G;
    unsigned char *base = smem + b * buf_bytes;
    unsigned char *tile = row < IP_P ? base + kk * a_item : base + IP_G * a_item + kk * b_item;
    const int rr = row < IP_P ? row : row - IP_P;
    *reinterpret_cast<uint4 *>(tile + canon_offset(rr, cblk * 8, a.kpad)) = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(IP_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const int total = a.L << a.upl_log2;
  const int grid = (int)gridDim.x;
  int unit = blockIdx.x;
  if (unit < total) ip_build(a, smem, unit, tid);
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const u32 tmem = *tmem_slot;
  // D fp32, A and B fp16, K-major, M = 128, N = 16
  const u32 idesc = (1u << 4) | ((u32)(16 >> 3) << 17) | ((u32)(IP_P >> 4) << 24);
  const u32 sbo = (u32)(a.kpad / 8) * 128;
  u32 phase = 0, pending = 0;
  auto issue = [&](int b) {
    if (tid == 0) {
      const u32 base = smem_u32(smem + b * buf_bytes);
      for (int kk = 0; kk < IP_G; ++kk) {
        const u32 sa = base + kk * a_item, sb = base + IP_G * a_item + kk * b_item;
        for (int ks = 0; ks < a.kpad / 16; ++ks) {
          const u64 ad = make_desc(sa + ks * 256, 128, sbo);
          const u64 bd = make_desc(sb + ks * 256, 128, sbo);
          const u32 acc = ks > 0 ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                  tmem + (u32)((b * IP_G + kk) * 16)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar + b)));
    }
    pending |= 1u << b;
  };
  bool failed = false;
  if (unit < total) issue(0);
  const int lq = warp & 3, cg = warp >> 2;
  const size_t limb = (size_t)a.L * a.n;
  for (int j = 0; unit < total; ++j, unit += grid) {
    const int cur = j & 1, nxt = cur ^ 1;
    const int next = unit + grid;
    if (next < total) ip_build(a, smem + nxt * buf_bytes, next, tid);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (next < total) issue(nxt);
    const u32 done = wait_parity(smem_u32(mbar + cur), (phase >> cur) & 1u, a.wait_ns);
    if (__syncthreads_or(done == 0)) {
      failed = true;
      break;
    }
    phase ^= 1u << cur;
    pending &= ~(1u << cur);
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: lanes 32 lq .. +31 = ciphertexts, coefficients cg and cg + 4 of the unit
    const int t = unit >> a.upl_log2;
    const u32 k0 = (u32)(unit & ((1 << a.upl_log2) - 1)) * IP_G;
    const int p = lq * 32 + lane;
    u64 *o0 = a.out + (size_t)(2 * p) * limb + (size_t)t * a.n + k0;
    const u32 tbase = tmem + ((u32)(lq * 32) << 16) + (u32)(cur * IP_G * 16);
    u32 v[16], u[16];
    tmem_ld16(v, tbase + (u32)(cg * 16));
    tmem_ld16(u, tbase + (u32)((cg + 4) * 16));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    o0[cg] = recombine_target(v, a.tg[t], 0);
    o0[limb + cg] = recombine_target(v + 8, a.tg[t], 0);
    o0[cg + 4] = recombine_target(u, a.tg[t], 0);
    o0[limb + cg + 4] = recombine_target(u + 8, a.tg[t], 0);
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  if (failed) {
    u32 drained = 1;
    for (int b = 0; b < 2; ++b)
      if ((pending >> b) & 1u) drained &= wait_parity(smem_u32(mbar + b), (phase >> b) & 1u, TC_DRAIN_NS);
    const int stuck = __syncthreads_or(drained == 0);
    if (tid == 0) atomicMax(a.err, stuck ? 2 : 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(IP_TMEM_COLS));
}

// The same product on the CUDA cores, for comparison: one thread per
// coefficient of one limb, the key words in registers, the ciphertexts in a
// loop; 128-bit sums, one reduction per output.
template <int NDIG>
__global__ void __launch_bounds__(256) k_inner_flat(const u64 *__restrict__ d, const u64 *__restrict__ key,
                                                   u64 *__restrict__ out, const ModInfo *mods, u32 n, int L,
                                                   int np) {
  const u32 k = blockIdx.x * 256 + threadIdx.x;
  const int t = blockIdx.y;
  if (k >= n) return;
  const ModInfo m = mods[t];
  const size_t limb = (size_t)L * n, off = (size_t)t * n + k;
  u64 kb[NDIG], ka[NDIG];
#pragma unroll
  for (int j = 0; j < NDIG; ++j) {
    kb[j] = __ldg(key + (size_t)(2 * j) * limb + off);
    ka[j] = __ldg(key + (size_t)(2 * j + 1) * limb + off);
  }
#pragma unroll 4
  for (int p = 0; p < np; ++p) {
    u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll
    for (int j = 0; j < NDIG; ++j) {
      const u64 v = __ldg(d + ((size_t)p * NDIG + j) * limb + off);
      mac128(h0, l0, v, kb[j]);
      mac128(h1, l1, v, ka[j]);
    }
    out[(size_t)(2 * p) * limb + off] = reduce128(h0, l0, m);
    out[(size_t)(2 * p + 1) * limb + off] = reduce128(h1, l1, m);
  }
}

}  // namespace

// Host: the byte-plane constant matrix of one conversion, cached on the device
// (built on first use, outside any graph capture), then the launch.
// key identifies the conversion (table offset); tab_host rows are [nt][ns].
static int launch_bconv_tc_ex(ckks_ctx *c, size_t key, const u64 *inv_host, const u64 *tab_host, int ns, int nt,
                              const int *src_mod, const int *dst_mod, const int *dst_pos, const u64 *const *src,
                              u64 *const *dst, int np, const u64 *src_add_host, const u64 *dst_sub_host,
                              const u64 *rdiv_host, const u64 *negs_host, u64 wait_ns, int test_expire,
                              u32 n_virt) {
  if (ns < 1 || ns > TC_MAX_S || nt < 1 || nt > TC_MAX_T || np < 1 || np > MAX_CTS) return CKKS_E_PARAM;
  if (n_virt % TC_M || n_virt == 0 || ((n_virt / TC_M) & (n_virt / TC_M - 1))) return CKKS_E_PARAM;
  const bool has_v = rdiv_host && negs_host;
  if (has_v && ns == TC_MAX_S) return CKKS_E_PARAM;  // the overflow column needs K <= 8 ns + 1 <= 128
  const int kpad = ((8 * ns + (has_v ? 1 : 0) + 15) / 16) * 16, npad = ((8 * nt + 15) / 16) * 16;
  if (!c->tc_err) {
    if (c->capturing) return CKKS_E_STATE;
    if (cudaMalloc(&c->tc_err, sizeof(int)) != cudaSuccess) return CKKS_E_OOM;
    CK_CUDA(cudaMemset(c->tc_err, 0, sizeof(int)));
  }
  auto it = c->tc_bmats.find(key);
  if (it == c->tc_bmats.end()) {
    if (c->capturing) return CKKS_E_STATE;
    // B[(t,b)][(i,a)] = byte b of (2^(8a) * c_(i,t) mod t)
    std::vector<__half> bm((size_t)npad * kpad, __float2half(0.f));
    for (int t = 0; t < nt; ++t) {
      const u64 m = c->mod[dst_mod[t]];
      for (int i = 0; i < ns; ++i) {
        const u64 cc = tab_host[(size_t)t * ns + i] % m;
        for (int aa = 0; aa < 8; ++aa) {
          const u64 cf = host_mulmod(cc, host_powmod(2, 8 * aa, m), m);
          for (int b = 0; b < 8; ++b)
            bm[(size_t)(t * 8 + b) * kpad + i * 8 + aa] = __float2half((float)((cf >> (8 * b)) & 0xFF));
        }
      }
      if (has_v)  // column 8 ns: the bytes of -S mod t, times v in A
        for (int b = 0; b < 8; ++b)
          bm[(size_t)(t * 8 + b) * kpad + 8 * ns] = __float2half((float)((negs_host[t] % m >> (8 * b)) & 0xFF));
    }
    void *d = nullptr;
    if (cudaMalloc(&d, bm.size() * sizeof(__half)) != cudaSuccess) return CKKS_E_OOM;
    CK_CUDA(cudaMemcpy(d, bm.data(), bm.size() * sizeof(__half), cudaMemcpyHostToDevice));
    it = c->tc_bmats.emplace(key, d).first;
  }
  TcArgs a;
  a.n = n_virt;
  a.ns = ns;
  a.nt = nt;
  a.kpad = kpad;
  a.npad = npad;
  a.bmat = reinterpret_cast<const __half *>(it->second);
  a.has_add = src_add_host != nullptr;
  a.has_sub = dst_sub_host != nullptr;
  a.has_v = has_v ? 1 : 0;
  for (int i = 0; i < ns; ++i) {
    a.sq[i] = c->mod[src_mod[i]];
    a.inv[i] = inv_host[2 * i];
    a.inv_s[i] = inv_host[2 * i + 1];
    a.src_add[i] = src_add_host ? src_add_host[i] : 0;
    a.rdiv[i] = has_v ? rdiv_host[i] : 0;
    a.rdiv_hi[i] = has_v ? rdiv_host[ns + i] : 0;
  }
  const unsigned __int128 two64 = (unsigned __int128)1 << 64;
  for (int t = 0; t < nt; ++t) {
    const u64 m = c->mod[dst_mod[t]];
    TcTarget &g = a.tg[t];
    g.q = m;
    g.one_s = (u64)(two64 / m);
    g.r64 = (u64)(two64 % m);
    g.r64_s = (u64)(((unsigned __int128)g.r64 << 64) / m);
    g.wide = m > (1ULL << 48) ? 1 : 0;
    g.m80 = g.wide ? (u32)(((unsigned __int128)1 << 80) / m) : 0;  // < 2^32 since t > 2^48
    g.sub = dst_sub_host ? dst_sub_host[t] : 0;
    a.dst_pos[t] = (unsigned char)dst_pos[t];
  }
  for (int i = 0; i < np; ++i) {
    a.src[i] = src[i];
    a.dst[i] = dst[i];
  }
  a.np = np;
  a.err = c->tc_err;
  a.wait_ns = wait_ns;
  a.test_expire = test_expire;
  // more than half of the SM's shared memory per CTA: one CTA per SM, so its
  // 512-column TMEM allocation never waits for another CTA's
  const size_t need = 2 * (size_t)TC_M * kpad * 2 + (size_t)npad * kpad * 2 + 32 + 4 * TC_M * 8;
  const size_t smem = std::max<size_t>(need, 120 * 1024);
  bool all_wide = true;
  for (int t = 0; t < nt; ++t) all_wide = all_wide && a.tg[t].wide;
  const int flags = a.has_add | a.has_sub << 1 | a.has_v << 2;
  auto kern = flags == 0   ? (all_wide ? k_bconv_tc<true, 0> : k_bconv_tc<false, 0>)
              : flags == 7 ? (all_wide ? k_bconv_tc<true, 7> : k_bconv_tc<false, 7>)
                           : (all_wide ? k_bconv_tc<true, -1> : k_bconv_tc<false, -1>);
  CK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int total = (int)(n_virt / TC_M) * np;
  const int grid = std::min(total, sms);
  PROF_LAUNCH(c, PK_BCONV_TC, (u64)np * nt * ns, (kern<<<grid, TC_THREADS, smem, c->stream>>>(a)));
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

int launch_bconv_tc(ckks_ctx *c, size_t key, const u64 *inv_host, const u64 *tab_host, int ns, int nt,
                    const int *src_mod, const int *dst_mod, const int *dst_pos, const u64 *const *src,
                    u64 *const *dst, int np, const u64 *src_add_host, const u64 *dst_sub_host,
                    const u64 *rdiv_host, const u64 *negs_host) {
  return launch_bconv_tc_ex(c, key, inv_host, tab_host, ns, nt, src_mod, dst_mod, dst_pos, src, dst, np,
                            src_add_host, dst_sub_host, rdiv_host, negs_host, TC_WAIT_NS, 0, c->n);
}

// TEST ONLY (ckks_debug_tc_expire): one launch of the conversion kernel on a
// one-source, one-target conversion of a scratch polynomial, whose CTAs wait
// on a barrier that nothing arrives on before issuing any MMA.  The wait runs
// out after wait_ns (clamped to 1 ms .. 1 s), the failure path records flag 1
// and frees the TMEM; the scratch target holds garbage afterwards.
extern "C" int ckks_debug_tc_expire(ckks_ctx *c, uint64_t wait_ns) {
  if (!c) return CKKS_E_PARAM;
  if (c->capturing) return CKKS_E_STATE;
  wait_ns = std::min<u64>(std::max<u64>(wait_ns, 1000000ULL), TC_WAIT_NS);
  int rc = ensure_scratch(c, 2 * (size_t)c->n);
  if (rc) return rc;
  const u64 inv[2] = {1, host_shoup(1, c->mod[0])}, tab[1] = {1};
  const int sm[1] = {0}, dm[1] = {1 % (c->n_q + c->n_p)}, dp[1] = {0};
  CK_CUDA(cudaMemsetAsync(c->scratch, 0, 2 * (size_t)c->n * sizeof(u64), c->stream));
  const u64 *src[1] = {c->scratch};
  u64 *dst[1] = {c->scratch + c->n};
  return launch_bconv_tc_ex(c, ~(size_t)0, inv, tab, 1, 1, sm, dm, dp, src, dst, 1, nullptr, nullptr, nullptr,
                            nullptr, wait_ns, 1, c->n);
}

// The same exact byte-split product on a strided view: `n_virt` coefficients
// per source and per target, source i at src + i n_virt (the tensor-core NTT
// stage prototype views a limb's 16-row blocks as 16 sources).
int launch_bconv_tc_view(ckks_ctx *c, size_t key, const u64 *inv_host, const u64 *tab_host, int ns, int nt,
                         const int *src_mod, const int *dst_mod, const int *dst_pos, const u64 *const *src,
                         u64 *const *dst, int np, u32 n_virt) {
  return launch_bconv_tc_ex(c, key, inv_host, tab_host, ns, nt, src_mod, dst_mod, dst_pos, src, dst, np, nullptr,
                            nullptr, nullptr, nullptr, TC_WAIT_NS, 0, n_virt);
}

// ---- key inner product prototype entry points ----
static int check_inner_args(const ckks_ctx *c, const uint64_t *d, const uint64_t *key, uint32_t n_cts,
                            uint32_t n_digits, uint32_t n_limbs, const uint64_t *out) {
  if (!c || !d || !key || !out) return CKKS_E_PARAM;
  if (n_digits < 1 || n_digits > 4 || n_limbs < 1 || n_limbs > (uint32_t)std::min(IP_MAX_L, c->n_q + c->n_p))
    return CKKS_E_PARAM;
  if (n_cts < 1) return CKKS_E_PARAM;
  if (c->capturing) return CKKS_E_STATE;
  return CKKS_OK;
}

extern "C" int ckks_ks_inner_tc(ckks_ctx *c, const uint64_t *d, const uint64_t *key, uint32_t n_cts,
                                uint32_t n_digits, uint32_t n_limbs, uint64_t *out) {
  int rc = check_inner_args(c, d, key, n_cts, n_digits, n_limbs, out);
  if (rc) return rc;
  if (n_cts != IP_P) return CKKS_E_PARAM;
  if ((((uintptr_t)d) | ((uintptr_t)key) | ((uintptr_t)out)) & 15) return CKKS_E_PARAM;
  IpTcArgs a;
  a.n = c->n;
  a.L = (int)n_limbs;
  a.ndig = (int)n_digits;
  a.kpad = (8 * (int)n_digits + 15) / 16 * 16;
  a.upl_log2 = c->log_n - 3;  // n / IP_G units per limb
  a.d = d;
  a.key = key;
  a.out = out;
  a.mods = c->d_mods;
  const unsigned __int128 two64 = (unsigned __int128)1 << 64;
  for (int t = 0; t < a.L; ++t) {
    const u64 m = c->mod[t];
    u64 w = 1 % m;
    for (int k = 0; k < 8; ++k) {
      a.pw[t][k] = w;
      w = (u64)(((unsigned __int128)w << 8) % m);
    }
    TcTarget &g = a.tg[t];
    g.q = m;
    g.one_s = (u64)(two64 / m);
    g.r64 = (u64)(two64 % m);
    g.r64_s = (u64)(((unsigned __int128)g.r64 << 64) / m);
    g.wide = m > (1ULL << 48) ? 1 : 0;
    g.m80 = g.wide ? (u32)(((unsigned __int128)1 << 80) / m) : 0;
    g.sub = 0;
  }
  a.err = c->tc_err;
  a.wait_ns = TC_WAIT_NS;
  const size_t smem = 2 * (size_t)IP_G * (IP_P * a.kpad * 2 + 16 * a.kpad * 2) + 32;
  CK_CUDA(cudaFuncSetAttribute(k_inner_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int total = a.L << a.upl_log2;
  const int grid = std::min(total, sms);
  PROF_LAUNCH(c, PK_INNER_TC, (u64)n_cts * n_limbs, (k_inner_tc<<<grid, TC_THREADS, smem, c->stream>>>(a)));
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

extern "C" int ckks_ks_inner_u64(ckks_ctx *c, const uint64_t *d, const uint64_t *key, uint32_t n_cts,
                                 uint32_t n_digits, uint32_t n_limbs, uint64_t *out) {
  int rc = check_inner_args(c, d, key, n_cts, n_digits, n_limbs, out);
  if (rc) return rc;
  dim3 g((c->n + 255) / 256, n_limbs);
  const int np = (int)n_cts, L = (int)n_limbs;
  switch (n_digits) {
#define FCASE(D)                                                                                             \
  case D:                                                                                                    \
    PROF_LAUNCH(c, PK_INNER_FLAT, (u64)n_cts * n_limbs,                                                      \
                (k_inner_flat<D><<<g, 256, 0, c->stream>>>(d, key, out, c->d_mods, c->n, L, np)));          \
    break;
    FCASE(1) FCASE(2) FCASE(3) FCASE(4)
#undef FCASE
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}
