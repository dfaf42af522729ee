// Full-slot CKKS bootstrapping on the GPU.
//
// ReBoot refreshes weights and velocities with CKKS bootstrapping (Sec. 3,
// last paragraph; Alg. 1, the two Bootstrap lines) and defers its construction
// to Cheon et al. 2018, Bossuat et al. 2021 and Bae et al. 2022; the paper fixes
// the structure (ModRaise, homomorphic encoding, scaled sine, decoding) and the
// level budget tau_bs = 16 (Sec. 5.1, Table 3).  The readings B1..B8 of the
// design notes make every step definite:
//   B1 ModRaise: centred lift of c0, c1 mod q0 into every limb; scale := q0.
//   B2 slots z = U (p_lo + i p_hi), U = S_n ... S_2 P (radix-2 DIT stages on
//      bit-reversed input, twiddle exp(2 pi i (5^j mod 4 len) / (4 len)));
//      CoeffToSlot applies P U^-1, SlotToCoeff U P^-1.
//   B3 three merged levels per transform, each with diagonals at offsets
//      k * step, evaluated by baby-step giant-step with hoisted baby rotations
//      and constants encoded at the scale of the prime the level drops.
//   B4 1/(2K) folded into the first CoeffToSlot level, 1/(2 pi) into the first
//      SlotToCoeff level.
//   B5 u_re = u + conj(u), u_im = -i (u - conj(u)); v = v_re + i v_im.
//   B6 EvalMod = degree-60 Chebyshev interpolant of cos(2 pi (K u - 1/4)/8)
//      on [-1, 1], then three double angles.
//   B7 Chebyshev basis and recursive split with exact scale targeting
//      (constants chosen so every sum meets at one scale; a higher operand is
//      brought down with an integer multiply and a rescale).
//   B8 output scale = (scale after SlotToCoeff) * Delta_in / q0.
// FP64 runs on the GPU for the constants: the stage products of the DFT
// factors (diagonal form), their pre-rotation, their canonical-embedding
// encoding, and the Chebyshev coefficients.
#include <algorithm>
#include <cmath>
#include <set>
#include <vector>

#include "ops.cuh"

namespace {

constexpr int TPB = 256;
constexpr int K_RANGE = 16;
constexpr int CHEB_DEGREE = 60;
constexpr int DOUBLE_ANGLES = 3;
constexpr int LEVELS_CTS = 3;
constexpr int LEVELS_STC = 3;
constexpr int EVALMOD_DEPTH = 7 + DOUBLE_ANGLES;
constexpr int BOOT_DEPTH = LEVELS_CTS + EVALMOD_DEPTH + LEVELS_STC;  // 16
constexpr int MAXB = 16;   // ciphertexts per fused launch
constexpr int MAXA = 32;   // baby steps (2^(w-1) at a level of w <= 6 stages: N <= 2^17)
constexpr int MAXT = 8;    // terms of an integer linear combination

// [k]_q of a signed integer (host)
static u64 host_sres(i64 k, u64 q) {
  if (k >= 0) return (u64)k % q;
  const u64 mag = ((u64)(-(k + 1)) + 1) % q;
  return mag ? q - mag : 0;
}

struct Giant {
  int b;
  std::vector<std::pair<int, int>> items;  // (a, k) ascending a
};

struct LinLevel {
  int s0 = 0, s1 = 0, w = 0, step = 1, g = 1, level = 0;
  bool inverse = false, wrap = false;
  int span = 0, W = 0, nd = 0;  // offsets mod n/step; window half-width; stored diagonals
  std::vector<Giant> plan;
  int first_const = 0, n_const = 0;
  int diag_index(int k) const { return wrap ? ((k % span) + span) % span : k + W; }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ u32 pow5_mod(u32 j, u32 m) {  // m a power of two
  u64 r = 1, b = 5;
  while (j) {
    if (j & 1) r = (r * b) & (m - 1);
    b = (b * b) & (m - 1);
    j >>= 1;
  }
  return (u32)r;
}

// Entry of butterfly stage S_(2 lenh) (or its inverse) in row rr at offset
// e in {0, +lenh, -lenh} (e_kind 0, 1, 2).
__device__ double2 stage_entry(u32 rr, int e_kind, u32 lenh, int inverse) {
  const u32 pos = rr % (2 * lenh);
  const bool upper = pos < lenh;
  const u32 j = upper ? pos : pos - lenh;
  double s, c;
  sincospi((double)pow5_mod(j, 8 * lenh) / (double)(4 * lenh), &s, &c);  // xi = exp(2 pi i e / 8 lenh)
  const double2 xi = make_double2(c, s);
  const double2 ixi = make_double2(c, -s);  // 1 / xi
  if (!inverse) {
    if (e_kind == 0) return upper ? make_double2(1.0, 0.0) : make_double2(-xi.x, -xi.y);
    if (e_kind == 1) return upper ? xi : make_double2(0.0, 0.0);
    return upper ? make_double2(0.0, 0.0) : make_double2(1.0, 0.0);
  }
  if (e_kind == 0) return upper ? make_double2(0.5, 0.0) : make_double2(-0.5 * ixi.x, -0.5 * ixi.y);
  if (e_kind == 1) return upper ? make_double2(0.5, 0.0) : make_double2(0.0, 0.0);
  return upper ? make_double2(0.0, 0.0) : make_double2(0.5 * ixi.x, 0.5 * ixi.y);
}

struct DiagShape {
  u32 n;
  int step, wrap, span, W, nd;
};
__device__ __forceinline__ int dindex(const DiagShape &s, int k) {
  return s.wrap ? ((k % s.span) + s.span) % s.span : k + s.W;
}

__global__ void k_diag_identity(double2 *D, DiagShape s) {
  const u32 r = blockIdx.x * TPB + threadIdx.x;
  const int idx = blockIdx.y;
  if (r >= s.n) return;
  D[(size_t)idx * s.n + r] = make_double2(idx == dindex(s, 0) ? 1.0 : 0.0, 0.0);
}

// C = M S for stage S_(2 lenh): C_k[r] = sum_e M_(k-e)[r] S_e[r + (k-e) step]
__global__ void k_diag_stage(const double2 *M, double2 *C, DiagShape s, u32 lenh, int inverse) {
  const u32 r = blockIdx.x * TPB + threadIdx.x;
  const int idx = blockIdx.y;
  if (r >= s.n) return;
  const int kout = s.wrap ? idx : idx - s.W;
  const int h = (int)(lenh / s.step);
  double2 sum = make_double2(0.0, 0.0);
  for (int ek = 0; ek < 3; ++ek) {
    const int e = ek == 0 ? 0 : (ek == 1 ? h : -h);
    const int kin = kout - e;
    if (!s.wrap && (kin < -s.W || kin > s.W)) continue;
    const double2 m = M[(size_t)dindex(s, kin) * s.n + r];
    if (m.x == 0.0 && m.y == 0.0) continue;
    const long long off = (long long)kin * s.step;
    const u32 rr = (u32)((((long long)r + off) % (long long)s.n + s.n) % s.n);
    const double2 v = cmul(m, stage_entry(rr, ek, lenh, inverse));
    sum.x += v.x;
    sum.y += v.y;
  }
  C[(size_t)idx * s.n + r] = sum;
}

// vec[r] = factor * D_k[(r - shift) mod n]
__global__ void k_diag_gather(const double2 *D, double2 *vec, DiagShape s, int idx, int shift, double factor) {
  const u32 r = blockIdx.x * TPB + threadIdx.x;
  if (r >= s.n) return;
  const u32 src = (u32)((((long long)r - shift) % (long long)s.n + s.n) % s.n);
  const double2 v = D[(size_t)idx * s.n + src];
  vec[r] = make_double2(v.x * factor, v.y * factor);
}

// B13: a diagonal of n_slots entries repeated across the N/2 slots
__global__ void k_tile_slots(double2 *vec, int n_slots, int half_n) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n_slots && i < half_n) vec[i] = vec[i % n_slots];
}

// c_k = 2/(d+1) sum_j f(x_j) cos(k pi (j + 1/2)/(d+1)), c_0 halved;
// f(x) = cos(2 pi (K x - 1/4) / 2^r)
__global__ void k_cheb(double *c, int d, double kr, int r) {
  const int k = threadIdx.x;
  if (k > d) return;
  double acc = 0.0;
  for (int j = 0; j <= d; ++j) {
    const double th = ((double)j + 0.5) / (double)(d + 1);  // theta / pi
    const double x = cospi(th);
    const double f = cospi(2.0 * (kr * x - 0.25) / (double)(1 << r));
    acc += f * cospi((double)k * th);
  }
  acc *= 2.0 / (double)(d + 1);
  c[k] = k == 0 ? acc / 2 : acc;
}

// ---------------------------------------------------------------- batched kernels
// ---- double-hoisted linear levels (B11) ----
constexpr int MAXG = 4;  // giant steps of a double-hoisted level
constexpr int MB_K = 128;          // coefficients per CTA of k_mac_ext
constexpr int MB_THREADS = 512;    // 4 groups of MB_K threads, each a share of the ciphertexts
constexpr int MB_GROUPS = MB_THREADS / MB_K;
struct MacExtArgs {
  const ModInfo *mods;
  u32 n;
  int ext, na, ng, nq, cn, npt;    // nq = l + 1 q-limbs; npt plaintexts of the level
  unsigned char mod_of[MAX_MODS];
  const u64 *pt[MAXG * MAXA];      // the level's plaintexts over Q_l P, slot s
  signed char slot[MAXG][MAXA];    // [giant][baby] -> slot, or -1 (no diagonal)
  const u64 *xq;                   // babies a >= 1: [ct][baby][2][ext][N] (slot 0 unused)
  size_t x_ct, x_baby;
  const u64 *c0[MAXB], *c1[MAXB];  // baby 0 = P x, formed on the fly from x over q_0..q_l
  u64 pm[CKKS_MAX_Q], pm_s[CKKS_MAX_Q];
  u64 *out;                        // giant terms: [ct][giant][2][ext][N]
  size_t o_ct, o_giant;
};
// inner_j = sum_a pt[j][a] x_a over Q_l P for every giant j of the level;
// x_0 = (P c0, P c1) on q-limbs and 0 on the special limbs.
// Grid (coefficient blocks of MB_K, extended limbs).  The CTA first stages
// the block's words of every plaintext of the level in shared memory (npt x
// MB_K words, 16-byte loads); its four thread groups then walk their shares
// of the ciphertexts, each thread streaming its coefficient of every baby once
// and keeping all giants' 128-bit sums.  Every byte of babies, plaintexts and
// outputs crosses HBM once.
__global__ void __launch_bounds__(MB_THREADS, 2) k_mac_ext(const MacExtArgs a) {
  extern __shared__ u64 spt[];     // [npt][MB_K]
  const int t = blockIdx.y;
  const u32 k0 = blockIdx.x * MB_K;
  for (int i = threadIdx.x; i < a.npt * (MB_K / 2); i += MB_THREADS) {
    const int s = i / (MB_K / 2), w = i % (MB_K / 2);
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(a.pt[s] + (size_t)t * a.n + k0) + w);
    spt[s * MB_K + 2 * w] = v.x;
    spt[s * MB_K + 2 * w + 1] = v.y;
  }
  __syncthreads();
  const int kk = threadIdx.x % MB_K, grp = threadIdx.x / MB_K;
  const ModInfo m = a.mods[a.mod_of[t]];
  const size_t poly = (size_t)a.ext * a.n, off = (size_t)t * a.n + k0 + kk;
  for (int c = grp; c < a.cn; c += MB_GROUPS) {
    u64 h[MAXG][2], lo[MAXG][2];
#pragma unroll
    for (int j = 0; j < MAXG; ++j) h[j][0] = h[j][1] = lo[j][0] = lo[j][1] = 0;
    if (t < a.nq) {  // baby 0: P x on the q-limbs, nothing on the special limbs
      const u64 x0 = shoup(__ldg(a.c0[c] + off), a.pm[t], a.pm_s[t], m.q);
      const u64 x1 = shoup(__ldg(a.c1[c] + off), a.pm[t], a.pm_s[t], m.q);
#pragma unroll
      for (int j = 0; j < MAXG; ++j) {
        const int s = j < a.ng ? a.slot[j][0] : -1;
        if (s < 0) continue;
        const u64 p = spt[s * MB_K + kk];
        mac128(h[j][0], lo[j][0], x0, p);
        mac128(h[j][1], lo[j][1], x1, p);
      }
    }
    const u64 *xb = a.xq + c * a.x_ct + off;
#pragma unroll 4
    for (int b = 1; b < a.na; ++b) {
      const u64 x0 = __ldg(xb + b * a.x_baby), x1 = __ldg(xb + b * a.x_baby + poly);
#pragma unroll
      for (int j = 0; j < MAXG; ++j) {
        const int s = j < a.ng ? a.slot[j][b] : -1;
        if (s < 0) continue;
        const u64 p = spt[s * MB_K + kk];
        mac128(h[j][0], lo[j][0], x0, p);
        mac128(h[j][1], lo[j][1], x1, p);
      }
    }
#pragma unroll
    for (int j = 0; j < MAXG; ++j) {
      if (j >= a.ng) continue;
      u64 *o = a.out + c * a.o_ct + j * a.o_giant + off;
      o[0] = reduce128(h[j][0], lo[j][0], m);
      o[poly] = reduce128(h[j][1], lo[j][1], m);
    }
  }
}

struct CombArgs {
  const ModInfo *mods;
  u32 n;
  int nt;
  u64 kr[MAXT][CKKS_MAX_Q];        // [k_i]_{q_t}, reduced on the host
  const u64 *x0[MAXB][MAXT], *x1[MAXB][MAXT];
  u64 *o0[MAXB], *o1[MAXB];
};
// o = sum_i k_i x_i
__global__ void k_lincomb(const CombArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[t];
  const size_t off = (size_t)t * a.n + k;
  u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll 4
  for (int i = 0; i < a.nt; ++i) {
    const u64 kk = a.kr[i][t];
    mac128(h0, l0, __ldg(a.x0[c][i] + off), kk);
    mac128(h1, l1, __ldg(a.x1[c][i] + off), kk);
  }
  a.o0[c][off] = reduce128(h0, l0, m);
  a.o1[c][off] = reduce128(h1, l1, m);
}

// The same, two coefficients per thread in 16-byte words (every pointer
// 16-byte aligned): twice the bytes in flight per load instruction.
__global__ void k_lincomb2(const CombArgs a) {
  const u32 k2 = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, c = blockIdx.z;
  if (2 * k2 >= a.n) return;
  const ModInfo m = a.mods[t];
  const size_t off = ((size_t)t * a.n) / 2 + k2;  // in 16-byte words
  u64 h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
#pragma unroll 4
  for (int i = 0; i < a.nt; ++i) {
    const u64 kk = a.kr[i][t];
    const ulonglong2 x0 = __ldg(reinterpret_cast<const ulonglong2 *>(a.x0[c][i]) + off);
    const ulonglong2 x1 = __ldg(reinterpret_cast<const ulonglong2 *>(a.x1[c][i]) + off);
    mac128(h[0], l[0], x0.x, kk);
    mac128(h[1], l[1], x0.y, kk);
    mac128(h[2], l[2], x1.x, kk);
    mac128(h[3], l[3], x1.y, kk);
  }
  reinterpret_cast<ulonglong2 *>(a.o0[c])[off] = make_ulonglong2(reduce128(h[0], l[0], m), reduce128(h[1], l[1], m));
  reinterpret_cast<ulonglong2 *>(a.o1[c])[off] = make_ulonglong2(reduce128(h[2], l[2], m), reduce128(h[3], l[3], m));
}

struct ConstArgs {
  const ModInfo *mods;
  u32 n;
  u64 kr[CKKS_MAX_Q];               // [k]_{q_t}, reduced on the host
  const u64 *x0[MAXB], *x1[MAXB];
  u64 *o0[MAXB], *o1[MAXB];
};
// o = x + k (the constant polynomial k added to c0; NTT of a constant is constant)
__global__ void k_add_const(const ConstArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[t];
  const size_t off = (size_t)t * a.n + k;
  a.o0[c][off] = addmod(a.x0[c][off], a.kr[t], m.q);
  a.o1[c][off] = a.x1[c][off];
}

struct RaiseArgs {
  const ModInfo *mods;
  u32 n;
  const u64 *coef[MAXB];   // [2][N] coefficient-domain limb 0
  u64 *o0[MAXB], *o1[MAXB];
};
// B1: every limb t receives [c]_centred(q0) mod q_t (coefficient domain)
__global__ void k_mod_raise(const RaiseArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const u64 q0 = a.mods[0].q;
  const ModInfo m = a.mods[t];
  for (int p = 0; p < 2; ++p) {
    const u64 v = a.coef[c][(size_t)p * a.n + k];
    u64 r;
    if (v > (q0 >> 1)) {
      const u64 mag = reduce128(0, q0 - v, m);
      r = mag ? m.q - mag : 0;
    } else {
      r = reduce128(0, v, m);
    }
    (p == 0 ? a.o0[c] : a.o1[c])[(size_t)t * a.n + k] = r;
  }
}

int ilog2(u32 x) {
  int r = 0;
  while ((1u << r) < x) ++r;
  return r;
}

void make_levels(int n_slots, bool inverse, std::vector<LinLevel> &out) {
  const int ls = ilog2((u32)n_slots);
  const int base = ls / 3, extra = ls % 3;
  std::vector<std::pair<int, int>> gr;
  int s = 0;
  for (int i = 0; i < 3; ++i) {
    const int w = base + (i < extra ? 1 : 0);
    gr.push_back({s, s + w});
    s += w;
  }
  if (inverse) std::reverse(gr.begin(), gr.end());  // CoeffToSlot applies the top group first
  out.clear();
  for (auto &pr : gr) {
    LinLevel L;
    L.s0 = pr.first;
    L.s1 = pr.second;
    L.w = L.s1 - L.s0;
    L.step = 1 << L.s0;
    L.g = 1 << std::max(L.w - 1, 0);  // B11: 2^(w-1) baby steps (16 x 4 giant steps at w = 5)
    L.inverse = inverse;
    L.span = n_slots / L.step;
    L.W = (1 << L.w) - 1;
    L.wrap = 2 * L.W + 1 > L.span;
    L.nd = L.wrap ? L.span : 2 * L.W + 1;
    std::set<int> ks;
    for (int k = -L.W; k <= L.W; ++k) {
      const int kk = ((k % L.span) + L.span) % L.span;
      ks.insert(kk <= L.span / 2 ? kk : kk - L.span);
    }
    std::vector<Giant> plan;
    for (int k : ks) {  // ascending
      const int b = (int)std::floor((double)k / L.g), a = k - b * L.g;
      if (plan.empty() || plan.back().b != b) plan.push_back({b, {}});
      plan.back().items.push_back({a, k});
    }
    for (auto &gi : plan) std::sort(gi.items.begin(), gi.items.end());
    L.plan = plan;
    out.push_back(L);
  }
}

}  // namespace

struct BootState {
  bool planned = false, have_consts = false;
  int top = 0, n_slots = 0, n_consts = 0;
  std::vector<LinLevel> cts, stc;
  std::vector<double> cheb;
  std::vector<u64 *> pts;   // NTT-domain plaintexts, plan order
  u64 *mono_p = nullptr, *mono_m = nullptr;
  std::vector<u64 *> chunks, free_slots;
  size_t slot_words = 0;
  u64 *acc_qp = nullptr;    // giant-step sums over Q_l P, [nct][2][l+1+K][N]
  size_t acc_qp_words = 0;
  u64 *baby_qp = nullptr;   // baby rotations over Q_l P, [nct][g][2][l+1+K][N]
  size_t baby_qp_words = 0;
  u64 *inner_qp = nullptr;  // giant terms over Q_l P, [nct][giants][2][l+1+K][N]
  size_t inner_qp_words = 0;
};

void boot_free(ckks_ctx *c) {
  BootState *b = c->boot;
  if (!b) return;
  for (u64 *p : b->pts) cudaFree(p);
  cudaFree(b->mono_p);
  cudaFree(b->mono_m);
  for (u64 *p : b->chunks) cudaFree(p);
  cudaFree(b->acc_qp);
  cudaFree(b->baby_qp);
  cudaFree(b->inner_qp);
  delete b;
  c->boot = nullptr;
}

int boot_ensure_plan(ckks_ctx *c) {
  if (c->boot && c->boot->planned) return CKKS_OK;
  if (c->n_q < BOOT_DEPTH + 1) return CKKS_E_PARAM;
  if (!c->boot) c->boot = new BootState();
  BootState &b = *c->boot;
  b.top = c->n_q - 1;
  b.n_slots = (int)(c->boot_slots ? c->boot_slots : c->n / 2);
  make_levels(b.n_slots, true, b.cts);
  make_levels(b.n_slots, false, b.stc);
  int idx = 0;
  for (size_t i = 0; i < b.cts.size(); ++i) {
    b.cts[i].level = b.top - (int)i;
    b.cts[i].first_const = idx;
    for (auto &gi : b.cts[i].plan) idx += (int)gi.items.size();
    b.cts[i].n_const = idx - b.cts[i].first_const;
  }
  for (size_t i = 0; i < b.stc.size(); ++i) {
    b.stc[i].level = b.top - LEVELS_CTS - EVALMOD_DEPTH - (int)i;
    b.stc[i].first_const = idx;
    for (auto &gi : b.stc[i].plan) idx += (int)gi.items.size();
    b.stc[i].n_const = idx - b.stc[i].first_const;
  }
  for (const auto *lvs : {&b.cts, &b.stc})
    for (const LinLevel &lv : *lvs) {
      if (lv.g > MAXA || (int)lv.plan.size() > MAXG) return CKKS_E_PARAM;
      for (auto &gi : lv.plan)
        if ((int)gi.items.size() > MAXA) return CKKS_E_PARAM;
    }
  b.n_consts = idx;
  b.planned = true;
  return CKKS_OK;
}

int boot_rotation_steps(ckks_ctx *c, std::vector<int> &steps) {
  int rc = boot_ensure_plan(c);
  if (rc) return rc;
  const BootState &b = *c->boot;
  std::set<int> rs;
  for (int k = b.n_slots; k < (int)(c->n / 2); k <<= 1) rs.insert(k);  // B13: the sub-sum
  for (const auto *lvs : {&b.cts, &b.stc})
    for (const LinLevel &lv : *lvs)
      for (const Giant &gi : lv.plan) {
        for (auto &it : gi.items)
          if (it.first) rs.insert(((it.first * lv.step) % b.n_slots + b.n_slots) % b.n_slots);
        if (gi.b) rs.insert(((lv.g * gi.b * lv.step) % b.n_slots + b.n_slots) % b.n_slots);
      }
  steps.assign(rs.begin(), rs.end());
  return CKKS_OK;
}

namespace {

// a diagonal plaintext over q_0..q_level and p_0..p_{K-1} (B11)
int alloc_pt(ckks_ctx *c, int level, u64 **out) {
  if (cudaMalloc(out, sizeof(u64) * (size_t)(level + 1 + c->n_p) * c->n) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  return CKKS_OK;
}

int make_monomials(ckks_ctx *c) {
  BootState &b = *c->boot;
  if (b.mono_p) return CKKS_OK;
  int rc = alloc_pt(c, b.top, &b.mono_p);
  if (!rc) rc = alloc_pt(c, b.top, &b.mono_m);
  if (rc) return rc;
  std::vector<i64> m(c->n, 0);
  m[c->n / 2] = 1;
  rc = ckks_pt_from_int(c, m.data(), b.top, b.mono_p);
  if (rc) return rc;
  m[c->n / 2] = -1;
  return ckks_pt_from_int(c, m.data(), b.top, b.mono_m);
}

// diagonals of one merged level (FP64 on the GPU), pre-rotated and encoded
int level_constants(ckks_ctx *c, const LinLevel &lv, double factor, double2 *D0, double2 *D1, double2 *vec,
                    int *flag) {
  BootState &b = *c->boot;
  const u32 n = (u32)b.n_slots;
  DiagShape s{n, lv.step, lv.wrap ? 1 : 0, lv.span, lv.W, lv.nd};
  const dim3 grid((n + TPB - 1) / TPB, lv.nd);
  k_diag_identity<<<grid, TPB, 0, c->stream>>>(D0, s);
  std::vector<u32> lenhs;
  for (int st = lv.s1 - 1; st >= lv.s0; --st) lenhs.push_back(1u << st);  // leftmost factor first
  if (lv.inverse) std::reverse(lenhs.begin(), lenhs.end());
  double2 *M = D0, *C = D1;
  for (u32 lh : lenhs) {
    k_diag_stage<<<grid, TPB, 0, c->stream>>>(M, C, s, lh, lv.inverse ? 1 : 0);
    std::swap(M, C);
  }
  if (cudaGetLastError() != cudaSuccess) return CKKS_E_CUDA;
  int idx = lv.first_const;
  const double scale = (double)c->mod[lv.level];
  for (const Giant &gi : lv.plan)
    for (auto &it : gi.items) {
      k_diag_gather<<<(n + TPB - 1) / TPB, TPB, 0, c->stream>>>(M, vec, s, lv.diag_index(it.second),
                                                                lv.g * gi.b * lv.step, factor);
      if (!b.pts[idx]) {
        int rc = alloc_pt(c, lv.level, &b.pts[idx]);
        if (rc) return rc;
      }
      if (n < c->n / 2)
        k_tile_slots<<<(c->n / 2 + TPB - 1) / TPB, TPB, 0, c->stream>>>(vec, (int)n, (int)(c->n / 2));
      int rc = encode_device_z_ext(c, vec, lv.level, scale, b.pts[idx], flag);
      if (rc) return rc;
      ++idx;
    }
  return CKKS_OK;
}

}  // namespace

// ---------------------------------------------------------------- evaluation
namespace {

struct BV {
  std::vector<ckks_ct> v;
  int level = 0;
  double scale = 1.0;
  bool owned = false;
};

struct Eval {
  ckks_ctx *c;
  BootState &b;
  int nct;
  int err = CKKS_OK;

  Eval(ckks_ctx *cc, int n) : c(cc), b(*cc->boot), nct(n) {}

  u64 *p1(const ckks_ct &ct) const { return ct.data + (size_t)ct.n_limbs * c->n; }

  int grow() {
    const size_t per = b.slot_words;
    const int cnt = std::max(8, 4 * nct);
    u64 *chunk = nullptr;
    if (cudaMalloc(&chunk, sizeof(u64) * per * cnt) != cudaSuccess) {
      cudaGetLastError();
      return CKKS_E_OOM;
    }
    b.chunks.push_back(chunk);
    for (int i = 0; i < cnt; ++i) b.free_slots.push_back(chunk + per * i);
    return CKKS_OK;
  }

  BV fresh(int level, double scale) {
    BV r;
    r.owned = true;
    r.level = level;
    r.scale = scale;
    for (int i = 0; i < nct; ++i) {
      if (b.free_slots.empty() && grow()) {
        err = CKKS_E_OOM;
        break;
      }
      ckks_ct ct;
      ct.data = b.free_slots.back();
      b.free_slots.pop_back();
      ct.log_n = c->log_n;
      ct.n_limbs = b.top + 1;
      ct.level = level;
      ct.is_ntt = 1;
      ct.scale = scale;
      r.v.push_back(ct);
    }
    return r;
  }

  void release(BV &x) {
    if (x.owned)
      for (auto &ct : x.v) b.free_slots.push_back(ct.data);
    x.v.clear();
    x.owned = false;
  }

  static BV view(const BV &x, int level) {
    BV r = x;
    r.owned = false;
    r.level = level;
    for (auto &ct : r.v) ct.level = level;
    return r;
  }

  void sync_fields(BV &x) {
    for (auto &ct : x.v) {
      ct.level = x.level;
      ct.scale = x.scale;
    }
  }

  // ---- primitive batched steps ----
  BV lincomb(const std::vector<const BV *> &xs, const std::vector<i64> &ks, int level) {
    BV o = fresh(level, 1.0);
    if (err) return o;
    for (int c0 = 0; c0 < nct; c0 += MAXB) {
      const int cn = std::min(MAXB, nct - c0);
      for (size_t t0 = 0; t0 < xs.size(); t0 += MAXT) {
        const int tn = (int)std::min<size_t>(MAXT, xs.size() - t0);
        CombArgs a;
        a.mods = c->d_mods;
        a.n = c->n;
        a.nt = tn;
        for (int i = 0; i < tn; ++i)
          for (int l = 0; l <= o.level; ++l) a.kr[i][l] = host_sres(ks[t0 + i], c->mod[l]);
        for (int cc = 0; cc < cn; ++cc) {
          for (int i = 0; i < tn; ++i) {
            a.x0[cc][i] = xs[t0 + i]->v[c0 + cc].data;
            a.x1[cc][i] = p1(xs[t0 + i]->v[c0 + cc]);
          }
          a.o0[cc] = o.v[c0 + cc].data;
          a.o1[cc] = p1(o.v[c0 + cc]);
        }
        if (t0 > 0) {  // chain: add the partial sum as a term with coefficient 1
          // never taken for MAXT >= 8 terms (leaves have at most 7)
          err = CKKS_E_PARAM;
          return o;
        }
        uintptr_t al = 0;
        for (int cc = 0; cc < cn; ++cc) {
          for (int i = 0; i < tn; ++i) al |= (uintptr_t)a.x0[cc][i] | (uintptr_t)a.x1[cc][i];
          al |= (uintptr_t)a.o0[cc] | (uintptr_t)a.o1[cc];
        }
        if (!(al & 15) && !(c->n & 1)) {
          const dim3 g((c->n / 2 + TPB - 1) / TPB, level + 1, cn);
          PROF_LAUNCH(c, PK_BOOT_LINCOMB, (u64)(level + 1) * cn * (2 * tn + 2),
                      (k_lincomb2<<<g, TPB, 0, c->stream>>>(a)));
        } else {
          const dim3 g((c->n + TPB - 1) / TPB, level + 1, cn);
          PROF_LAUNCH(c, PK_BOOT_LINCOMB, (u64)(level + 1) * cn * (2 * tn + 2),
                      (k_lincomb<<<g, TPB, 0, c->stream>>>(a)));
        }
      }
    }
    if (cudaGetLastError() != cudaSuccess) err = CKKS_E_CUDA;
    return o;
  }

  BV addsub(const BV &x, const BV &y, bool sub) {  // same level, scale of x
    BV o = fresh(x.level, x.scale);
    if (err) return o;
    for (int c0 = 0; c0 < nct; c0 += MAX_CTS) {
      const int cn = std::min(MAX_CTS, nct - c0);
      EwArgs e;
      for (int i = 0; i < cn; ++i) {
        e.x0[i] = x.v[c0 + i].data;
        e.x1[i] = p1(x.v[c0 + i]);
        e.y0[i] = y.v[c0 + i].data;
        e.y1[i] = p1(y.v[c0 + i]);
        e.o0[i] = o.v[c0 + i].data;
        e.o1[i] = p1(o.v[c0 + i]);
      }
      int rc = ew_addsub(c, e, x.level + 1, cn, sub);
      if (rc) err = rc;
    }
    return o;
  }

  BV rescale(BV x) {  // in place on an owned value
    sync_fields(x);
    for (int c0 = 0; c0 < nct && !err; c0 += MAX_CTS) {
      int rc = rescale_chunk(c, x.v.data() + c0, std::min(MAX_CTS, nct - c0));
      if (rc) err = rc;
    }
    x.level -= 1;
    x.scale = x.v.empty() ? x.scale / (double)c->mod[x.level + 1] : x.v[0].scale;
    return x;
  }

  BV add_const(const BV &x, double cst) {
    const i64 k = llround(cst * x.scale);
    BV o = fresh(x.level, x.scale);
    if (err) return o;
    for (int c0 = 0; c0 < nct; c0 += MAXB) {
      const int cn = std::min(MAXB, nct - c0);
      ConstArgs a;
      a.mods = c->d_mods;
      a.n = c->n;
      for (int l = 0; l <= x.level; ++l) a.kr[l] = host_sres(k, c->mod[l]);
      for (int i = 0; i < cn; ++i) {
        a.x0[i] = x.v[c0 + i].data;
        a.x1[i] = p1(x.v[c0 + i]);
        a.o0[i] = o.v[c0 + i].data;
        a.o1[i] = p1(o.v[c0 + i]);
      }
      const dim3 g((c->n + TPB - 1) / TPB, x.level + 1, cn);
      PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)(x.level + 1) * cn, (k_add_const<<<g, TPB, 0, c->stream>>>(a)));
    }
    if (cudaGetLastError() != cudaSuccess) err = CKKS_E_CUDA;
    return o;
  }

  BV mul_int(const BV &x, i64 k) {
    BV o = lincomb({&x}, {k}, x.level);
    o.scale = x.scale;
    return o;
  }

  BV times_i(const BV &x, int sign) {
    BV o = fresh(x.level, x.scale);
    if (err) return o;
    const u64 *pt = sign > 0 ? b.mono_p : b.mono_m;
    for (int c0 = 0; c0 < nct; c0 += MAX_CTS) {
      const int cn = std::min(MAX_CTS, nct - c0);
      EwArgs e;
      for (int i = 0; i < cn; ++i) {
        e.x0[i] = x.v[c0 + i].data;
        e.x1[i] = p1(x.v[c0 + i]);
        e.y0[i] = pt;
        e.o0[i] = o.v[c0 + i].data;
        e.o1[i] = p1(o.v[c0 + i]);
      }
      int rc = ew_plain(c, e, x.level + 1, cn, 0);
      if (rc) err = rc;
    }
    return o;
  }

  BV automorph(const BV &x, u64 g) {
    BV o = fresh(x.level, x.scale);
    if (err) return o;
    BV xin = x;
    sync_fields(xin);
    std::vector<u64> gs(nct, g);
    for (int c0 = 0; c0 < nct && !err; c0 += MAX_CTS) {
      int rc = automorph_chunk(c, xin.v.data() + c0, gs.data() + c0, o.v.data() + c0, std::min(MAX_CTS, nct - c0));
      if (rc) err = rc;
    }
    o.level = x.level;
    o.scale = x.scale;
    return o;
  }

  BV mul(const BV &a, const BV &bb) {
    const int lv = std::min(a.level, bb.level);
    BV x = view(a, lv), y = view(bb, lv);
    sync_fields(x);
    sync_fields(y);
    BV o = fresh(lv, a.scale * bb.scale);
    if (err) return o;
    // relinearised product with ModDown and rescale merged (reading C21)
    for (int c0 = 0; c0 < nct && !err; c0 += MAX_CTS) {
      int rc = mul_relin_chunk(c, x.v.data() + c0, y.v.data() + c0, o.v.data() + c0, std::min(MAX_CTS, nct - c0),
                               true);
      if (rc) err = rc;
    }
    o.level = lv - 1;
    o.scale = o.v.empty() ? a.scale * bb.scale / (double)c->mod[lv] : o.v[0].scale;
    return o;
  }

  // bring ct to `level` at exactly `scale` (B7)
  BV align(const BV &ct, int level, double scale) {
    if (ct.level > level) {
      const double ql = (double)c->mod[ct.level];
      const i64 k = llround(scale * ql / ct.scale);
      BV r = lincomb({&ct}, {k}, ct.level);
      r.scale = scale * ql;
      r = rescale(r);
      r.level = level;
      return r;
    }
    return view(ct, level);
  }

  BV add(const BV &a, const BV &bb, bool sub = false) {
    BV x, y;
    double s;
    BV tmp;
    if (a.level > bb.level) {
      tmp = align(a, bb.level, bb.scale);
      x = tmp;
      y = bb;
      s = bb.scale;
    } else if (bb.level > a.level) {
      tmp = align(bb, a.level, a.scale);
      x = a;
      y = tmp;
      s = a.scale;
    } else {
      x = a;
      y = bb;
      s = a.scale;
    }
    BV o = addsub(x, y, sub);
    o.scale = s;
    release(tmp);
    return o;
  }

  // ---- B1 ----
  BV mod_raise(const ckks_ct *in) {
    const u32 n = c->n;
    BV x = fresh(b.top, (double)c->mod[0]);
    if (err) return x;
    int rc = ensure_scratch(c, (size_t)2 * n * nct);
    if (rc) { err = rc; return x; }
    std::vector<const u64 *> src(2 * nct);
    std::vector<u64 *> dst(2 * nct);
    for (int i = 0; i < nct; ++i) {
      src[2 * i] = in[i].data;
      src[2 * i + 1] = in[i].data + (size_t)in[i].n_limbs * n;
      dst[2 * i] = c->scratch + (size_t)2 * n * i;
      dst[2 * i + 1] = dst[2 * i] + n;
    }
    int m0[1] = {0};
    rc = launch_ntt(c, src.data(), dst.data(), 2 * nct, 1, m0, true);
    if (rc) { err = rc; return x; }
    for (int c0 = 0; c0 < nct; c0 += MAXB) {
      const int cn = std::min(MAXB, nct - c0);
      RaiseArgs a;
      a.mods = c->d_mods;
      a.n = n;
      for (int i = 0; i < cn; ++i) {
        a.coef[i] = c->scratch + (size_t)2 * n * (c0 + i);
        a.o0[i] = x.v[c0 + i].data;
        a.o1[i] = p1(x.v[c0 + i]);
      }
      const dim3 g((n + TPB - 1) / TPB, b.top + 1, cn);
      PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)(b.top + 1) * cn, (k_mod_raise<<<g, TPB, 0, c->stream>>>(a)));
    }
    std::vector<const u64 *> ps(2 * nct);
    std::vector<u64 *> pd(2 * nct);
    for (int i = 0; i < nct; ++i) {
      pd[2 * i] = x.v[i].data;
      pd[2 * i + 1] = p1(x.v[i]);
      ps[2 * i] = pd[2 * i];
      ps[2 * i + 1] = pd[2 * i + 1];
    }
    int mods[MAX_MODS];
    for (int t = 0; t <= b.top; ++t) mods[t] = t;
    rc = launch_ntt(c, ps.data(), pd.data(), 2 * nct, b.top + 1, mods, false);
    if (rc) err = rc;
    return x;
  }

  // ---- B3 ----
  // device buffer of at least `words` words, grown outside graph capture
  int grow_buf(u64 *&buf, size_t &have, size_t words) {
    if (have >= words) return CKKS_OK;
    if (c->capturing) return CKKS_E_STATE;
    cudaFree(buf);
    buf = nullptr;
    have = 0;
    if (cudaMalloc(&buf, sizeof(u64) * words) != cudaSuccess) {
      cudaGetLastError();
      return CKKS_E_OOM;
    }
    have = words;
    return CKKS_OK;
  }

  // One merged level, double hoisted (B10, B11): baby rotations over Q_l P
  // (x_0 = P x, x_a = (P sigma_a(c0) + acc0_a, acc1_a), no ModDown), every
  // giant term inner_b = sum_a pt_{b,a} x_a over Q_l P in one pass, inner_0
  // joins the sum X as it is, each other inner_b is ModDown'd (C9) and rotated
  // as in B10 (X += KS_acc(sigma_b(c1)), base0 += sigma_b(c0)); one merged
  // ModDown-rescale (C21) divides X + P base by P q_l.
  BV linear(const BV &xin, const LinLevel &lv) {
    BV x = view(xin, lv.level);
    sync_fields(x);
    const int l = lv.level, nl = l + 1, ext = nl + c->n_p, ng = (int)lv.plan.size();
    const size_t N = c->n, poly = (size_t)ext * N;
    if (ng > MAXG || lv.g > MAXA || nct > MAX_CTS) err = err ? err : CKKS_E_PARAM;
    std::vector<int> rot_as;
    for (const Giant &gi : lv.plan)
      for (auto &it : gi.items)
        if (it.first) rot_as.push_back(it.first);
    std::sort(rot_as.begin(), rot_as.end());
    rot_as.erase(std::unique(rot_as.begin(), rot_as.end()), rot_as.end());
    const int na = lv.g;
    const size_t x_baby = 2 * poly, x_ct = (size_t)na * x_baby, o_giant = 2 * poly, o_ct = (size_t)ng * o_giant;
    if (!err) err = grow_buf(b.baby_qp, b.baby_qp_words, x_ct * nct);
    if (!err) err = grow_buf(b.inner_qp, b.inner_qp_words, o_ct * nct);
    // scratch for every step below, reserved once so that no call reallocates it
    size_t ws = std::max(ks_modup_words(c, l, nct), ks_merged_words(c, l, nct));
    ws = std::max(ws, (size_t)2 * nl * N * nct + ks_modup_words(c, l, nct));
    if (!err) err = ensure_scratch(c, ws);
    BV out = fresh(l - 1, x.scale);
    if (err) return out;
    auto baby = [&](int i, int a) { return b.baby_qp + i * x_ct + a * x_baby; };
    std::vector<const u64 *> x0(nct), x1(nct);
    for (int i = 0; i < nct; ++i) {
      x0[i] = x.v[i].data;
      x1[i] = p1(x.v[i]);
    }
    // baby rotations: one ModUp of c1, one inner product per step with sigma_a,
    // whose output gets P sigma_a(c0) on poly 0's q-limbs (baby 0 = P x is
    // formed inside the MAC)
    if (!rot_as.empty() && !err) {
      std::vector<u64 *> eb(nct);
      err = ks_modup(c, l, nct, x1.data(), c->scratch, eb.data());
      std::vector<const u64 *> ebc(eb.begin(), eb.end());
      for (int a : rot_as) {
        if (err) break;
        const u64 g = ckks_galois_elt(c, a * lv.step);
        const u64 *key = galois_key_data(c, g);
        if (!key) {
          err = CKKS_E_NOKEY;
          break;
        }
        std::vector<const u64 *> keys(nct, key);
        std::vector<u32> gal(nct, (u32)g);
        std::vector<u64 *> acc(nct);
        for (int i = 0; i < nct; ++i) acc[i] = baby(i, a);
        err = ks_accumulate(c, l, nct, x1.data(), ebc.data(), keys.data(), gal.data(), acc.data(), false,
                            x0.data());
      }
    }
    // every giant term in one pass over the babies
    for (int c0 = 0; c0 < nct && !err; c0 += MAXB) {
      const int cn = std::min(MAXB, nct - c0);
      MacExtArgs a;
      a.mods = c->d_mods;
      a.n = c->n;
      a.ext = ext;
      a.na = na;
      a.ng = ng;
      a.nq = nl;
      for (int t = 0; t < ext; ++t) a.mod_of[t] = (unsigned char)c->ext_mod(l, t);
      for (int t = 0; t < nl; ++t) {
        const u64 q = c->mod[t];
        u64 pm = 1;
        for (int k = 0; k < c->n_p; ++k) pm = host_mulmod(pm, c->mod[c->n_q + k] % q, q);
        a.pm[t] = pm;
        a.pm_s[t] = host_shoup(pm, q);
      }
      for (int i = 0; i < cn; ++i) {
        a.c0[i] = x0[c0 + i];
        a.c1[i] = x1[c0 + i];
      }
      for (int j = 0; j < MAXG; ++j)
        for (int t = 0; t < MAXA; ++t) a.slot[j][t] = -1;
      int ci = lv.first_const, npt = 0;
      for (int j = 0; j < ng; ++j)
        for (auto &it : lv.plan[j].items) {
          a.pt[npt] = b.pts[ci++];
          a.slot[j][it.first] = (signed char)npt++;
        }
      a.npt = npt;
      a.cn = cn;
      a.xq = baby(c0, 0);
      a.x_ct = x_ct;
      a.x_baby = x_baby;
      a.out = b.inner_qp + c0 * o_ct;
      a.o_ct = o_ct;
      a.o_giant = o_giant;
      // limbs moved: babies 1.. and outputs per ciphertext, x's q-limbs, the plaintexts once
      const u64 moved = (u64)cn * ext * (2 * (na - 1) + 2 * ng) + (u64)cn * 2 * nl + (u64)npt * ext;
      const size_t smem = (size_t)npt * MB_K * sizeof(u64);
      // the opt-in above 48 KB is a per-device function attribute: set before each launch
      if (cudaFuncSetAttribute(k_mac_ext, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               MAXG * MAXA * MB_K * (int)sizeof(u64)) != cudaSuccess) {
        err = CKKS_E_CUDA;
        break;
      }
      if (c->n % MB_K || npt > MAXG * MAXA) {
        err = CKKS_E_PARAM;
        break;
      }
      const dim3 g(c->n / MB_K, ext);
      // 128-bit multiply-accumulates: two polynomials per (ciphertext, limb,
      // coefficient, diagonal); baby 0 only on the q-limbs
      u64 macs = 0;
      for (int j = 0; j < ng; ++j)
        for (auto &it : lv.plan[j].items) macs += it.first ? (u64)ext : (u64)nl;
      c->prof.count(PK_BOOT_MAC_MACS, macs * 2 * cn * c->n);
      PROF_LAUNCH(c, PK_BOOT_MAC, moved, (k_mac_ext<<<g, MB_THREADS, smem, c->stream>>>(a)));
      if (cudaGetLastError() != cudaSuccess) err = CKKS_E_CUDA;
    }
    auto inner = [&](int i, int j) { return b.inner_qp + i * o_ct + j * o_giant; };
    // X: the b = 0 term itself, or zero
    int j0 = -1;
    for (int j = 0; j < ng; ++j)
      if (lv.plan[j].b == 0) j0 = j;
    std::vector<u64 *> X(nct);
    if (j0 < 0) {
      if (!err) err = grow_buf(b.acc_qp, b.acc_qp_words, 2 * poly * nct);
      for (int i = 0; i < nct && !err; ++i) {
        X[i] = b.acc_qp + 2 * poly * i;
        if (cudaMemsetAsync(X[i], 0, sizeof(u64) * 2 * poly, c->stream)) err = CKKS_E_CUDA;
      }
    } else {
      for (int i = 0; i < nct; ++i) X[i] = inner(i, j0);
    }
    BV base = fresh(l, x.scale);
    for (auto &ct : base.v)
      if (!err && cudaMemsetAsync(ct.data, 0, sizeof(u64) * 2 * (size_t)ct.n_limbs * N, c->stream)) err = CKKS_E_CUDA;
    for (int j = 0; j < ng && !err; ++j) {
      if (j == j0) continue;
      BV cb = fresh(l, x.scale);  // ModDown of the giant term (C9)
      std::vector<u64 *> acc(nct), o0(nct), o1(nct), b0(nct);
      for (int i = 0; i < nct; ++i) {
        acc[i] = inner(i, j);
        o0[i] = cb.v[i].data;
        o1[i] = p1(cb.v[i]);
        b0[i] = base.v[i].data;
      }
      if (!err) err = ks_moddown_finish(c, l, nct, acc.data(), o0.data(), o1.data(), c->scratch);
      sync_fields(cb);
      const int amt = lv.g * lv.plan[j].b * lv.step;
      const u64 gal = ckks_galois_elt(c, (amt % b.n_slots + b.n_slots) % b.n_slots);  // B13: mod the slots
      if (!err) err = rotate_accumulate_chunk(c, cb.v.data(), gal, nct, X.data(), b0.data(), true);
      release(cb);
    }
    std::vector<const u64 *> b0(nct), b1(nct);
    std::vector<u64 *> o0(nct), o1(nct);
    for (int i = 0; i < nct; ++i) {
      b0[i] = base.v[i].data;
      b1[i] = p1(base.v[i]);
      o0[i] = out.v[i].data;
      o1[i] = p1(out.v[i]);
    }
    if (!err) err = ks_merged_finish(c, l, nct, X.data(), b0.data(), b1.data(), o0.data(), o1.data(), c->scratch);
    release(base);
    // the level's plaintexts sit at scale q_l: (x.scale q_l) / q_l, as a rescale would give
    out.scale = x.scale * (double)c->mod[l] / (double)c->mod[l];
    sync_fields(out);
    return out;
  }

  // ---- B7 ----
  std::vector<BV> T;  // index k: T_k (T[1] is a view of the input)

  BV dbl(int k) {
    BV p = mul(T[k], T[k]);
    BV r = mul_int(p, 2);
    release(p);
    BV o = add_const(r, -1.0);
    release(r);
    return o;
  }
  BV combine(int a, int bb) {
    BV p = mul(T[a], T[bb]);
    BV r = mul_int(p, 2);
    release(p);
    BV o = add(r, T[std::abs(a - bb)], true);
    release(r);
    return o;
  }
  void basis(const BV &u) {
    T.assign(33, BV());
    T[1] = view(u, u.level);
    T[2] = dbl(1);
    T[3] = combine(1, 2);
    T[4] = dbl(2);
    T[5] = combine(2, 3);
    T[6] = dbl(3);
    T[7] = combine(3, 4);
    T[8] = dbl(4);
    T[16] = dbl(8);
    T[32] = dbl(16);
  }
  void free_basis() {
    for (auto &t : T) release(t);
    T.clear();
  }

  static int split_point(int deg) { return deg >= 32 ? 32 : (deg >= 16 ? 16 : 8); }
  int poly_level(int deg) {
    if (deg < 8) {
      int lv = 1 << 30;
      for (int k = 1; k <= std::max(deg, 1); ++k) lv = std::min(lv, T[k].level);
      return lv - 1;
    }
    const int g = split_point(deg);
    const int m = std::min(poly_level(deg - g), T[g].level);
    return std::min(m - 1, poly_level(g - 1));
  }

  BV leaf(std::vector<double> cf, double target) {
    int deg = (int)cf.size() - 1;
    if (deg == 0) {
      cf.push_back(0.0);
      deg = 1;
    }
    int lvl = 1 << 30;
    for (int k = 1; k <= deg; ++k) lvl = std::min(lvl, T[k].level);
    const double ql = (double)c->mod[lvl];
    std::vector<BV> tv;
    std::vector<const BV *> ptrs;
    std::vector<i64> ks;
    for (int k = 1; k <= deg; ++k) {
      tv.push_back(view(T[k], lvl));
      ks.push_back(llround(cf[k] * (ql * target / T[k].scale)));
    }
    for (auto &t : tv) ptrs.push_back(&t);
    BV acc = lincomb(ptrs, ks, lvl);
    acc.scale = ql * target;
    acc = rescale(acc);
    BV o = add_const(acc, cf[0]);
    release(acc);
    return o;
  }

  BV poly(const std::vector<double> &cf, double target) {
    const int deg = (int)cf.size() - 1;
    if (deg < 8) return leaf(cf, target);
    const int g = split_point(deg);
    std::vector<double> q(deg - g + 1, 0.0), r(cf.begin(), cf.begin() + g);
    q[0] = cf[g];
    for (int k = g + 1; k <= deg; ++k) {
      q[k - g] = 2 * cf[k];
      r[2 * g - k] -= cf[k];
    }
    const int m = std::min(poly_level(deg - g), T[g].level);
    const double q_scale = target * (double)c->mod[m] / T[g].scale;
    BV pq = poly(q, q_scale);
    BV prod = mul(pq, T[g]);
    release(pq);
    prod.scale = target;
    BV pr = poly(r, target);
    BV o = add(prod, pr);
    release(prod);
    release(pr);
    return o;
  }

  BV evalmod(const BV &u, const std::vector<double> &cheb) {
    basis(u);
    BV v = poly(cheb, u.scale);
    free_basis();
    for (int i = 0; i < DOUBLE_ANGLES; ++i) {
      BV p = mul(v, v);
      release(v);
      BV r = mul_int(p, 2);
      release(p);
      v = add_const(r, -1.0);
      release(r);
    }
    return v;
  }
};

}  // namespace

static int boot_check(ckks_ctx *c, const ckks_ct *in, ckks_ct *out, int n) {
  if (!c || !in || !out || n < 0) return CKKS_E_PARAM;
  if (n == 0) return CKKS_OK;
  if (!c->boot || !c->boot->have_consts) return CKKS_E_STATE;
  const int out_level = c->boot->top - BOOT_DEPTH;
  for (int i = 0; i < n; ++i) {
    if (!in[i].data || in[i].log_n != (u32)c->log_n || in[i].n_limbs < 1 || !out[i].data) return CKKS_E_PARAM;
    if ((int)out[i].n_limbs < out_level + 1) return CKKS_E_LEVEL;
  }
  if (c->relin.data == nullptr || !c->have_secret) return CKKS_E_NOKEY;
  c->boot->slot_words = (size_t)2 * (c->boot->top + 1) * c->n;
  return CKKS_OK;
}

// ModRaise, CoeffToSlot, EvalMod, SlotToCoeff (B1-B8) of ev.nct ciphertexts
// read at level 0; the result sits at the output level with the circuit's
// own scale (the caller applies Delta_in / q_0, B8).
static BV boot_core(Eval &ev, const ckks_ct *in) {
  ckks_ctx *c = ev.c;
  BootState &b = *c->boot;
  BV x = ev.mod_raise(in);
  for (int k = b.n_slots; k < (int)(c->n / 2) && !ev.err; k <<= 1) {  // B13: the trace onto the subring
    BV r = ev.automorph(x, ckks_galois_elt(c, k));
    BV y = ev.addsub(x, r, false);
    ev.release(x);
    ev.release(r);
    x = y;
  }
  for (const LinLevel &lv : b.cts) {
    BV y = ev.linear(x, lv);
    ev.release(x);
    x = y;
  }
  BV xc = ev.automorph(x, 2ULL * c->n - 1);
  BV ure = ev.addsub(x, xc, false);
  BV d = ev.addsub(x, xc, true);
  ev.release(x);
  ev.release(xc);
  BV uim = ev.times_i(d, -1);
  ev.release(d);
  BV vre = ev.evalmod(ure, b.cheb);
  ev.release(ure);
  BV vim = ev.evalmod(uim, b.cheb);
  ev.release(uim);
  BV vi = ev.times_i(vim, 1);
  ev.release(vim);
  BV v = ev.add(vre, vi);
  ev.release(vre);
  ev.release(vi);
  for (const LinLevel &lv : b.stc) {
    BV y = ev.linear(v, lv);
    ev.release(v);
    v = y;
  }
  if (!ev.err && v.level != b.top - BOOT_DEPTH) ev.err = CKKS_E_STATE;
  return v;
}

static int boot_copy_out(Eval &ev, const BV &v, ckks_ct *out, const double *scales) {
  ckks_ctx *c = ev.c;
  for (int i = 0; i < ev.nct; ++i) {
    ckks_ct &o = out[i];
    const size_t w = (size_t)(v.level + 1) * c->n;
    CK_CUDA(cudaMemcpyAsync(o.data, v.v[i].data, w * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK_CUDA(cudaMemcpyAsync(o.data + (size_t)o.n_limbs * c->n, ev.p1(v.v[i]), w * 8, cudaMemcpyDeviceToDevice,
                            c->stream));
    o.level = v.level;
    o.scale = scales[i];
    o.is_ntt = 1;
    o.log_n = c->log_n;
  }
  return CKKS_OK;
}

extern "C" {

int ckks_boot_set_slots(ckks_ctx *c, uint32_t n_slots) {
  if (!c || n_slots < 2 || n_slots > c->n / 2 || (n_slots & (n_slots - 1))) return CKKS_E_PARAM;
  if (c->boot && c->boot->planned && (u32)c->boot->n_slots != n_slots) return CKKS_E_STATE;
  c->boot_slots = n_slots == c->n / 2 ? 0 : n_slots;
  return CKKS_OK;
}

int ckks_boot_setup(ckks_ctx *c) {
  if (!c) return CKKS_E_PARAM;
  int rc = boot_ensure_plan(c);
  if (rc) return rc;
  BootState &b = *c->boot;
  rc = make_monomials(c);
  if (rc) return rc;
  b.pts.resize(b.n_consts, nullptr);
  const u32 n = (u32)b.n_slots;
  int maxnd = 0;
  for (auto *lvs : {&b.cts, &b.stc})
    for (auto &lv : *lvs) maxnd = std::max(maxnd, lv.nd);
  double2 *D0 = nullptr, *D1 = nullptr, *vec = nullptr;
  int *flag = nullptr;
  double *dcheb = nullptr;
  const size_t dbytes = sizeof(double2) * (size_t)maxnd * n;
  if (cudaMalloc(&D0, dbytes) != cudaSuccess || cudaMalloc(&D1, dbytes) != cudaSuccess ||
      cudaMalloc(&vec, sizeof(double2) * (c->n / 2)) != cudaSuccess || cudaMalloc(&flag, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&dcheb, sizeof(double) * (CHEB_DEGREE + 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(D0); cudaFree(D1); cudaFree(vec); cudaFree(flag); cudaFree(dcheb);
    return CKKS_E_OOM;
  }
  cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
  // B4 (and B13: 1/d, d = N / (2 n_slots), for the sub-sum's factor)
  const double d_sub = (double)(c->n / 2) / (double)n;
  for (size_t i = 0; i < b.cts.size() && !rc; ++i)
    rc = level_constants(c, b.cts[i], i == 0 ? 1.0 / (2.0 * K_RANGE * d_sub) : 1.0, D0, D1, vec, flag);
  for (size_t i = 0; i < b.stc.size() && !rc; ++i)
    rc = level_constants(c, b.stc[i], i == 0 ? 1.0 / (2.0 * M_PI) : 1.0, D0, D1, vec, flag);
  if (!rc) {
    k_cheb<<<1, 64, 0, c->stream>>>(dcheb, CHEB_DEGREE, (double)K_RANGE, DOUBLE_ANGLES);
    b.cheb.assign(CHEB_DEGREE + 1, 0.0);
    if (cudaMemcpyAsync(b.cheb.data(), dcheb, sizeof(double) * (CHEB_DEGREE + 1), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
      rc = CKKS_E_CUDA;
  }
  int h_flag = 0;
  if (!rc && cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = CKKS_E_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = CKKS_E_CUDA;
  cudaFree(D0); cudaFree(D1); cudaFree(vec); cudaFree(flag); cudaFree(dcheb);
  if (rc) return rc;
  if (h_flag) return CKKS_E_SCALE;
  b.have_consts = true;
  return CKKS_OK;
}

int ckks_boot_rotation_steps(ckks_ctx *c, int32_t *out, int cap) {
  if (!c) return CKKS_E_PARAM;
  std::vector<int> steps;
  int rc = boot_rotation_steps(c, steps);
  if (rc) return rc;
  for (int i = 0; i < (int)steps.size() && i < cap && out; ++i) out[i] = steps[i];
  return (int)steps.size();
}

int ckks_boot_constant_count(ckks_ctx *c) {
  if (!c) return CKKS_E_PARAM;
  int rc = boot_ensure_plan(c);
  if (rc) return rc;
  return c->boot->n_consts;
}

int ckks_boot_import(ckks_ctx *c, const int64_t *coeffs, int count, const double *cheb, int n_cheb) {
  if (!c || !coeffs || !cheb || n_cheb != CHEB_DEGREE + 1) return CKKS_E_PARAM;
  int rc = boot_ensure_plan(c);
  if (rc) return rc;
  BootState &b = *c->boot;
  if (count != b.n_consts) return CKKS_E_PARAM;
  rc = make_monomials(c);
  if (rc) return rc;
  b.pts.resize(b.n_consts, nullptr);
  for (auto *lvs : {&b.cts, &b.stc})
    for (auto &lv : *lvs)
      for (int i = 0; i < lv.n_const; ++i) {
        const int idx = lv.first_const + i;
        if (!b.pts[idx] && (rc = alloc_pt(c, lv.level, &b.pts[idx]))) return rc;
        rc = pt_from_int_ext(c, coeffs + (size_t)idx * c->n, lv.level, b.pts[idx]);
        if (rc) return rc;
      }
  b.cheb.assign(cheb, cheb + n_cheb);
  b.have_consts = true;
  return CKKS_OK;
}

int ckks_boot_export(ckks_ctx *c, int64_t *coeffs, int count, double *cheb, int n_cheb) {
  if (!c || !c->boot || !c->boot->have_consts) return CKKS_E_STATE;
  BootState &b = *c->boot;
  if ((coeffs && count != b.n_consts) || (cheb && n_cheb != CHEB_DEGREE + 1)) return CKKS_E_PARAM;
  const u32 n = c->n;
  if (coeffs) {
    int rc = ensure_scratch(c, n);
    if (rc) return rc;
    std::vector<u64> host(n);
    const u64 q0 = c->mod[0];
    for (int idx = 0; idx < b.n_consts; ++idx) {
      CK_CUDA(cudaMemcpyAsync(c->scratch, b.pts[idx], sizeof(u64) * n, cudaMemcpyDeviceToDevice, c->stream));
      int m0[1] = {0};
      const u64 *s1[1] = {c->scratch};
      u64 *d1[1] = {c->scratch};
      rc = launch_ntt(c, s1, d1, 1, 1, m0, true);
      if (rc) return rc;
      CK_CUDA(cudaMemcpyAsync(host.data(), c->scratch, sizeof(u64) * n, cudaMemcpyDeviceToHost, c->stream));
      CK_CUDA(cudaStreamSynchronize(c->stream));
      for (u32 k = 0; k < n; ++k)
        coeffs[(size_t)idx * n + k] = host[k] > q0 / 2 ? -(i64)(q0 - host[k]) : (i64)host[k];
    }
  }
  if (cheb) std::copy(b.cheb.begin(), b.cheb.end(), cheb);
  return CKKS_OK;
}

int ckks_bootstrap_batch(ckks_ctx *c, const ckks_ct *in, ckks_ct *out, int n) {
  int rc = boot_check(c, in, out, n);
  if (rc || n == 0) return rc;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    Eval ev(c, cnt);
    BV v = boot_core(ev, in + i0);
    if (ev.err) {
      ev.release(v);
      return ev.err;
    }
    std::vector<double> sc(cnt);
    for (int i = 0; i < cnt; ++i) sc[i] = v.scale * in[i0 + i].scale / (double)c->mod[0];
    rc = boot_copy_out(ev, v, out + i0, sc.data());
    ev.release(v);
    if (rc) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

// Iterative bootstrapping (reading B12): ct1 = Bootstrap(ct); the level-0
// difference align(ct1, 0, Delta) - ct, times 2^k, is bootstrapped again with
// the same scale label (ct2); the result 2^k ct1 - ct2 is read at scale
// 2^k * scale(ct1), which divides the correction by 2^k without a level.
int ckks_bootstrap_iterative_batch(ckks_ctx *c, const ckks_ct *in, ckks_ct *out, int n, int log2_k) {
  if (log2_k < 1 || log2_k > 30) return CKKS_E_PARAM;
  int rc = boot_check(c, in, out, n);
  if (rc || n == 0) return rc;
  const double delta = in[0].scale;
  for (int i = 1; i < n; ++i)
    if (in[i].scale != delta) return CKKS_E_SCALE;
  const i64 two_k = (i64)1 << log2_k;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    Eval ev(c, cnt);
    BV v1 = boot_core(ev, in + i0);
    if (ev.err) {
      ev.release(v1);
      return ev.err;
    }
    v1.scale *= delta / (double)c->mod[0];
    const double out_scale = v1.scale * (double)two_k;
    // the first bootstrap's error, at level 0 and scale Delta, times 2^k
    BV a = ev.align(v1, 0, delta);
    BV x0;
    x0.level = 0;
    x0.scale = delta;
    for (int i = 0; i < cnt; ++i) x0.v.push_back(in[i0 + i]);
    BV d = ev.err ? BV() : ev.addsub(a, x0, true);
    ev.release(a);
    BV d2 = ev.err ? BV() : ev.mul_int(d, two_k);
    ev.release(d);
    if (ev.err) {
      ev.release(d2);
      ev.release(v1);
      return ev.err;
    }
    d2.scale = delta;
    ev.sync_fields(d2);
    BV v2 = boot_core(ev, d2.v.data());
    ev.release(d2);
    if (ev.err) {
      ev.release(v2);
      ev.release(v1);
      return ev.err;
    }
    BV up = ev.mul_int(v1, two_k);
    ev.release(v1);
    BV o = ev.err ? BV() : ev.addsub(up, v2, true);
    ev.release(up);
    ev.release(v2);
    if (ev.err) {
      ev.release(o);
      return ev.err;
    }
    o.scale = out_scale;
    std::vector<double> sc(cnt, o.scale);
    rc = boot_copy_out(ev, o, out + i0, sc.data());
    ev.release(o);
    if (rc) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

int ckks_bootstrap(ckks_ctx *c, const ckks_ct *in, ckks_ct *out) { return ckks_bootstrap_batch(c, in, out, 1); }

// One merged level of the circuit's special DFT (B3, B10, B11) on n
// ciphertexts: plan level `index` (CoeffToSlot levels first, then SlotToCoeff),
// the same launches ckks_bootstrap runs for it.
int ckks_boot_linear(ckks_ctx *c, int index, const ckks_ct *in, ckks_ct *out, int n) {
  if (!c || !in || !out || n < 0) return CKKS_E_PARAM;
  if (!c->boot || !c->boot->have_consts) return CKKS_E_STATE;
  BootState &b = *c->boot;
  const int nlev = (int)(b.cts.size() + b.stc.size());
  if (index < 0 || index >= nlev) return CKKS_E_PARAM;
  if (n == 0) return CKKS_OK;
  const LinLevel &lv = index < (int)b.cts.size() ? b.cts[index] : b.stc[index - b.cts.size()];
  for (int i = 0; i < n; ++i) {
    if (!in[i].data || !out[i].data || in[i].log_n != (u32)c->log_n || out[i].log_n != (u32)c->log_n)
      return CKKS_E_PARAM;
    if ((int)in[i].level < lv.level || in[i].n_limbs < in[i].level + 1 || (int)out[i].n_limbs < lv.level)
      return CKKS_E_LEVEL;
    if (in[i].scale != in[0].scale) return CKKS_E_SCALE;
  }
  if (c->relin.data == nullptr || !c->have_secret) return CKKS_E_NOKEY;
  b.slot_words = (size_t)2 * (b.top + 1) * c->n;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    Eval ev(c, cnt);
    BV x;
    x.level = (int)in[i0].level;
    x.scale = in[i0].scale;
    for (int i = 0; i < cnt; ++i) x.v.push_back(in[i0 + i]);
    for (int i = 0; i < cnt; ++i) x.v[i].level = in[i0].level;
    BV y = ev.linear(x, lv);
    if (ev.err) {
      ev.release(y);
      return ev.err;
    }
    std::vector<double> sc(cnt, y.scale);
    int rc = boot_copy_out(ev, y, out + i0, sc.data());
    ev.release(y);
    if (rc) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

}  // extern "C"
