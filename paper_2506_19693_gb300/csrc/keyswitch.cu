// Hybrid key switching (readings C7-C9): ModUp by fast basis conversion,
// inner product with the switching key, ModDown.
//
// For polynomials d (NTT domain, limbs q_0..q_l) and one key per
// polynomial, computes (u0, u1) with u0 + u1 s ~ d s' and writes
//   o0 = base0 + u0,   o1 = base1 + u1      (base may be null -> 0).
//
// Data flow (all buffers limb-major uint64):
//   ModUp (per input polynomial):
//     dc   = iNTT(d)                                   [l+1][N]
//     for each active digit j (q-limbs [lo, hi) of the top-level digit j):
//       ext_j[t] = NTT(BConv_{D_j -> t}(dc[lo:hi]))  for t outside [lo, hi)   (C8)
//       positions inside [lo, hi) are d itself
//   Tail (per output; several outputs may share one ModUp -- hoisting):
//     acc_c[t] = sum_j sigma_g(ext_j)[t] * key_j,c[t]   (c = 0 for b, 1 for a)
//     acc_c[P] = iNTT(acc_c[P]);  z_c = NTT(BConv_{P -> Q_l}(acc_c[P]))  (C9)
//     o_c      = base_c + (acc_c[Q] - z_c) * P^-1
// sigma_g is the Galois automorphism of the output (g = 1: none), applied in
// the NTT domain as a gather: it maps aligned 32-word blocks onto aligned
// 32-word blocks, so the gathered reads stay coalesced.  base0 may be read
// through sigma_g too (rotations add sigma_g(c0)).
// The key is read once per launch for a batch that shares it: the inner
// product loops over the batch with the key words held in registers.
#include "ops.cuh"

namespace {

constexpr int TPB = 256;
constexpr int MAXS = 16;   // source limbs of one basis conversion
constexpr int MAXD = 8;    // digits


struct BConvArgs {
  const ModInfo *mods;
  u32 n;
  int nt;
  const u64 *inv;                  // [ns] pairs: [Bhat_i^-1]_{b_i}, Shoup
  const u64 *tab;                  // [nt][ns]: Bhat_i mod target
  unsigned char src_mod[MAXS];
  unsigned char dst_mod[MAX_MODS];
  unsigned char dst_pos[MAX_MODS];
  const u64 *src[MAX_CTS];         // first source limb (limbs contiguous)
  u64 *dst[MAX_CTS];               // output polynomial base (limb positions dst_pos)
  const u64 *src_add = nullptr;    // [ns] or null: added to y_i mod b_i
  const u64 *dst_sub = nullptr;    // [nt] or null: subtracted from y_t mod t
  // overflow removal (or null): v = floor(sum_i floor(y_i R_i / 2^64) / 2^32),
  // the overflow sum_i y_i / s_i in 32.32 fixed point; y_t += v negs_t
  const u64 *rdiv = nullptr;       // [2][ns]: R_i = floor(2^96 / b_i), low then high words
  const u64 *negs = nullptr;       // [nt] -B mod t
};

// The conversion constants ([nt][NS] words, at most 40 x 16) are staged in
// shared memory once per CTA, and the targets are taken in pairs, so that two
// independent 128-bit sums (and their constant loads) are in flight per thread.
constexpr int BCONV_MAX_TAB = MAX_MODS * 16;

// MERGED: the merged ModDown-rescale's options (src_add, dst_sub, rdiv and negs
// all given), else none of them: fixed per instantiation, no branch per value.
template <int NS, bool MERGED>
__global__ void __launch_bounds__(TPB) k_bconv(const BConvArgs a) {
  __shared__ u64 stab[BCONV_MAX_TAB];
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int p = blockIdx.y;
  for (int x = threadIdx.x; x < a.nt * NS; x += TPB) stab[x] = __ldg(a.tab + x);
  __syncthreads();
  if (k >= a.n) return;
  const u64 *src = a.src[p];
  u64 y[NS];
  u64 fix = 0;  // overflow estimate in 32.32 fixed point
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const u64 q = a.mods[a.src_mod[i]].q;
    y[i] = shoup(src[(size_t)i * a.n + k], a.inv[2 * i], a.inv[2 * i + 1], q);
    if (MERGED) y[i] = addmod(y[i], __ldg(a.src_add + i), q);
    // y_i R_hi is nonzero only for b_i < 2^32, where y_i < 2^32 keeps it below 2^44
    if (MERGED) fix += __umul64hi(y[i], __ldg(a.rdiv + i)) + y[i] * __ldg(a.rdiv + NS + i);
  }
  const u64 v = fix >> 32;
  u64 *dst = a.dst[p];
  for (int t = 0; t < a.nt; t += 2) {
    const bool two = t + 1 < a.nt;
    const u64 *r0 = stab + t * NS, *r1 = stab + (two ? t + 1 : t) * NS;
    u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      mac128(h0, l0, y[i], r0[i]);
      mac128(h1, l1, y[i], r1[i]);
    }
    if (MERGED) {
      mac128(h0, l0, v, __ldg(a.negs + t));
      if (two) mac128(h1, l1, v, __ldg(a.negs + t + 1));
    }
    const ModInfo m0 = a.mods[a.dst_mod[t]];
    u64 o0 = reduce128(h0, l0, m0);
    if (MERGED) o0 = submod(o0, __ldg(a.dst_sub + t), m0.q);
    dst[(size_t)a.dst_pos[t] * a.n + k] = o0;
    if (two) {
      const ModInfo m1 = a.mods[a.dst_mod[t + 1]];
      u64 o1 = reduce128(h1, l1, m1);
      if (MERGED) o1 = submod(o1, __ldg(a.dst_sub + t + 1), m1.q);
      dst[(size_t)a.dst_pos[t + 1] * a.n + k] = o1;
    }
  }
}

struct IPArgs {
  const ModInfo *mods;
  u32 n;
  int log_n;
  int ext, ndig, key_ext, np;
  unsigned char mod_of[MAX_MODS];
  unsigned char keylimb_of[MAX_MODS];
  int lo[MAXD], hi[MAXD];
  const u64 *d[MAX_CTS];
  const u64 *ext_buf[MAX_CTS];     // [ndig][ext][N]
  const u64 *key[MAX_CTS];         // [n_digits][2][key_ext][N], Montgomery form; compressed (C22):
                                   // KEY_HDR seeds, then the b rows [n_digits][key_ext][N]
  int kc;                          // keys compressed
  u32 gal[MAX_CTS];
  u64 *acc[MAX_CTS];               // [2][ext][N]
  // IP_BASE: poly 0 q-limbs t <= l also get [P]_{q_t} sigma_gal(base0)[t]
  const u64 *base0[MAX_CTS];
  int nq_base;                     // l + 1
  u64 pm_mont[CKKS_MAX_Q];         // [P]_{q_t} 2^64 mod q_t
};

enum IPMode { IP_SET = 0, IP_BASE = 1, IP_ACC = 2 };  // acc = r; acc = r + P base0; acc += r

// Grid: (groups of IP_GROUP outputs, coefficient blocks, extended limbs).
// The group index varies fastest, so the CTAs that read one block of the
// lifted digits (all outputs of a hoisted rotation set, all ciphertexts of a
// relinearisation batch) run back to back and share it through L2.  Within a
// group the thread walks the outputs, reloading key words only when the key
// changes.  The products sum in 128 bits against Montgomery-form keys, and one
// Montgomery reduction per output removes the 2^64.  That reduction needs its
// input below 2^65 q; with T terms (the digits, plus the base term in IP_BASE)
// of reduced factors below q the sum is below T q^2, so T q < 2^65 suffices.
// launch_inner checks T q < 2^65 on the host for every limb's modulus and
// refuses the launch otherwise (T <= 7 for 62-bit primes, T <= 9 below 2^61.8).
// The group size (outputs per thread) is a per-context tunable (ckks_tune).
template <int NDIG, int MODE, bool KC>
__global__ void __launch_bounds__(TPB, NDIG <= 3 ? 4 : 2) k_inner(const IPArgs a, int group) {
  const u32 k = blockIdx.y * TPB + threadIdx.x;
  const int t = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[a.mod_of[t]];
  const int kl = a.keylimb_of[t];
  u64 kb[NDIG], ka[NDIG];
  const u64 *cur = nullptr;
  const int p_end = min(a.np, (int)(blockIdx.x + 1) * group);
  const bool with_base = MODE == IP_BASE && t < a.nq_base;
  const u64 pm = with_base ? a.pm_mont[t] : 0;
  // digits and keys are read-only here: non-coherent loads let the unrolled
  // iterations issue their loads ahead of the previous ciphertexts' stores
#pragma unroll 4
  for (int p = blockIdx.x * group; p < p_end; ++p) {
    if (a.key[p] != cur) {
      cur = a.key[p];
#pragma unroll
      for (int j = 0; j < NDIG; ++j) {
        if (KC) {  // a regenerated from the digit's seed, then put in Montgomery form (C22)
          kb[j] = __ldg(cur + KEY_HDR + ((size_t)j * a.key_ext + kl) * a.n + k);
          ka[j] = shoup(uniform_dev(__ldg(cur + j), (u64)kl * a.n + k, m), m.r64, m.r64_s, m.q);
        } else {
          kb[j] = __ldg(cur + ((size_t)(2 * j) * a.key_ext + kl) * a.n + k);
          ka[j] = __ldg(cur + ((size_t)(2 * j + 1) * a.key_ext + kl) * a.n + k);
        }
      }
    }
    const u32 src = gal_src(k, a.gal[p], a.n, a.log_n);
    u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll
    for (int j = 0; j < NDIG; ++j) {
      // digit j's limb t: the input's own limb (t in [lo_j, hi_j)) or a lifted one
      const u64 v = (t >= a.lo[j] && t < a.hi[j]) ? __ldg(a.d[p] + (size_t)t * a.n + src)
                                                   : __ldg(a.ext_buf[p] + ((size_t)j * a.ext + t) * a.n + src);
      mac128(h0, l0, v, kb[j]);
      mac128(h1, l1, v, ka[j]);
    }
    if (MODE == IP_BASE && with_base) mac128(h0, l0, __ldg(a.base0[p] + (size_t)t * a.n + src), pm);
    u64 r0 = redc128(h0, l0, m), r1 = redc128(h1, l1, m);
    u64 *o0 = a.acc[p] + (size_t)t * a.n + k, *o1 = a.acc[p] + ((size_t)a.ext + t) * a.n + k;
    if (MODE == IP_ACC) {
      r0 = addmod(r0, *o0, m.q);
      r1 = addmod(r1, *o1, m.q);
    }
    *o0 = r0;
    *o1 = r1;
  }
}

// The same product for groups whose outputs share one key and one
// automorphism (a relinearisation batch; the outputs of one rotation step of a
// hoisted set), which the host checks per group: the key words, the gathered
// source index and the digit layout are fixed before the loop, so each output
// costs its loads, the multiply-accumulates, two reductions and two stores.
template <int NDIG, int MODE>
__global__ void __launch_bounds__(TPB, 4) k_inner_uni(const IPArgs a, int group) {
  const u32 k = blockIdx.y * TPB + threadIdx.x;
  const int t = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[a.mod_of[t]];
  const int kl = a.keylimb_of[t];
  const int p0 = blockIdx.x * group, p_end = min(a.np, p0 + group);
  const u64 *key = a.key[p0];
  u64 kb[NDIG], ka[NDIG];
  size_t off[NDIG];
  bool own[NDIG];
  const u32 src = gal_src(k, a.gal[p0], a.n, a.log_n);
#pragma unroll
  for (int j = 0; j < NDIG; ++j) {
    kb[j] = __ldg(key + ((size_t)(2 * j) * a.key_ext + kl) * a.n + k);
    ka[j] = __ldg(key + ((size_t)(2 * j + 1) * a.key_ext + kl) * a.n + k);
    own[j] = t >= a.lo[j] && t < a.hi[j];
    off[j] = (own[j] ? (size_t)t : (size_t)j * a.ext + t) * a.n + src;
  }
  const bool with_base = MODE == IP_BASE && t < a.nq_base;
  const u64 pm = with_base ? a.pm_mont[t] : 0;
  const size_t o_off = (size_t)t * a.n + k, o_pol = (size_t)a.ext * a.n;
  const size_t b_off = (size_t)t * a.n + src;
#pragma unroll 4
  for (int p = p0; p < p_end; ++p) {
    const u64 *dp = a.d[p], *ep = a.ext_buf[p];
    u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll
    for (int j = 0; j < NDIG; ++j) {
      const u64 v = __ldg((own[j] ? dp : ep) + off[j]);
      mac128(h0, l0, v, kb[j]);
      mac128(h1, l1, v, ka[j]);
    }
    if (MODE == IP_BASE && with_base) mac128(h0, l0, __ldg(a.base0[p] + b_off), pm);
    u64 r0 = redc128(h0, l0, m), r1 = redc128(h1, l1, m);
    u64 *o = a.acc[p] + o_off;
    if (MODE == IP_ACC) {
      r0 = addmod(r0, o[0], m.q);
      r1 = addmod(r1, o[o_pol], m.q);
    }
    o[0] = r0;
    o[o_pol] = r1;
  }
}

struct CombineArgs {
  const ModInfo *mods;
  u32 n;
  int log_n;
  int ext;
  const u64 *pinv;                 // [n_q] pairs
  const u64 *acc[MAX_CTS];
  const u64 *z[MAX_CTS];           // [2][l+1][N]
  const u64 *base0[MAX_CTS], *base1[MAX_CTS];
  u32 base0_gal[MAX_CTS];          // base0 read through sigma_g (1: as is)
  u64 *o0[MAX_CTS], *o1[MAX_CTS];
};

__global__ void __launch_bounds__(TPB) k_combine(const CombineArgs a, int nl) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, p = blockIdx.z;
  if (k >= a.n) return;
  const u64 q = a.mods[t].q, w = a.pinv[2 * t], ws = a.pinv[2 * t + 1];
  const size_t off = (size_t)t * a.n + k;
  const u64 x0 = a.acc[p][off], x1 = a.acc[p][(size_t)a.ext * a.n + off];
  const u64 z0 = a.z[p][off], z1 = a.z[p][(size_t)nl * a.n + off];
  u64 r0 = shoup(submod(x0, z0, q), w, ws, q);
  u64 r1 = shoup(submod(x1, z1, q), w, ws, q);
  if (a.base0[p]) r0 = addmod(r0, a.base0[p][(size_t)t * a.n + gal_src(k, a.base0_gal[p], a.n, a.log_n)], q);
  if (a.base1[p]) r1 = addmod(r1, a.base1[p][off], q);
  a.o0[p][off] = r0;
  a.o1[p][off] = r1;
}

// ---- ModDown and rescale merged (reading C21) ----
// Word offsets inside the level-l table block (ConvTables::mdr_off).
struct MdrLayout {
  size_t inv, tab, src_add, dst_sub, sinv, qlinv, pmod, rdiv, negs;
  MdrLayout(size_t off, int K, int l) {
    inv = off;
    tab = inv + 2 * (size_t)(K + 1);
    src_add = tab + (size_t)l * (K + 1);
    dst_sub = src_add + (K + 1);
    sinv = dst_sub + l;
    qlinv = sinv + 2 * (size_t)l;
    pmod = qlinv + 2 * (size_t)l;
    rdiv = pmod + 2;
    negs = rdiv + 2 * (size_t)(K + 1);
  }
};

struct FoldArgs {
  u32 n;
  int ext, l;
  u64 q, pm, pm_s;                 // q_l, [P]_{q_l} and its Shoup companion
  u64 *acc[MAX_CTS];               // [2][ext][N]
  const u64 *d0[MAX_CTS], *d1[MAX_CTS];
};

// acc_c[l] += [P]_{q_l} d_c[l]: the tensor term P d joins the top source limb
__global__ void __launch_bounds__(TPB) k_fold_top(const FoldArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int p = blockIdx.y, cc = blockIdx.z;
  if (k >= a.n) return;
  u64 *x = a.acc[p] + ((size_t)cc * a.ext + a.l) * a.n;
  const u64 *d = (cc ? a.d1[p] : a.d0[p]) + (size_t)a.l * a.n;
  x[k] = addmod(x[k], shoup(d[k], a.pm, a.pm_s, a.q), a.q);
}

struct CombineRArgs {
  const ModInfo *mods;
  u32 n;
  int ext, l;
  const u64 *sinv, *qlinv;         // [l] pairs: S^-1 and q_l^-1 mod q_t
  const u64 *acc[MAX_CTS];         // [2][ext][N]
  const u64 *z[MAX_CTS];           // [2][l][N]
  const u64 *d0[MAX_CTS], *d1[MAX_CTS];
  u64 *o0[MAX_CTS], *o1[MAX_CTS];
};

// out_c[t] = (acc_c[t] - z_c[t]) S^-1 + d_c[t] q_l^-1 mod q_t, t < l
// (= (acc + P d - z) S^-1; d and out may alias: each element is read first)
__global__ void __launch_bounds__(TPB) k_combine_rescale(const CombineRArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, p = blockIdx.z;
  if (k >= a.n) return;
  const u64 q = a.mods[t].q;
  const u64 sw = a.sinv[2 * t], sws = a.sinv[2 * t + 1], qw = a.qlinv[2 * t], qws = a.qlinv[2 * t + 1];
  const size_t off = (size_t)t * a.n + k;
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    const u64 x = a.acc[p][(size_t)cc * a.ext * a.n + off];
    const u64 zz = a.z[p][(size_t)cc * a.l * a.n + off];
    const u64 d = (cc ? a.d1[p] : a.d0[p])[off];
    const u64 r = addmod(shoup(submod(x, zz, q), sw, sws, q), shoup(d, qw, qws, q), q);
    (cc ? a.o1[p] : a.o0[p])[off] = r;
  }
}

int launch_bconv(ckks_ctx *c, BConvArgs &a, int ns, int np) {
  if (a.nt * ns > BCONV_MAX_TAB) return CKKS_E_PARAM;
  a.mods = c->d_mods;
  a.n = c->n;
  const bool merged = a.src_add && a.dst_sub && a.rdiv && a.negs;
  if (!merged && (a.src_add || a.dst_sub || a.rdiv || a.negs)) return CKKS_E_PARAM;  // all or none
  dim3 g((c->n + TPB - 1) / TPB, np);
  switch (ns) {
#define CASE(S)                                                                                         \
  case S:                                                                                               \
    if (merged)                                                                                         \
      PROF_LAUNCH(c, PK_BCONV, (u64)np * a.nt * S, (k_bconv<S, true><<<g, TPB, 0, c->stream>>>(a)));    \
    else                                                                                                \
      PROF_LAUNCH(c, PK_BCONV, (u64)np * a.nt * S, (k_bconv<S, false><<<g, TPB, 0, c->stream>>>(a)));   \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
    default: return CKKS_E_PARAM;
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

int check_shape(const ckks_ctx *c, int level) {
  const int nl = level + 1;
  const int ndig = (nl + c->alpha - 1) / c->alpha;
  if (ndig > MAXD || c->alpha > MAXS || c->n_p > MAXS) return CKKS_E_PARAM;
  return CKKS_OK;
}

}  // namespace

size_t ks_modup_words(const ckks_ctx *c, int level, int np) {
  const int nl = level + 1, ext = nl + c->n_p;
  const int ndig = (nl + c->alpha - 1) / c->alpha;
  return (size_t)c->n * (nl + (size_t)ndig * ext) * np;
}

size_t ks_tail_words(const ckks_ctx *c, int level, int nv) {
  const int nl = level + 1, ext = nl + c->n_p;
  return (size_t)c->n * (2 * ext + 2 * nl) * nv;
}

size_t ks_ws_words(const ckks_ctx *c, int level, int np) {
  return ks_modup_words(c, level, np) + ks_tail_words(c, level, np);
}

// ModUp of np <= MAX_CTS polynomials; ws holds per polynomial dc [l+1] then
// ext [ndig][l+1+K].  ext_out[i] receives polynomial i's ext pointer.
int ks_modup(ckks_ctx *c, int level, int np, const u64 *const *d, u64 *ws, u64 **ext_out) {
  if (np <= 0) return CKKS_OK;
  if (np > MAX_CTS) return CKKS_E_PARAM;
  int rc = check_shape(c, level);
  if (rc) return rc;
  const u32 n = c->n;
  const int nl = level + 1, ext = nl + c->n_p;
  const int ndig = (nl + c->alpha - 1) / c->alpha;
  const size_t per = ks_modup_words(c, level, 1);
  std::vector<u64 *> dc(np), eb(np);
  for (int i = 0; i < np; ++i) {
    dc[i] = ws + per * i;
    eb[i] = dc[i] + (size_t)nl * n;
    ext_out[i] = eb[i];
  }
  int mods[MAX_MODS];
  for (int t = 0; t < ext; ++t) mods[t] = c->ext_mod(level, t);
  if (c->use_fused && conv_fused_supported(c)) {
    // the fused pipeline: inverse row pass of every limb, one launch of the
    // fused column pass for all digits, the forward row pass of their targets
    rc = launch_ntt_part(c, d, dc.data(), np, nl, mods, true, NTT_ROWS);
    if (rc) return rc;
    FusedConv f;
    f.ndig = ndig;
    for (int j = 0; j < ndig; ++j) {
      const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, nl), ns = hi - lo;
      const u64 *tbl = c->d_conv + c->conv.modup_off[(size_t)level * c->n_digits + j];
      FusedConv::Digit &g = f.dig[j];
      g.ns = ns;
      g.nt = ext - ns;
      g.gap_lo = lo;
      g.gap_hi = hi;
      g.src_off = (size_t)lo * n;
      g.dst_off = (size_t)j * ext * n;
      for (int i = 0; i < ns; ++i) g.src_mod[i] = lo + i;
      g.inv = tbl;
      g.tab = tbl + 2 * ns;
    }
    for (int t = 0; t < ext; ++t) f.pos_mod[t] = mods[t];
    std::vector<const u64 *> dcc(dc.begin(), dc.end());
    rc = launch_conv_fused(c, f, dcc.data(), eb.data(), np);
    if (rc) return rc;
    std::vector<const u64 *> s2(np);
    std::vector<u64 *> d2(np);
    for (int j = 0; j < ndig; ++j) {
      const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, nl);
      if (lo > 0) {
        for (int i = 0; i < np; ++i) d2[i] = eb[i] + (size_t)j * ext * n, s2[i] = d2[i];
        rc = launch_ntt_part(c, s2.data(), d2.data(), np, lo, mods, false, NTT_ROWS);
        if (rc) return rc;
      }
      for (int i = 0; i < np; ++i) d2[i] = eb[i] + ((size_t)j * ext + hi) * n, s2[i] = d2[i];
      rc = launch_ntt_part(c, s2.data(), d2.data(), np, ext - hi, mods + hi, false, NTT_ROWS);
      if (rc) return rc;
    }
    return CKKS_OK;
  }
  rc = launch_ntt(c, d, dc.data(), np, nl, mods, true);
  if (rc) return rc;
  std::vector<const u64 *> srcs(np);
  std::vector<u64 *> dsts(np);
  for (int j = 0; j < ndig; ++j) {
    const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, nl), ns = hi - lo;
    BConvArgs a;
    const u64 *tbl = c->d_conv + c->conv.modup_off[(size_t)level * c->n_digits + j];
    a.inv = tbl;
    a.tab = tbl + 2 * ns;
    a.nt = ext - ns;
    for (int i = 0; i < ns; ++i) a.src_mod[i] = (unsigned char)(lo + i);
    int tt = 0;
    for (int t = 0; t < ext; ++t) {
      if (t >= lo && t < hi) continue;
      a.dst_mod[tt] = (unsigned char)mods[t];
      a.dst_pos[tt] = (unsigned char)t;
      ++tt;
    }
    for (int i = 0; i < np; ++i) {
      a.src[i] = dc[i] + (size_t)lo * n;
      a.dst[i] = eb[i] + (size_t)j * ext * n;
    }
    if (c->use_tc) {
      const size_t off = c->conv.modup_off[(size_t)level * c->n_digits + j];
      int sm[MAXS], dm[MAX_MODS], dp[MAX_MODS];
      for (int i = 0; i < ns; ++i) sm[i] = a.src_mod[i];
      for (int t = 0; t < a.nt; ++t) dm[t] = a.dst_mod[t], dp[t] = a.dst_pos[t];
      rc = launch_bconv_tc(c, off << 8 | (size_t)a.nt, c->h_conv.data() + off, c->h_conv.data() + off + 2 * ns, ns,
                           a.nt, sm, dm, dp, a.src, a.dst, np, nullptr, nullptr, nullptr, nullptr);
    } else {
      rc = launch_bconv(c, a, ns, np);
    }
    if (rc) return rc;
    if (lo > 0) {
      for (int i = 0; i < np; ++i) dsts[i] = eb[i] + (size_t)j * ext * n, srcs[i] = dsts[i];
      rc = launch_ntt(c, srcs.data(), dsts.data(), np, lo, mods, false);
      if (rc) return rc;
    }
    for (int i = 0; i < np; ++i) dsts[i] = eb[i] + ((size_t)j * ext + hi) * n, srcs[i] = dsts[i];
    rc = launch_ntt(c, srcs.data(), dsts.data(), np, ext - hi, mods + hi, false);
    if (rc) return rc;
  }
  return CKKS_OK;
}

// Inner product + ModDown for nv <= MAX_CTS outputs.  Output v uses input
// polynomial d[v] with its lifted digits ext[v], key keys[v] and automorphism
// gal[v]; ws holds per output acc [2][l+1+K] then z [2][l+1].
// Key inner product of nv outputs into acc[i] ([2][ext][N], NTT domain),
// overwriting or (accumulate) adding.
static int launch_inner(ckks_ctx *c, int level, int nv, const u64 *const *d, const u64 *const *ext_digits,
                        const u64 *const *keys, const u32 *gal, u64 *const *acc, bool accumulate,
                        const u64 *const *pbase0 = nullptr) {
  const u32 n = c->n;
  const int nl = level + 1, ext = nl + c->n_p;
  const int ndig = (nl + c->alpha - 1) / c->alpha;
  if (pbase0 && accumulate) return CKKS_E_PARAM;
  // the Montgomery reduction's input bound: (terms) max q < 2^65
  for (int t = 0; t < ext; ++t)
    if ((unsigned __int128)(ndig + (pbase0 ? 1 : 0)) * c->mod[c->ext_mod(level, t)] >= ((unsigned __int128)1 << 65))
      return CKKS_E_PARAM;
  IPArgs a;
  a.mods = c->d_mods;
  a.n = n;
  a.log_n = c->log_n;
  a.ext = ext;
  a.ndig = ndig;
  a.key_ext = c->n_q + c->n_p;
  a.kc = c->key_compressed ? 1 : 0;
  a.np = nv;
  a.nq_base = pbase0 ? nl : 0;
  if (pbase0)
    for (int t = 0; t < nl; ++t) {
      const u64 q = c->mod[t];
      u64 pm = 1;
      for (int k = 0; k < c->n_p; ++k) pm = host_mulmod(pm, c->mod[c->n_q + k] % q, q);
      a.pm_mont[t] = host_mulmod(pm, (u64)(((unsigned __int128)1 << 64) % q), q);
    }
  for (int t = 0; t < ext; ++t) {
    a.mod_of[t] = (unsigned char)c->ext_mod(level, t);
    a.keylimb_of[t] = (unsigned char)c->key_limb(level, t);
  }
  for (int j = 0; j < ndig; ++j) {
    a.lo[j] = j * c->alpha;
    a.hi[j] = std::min((j + 1) * c->alpha, nl);
  }
  for (int i = 0; i < nv; ++i) {
    a.d[i] = d[i];
    a.ext_buf[i] = ext_digits[i];
    a.key[i] = keys[i];
    a.gal[i] = gal ? gal[i] : 1u;
    a.acc[i] = acc[i];
    a.base0[i] = pbase0 ? pbase0[i] : nullptr;
  }
  int group = c->ip_group > 0 ? c->ip_group : 8;
  c->prof.count_ks(level, (unsigned long long)nv);
  // every group of outputs on one key and one automorphism: the uniform kernel,
  // at the largest group (the tuned one, halved as needed) for which that holds
  auto uniform = [&](int gs) {
    for (int p = 0; p < nv; ++p) {
      const int q0 = p - p % gs;
      if (a.key[p] != a.key[q0] || a.gal[p] != a.gal[q0]) return false;
    }
    return true;
  };
  bool uni = false;
  if (!a.kc && ndig <= 4)
    for (int gs = group; gs >= 4 && !uni; gs /= 2)
      if (uniform(gs)) {
        uni = true;
        group = gs;
      }
  dim3 g((nv + group - 1) / group, (n + TPB - 1) / TPB, ext);
  if (uni) {
    switch (ndig) {
#define UCASE(D)                                                                                          \
  case D:                                                                                                 \
    if (pbase0)                                                                                           \
      PROF_LAUNCH(c, PK_INNER, (u64)nv * ext, (k_inner_uni<D, IP_BASE><<<g, TPB, 0, c->stream>>>(a, group))); \
    else if (accumulate)                                                                                  \
      PROF_LAUNCH(c, PK_INNER, (u64)nv * ext, (k_inner_uni<D, IP_ACC><<<g, TPB, 0, c->stream>>>(a, group)));  \
    else                                                                                                  \
      PROF_LAUNCH(c, PK_INNER, (u64)nv * ext, (k_inner_uni<D, IP_SET><<<g, TPB, 0, c->stream>>>(a, group)));  \
    break;
      UCASE(1) UCASE(2) UCASE(3) UCASE(4)
#undef UCASE
    }
    return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
  }
  switch (ndig) {
#define ILAUNCH(D, M)                                                                                        \
  do {                                                                                                       \
    if (a.kc)                                                                                                \
      PROF_LAUNCH(c, PK_INNER, (u64)nv * ext, (k_inner<D, M, true><<<g, TPB, 0, c->stream>>>(a, group)));   \
    else                                                                                                     \
      PROF_LAUNCH(c, PK_INNER, (u64)nv * ext, (k_inner<D, M, false><<<g, TPB, 0, c->stream>>>(a, group)));  \
  } while (0)
#define ICASE(D)                                                                                    \
  case D:                                                                                           \
    if (pbase0)                                                                                     \
      ILAUNCH(D, IP_BASE);                                                                          \
    else if (accumulate)                                                                            \
      ILAUNCH(D, IP_ACC);                                                                           \
    else                                                                                            \
      ILAUNCH(D, IP_SET);                                                                           \
    break;
    ICASE(1) ICASE(2) ICASE(3) ICASE(4) ICASE(5) ICASE(6) ICASE(7) ICASE(8)
#undef ICASE
#undef ILAUNCH
    default: return CKKS_E_PARAM;
  }
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

static int combine_rescale(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *z,
                           const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1,
                           const MdrLayout &L);
static int finish_rescale(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *z,
                          const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1,
                          const MdrLayout &L, int part);

// The fused finish moves 16-byte words: accumulators, outputs and bases read
// as they are must be 16-byte aligned (else the separate combine kernels run).
static bool finish_aligned(const RowFinish &f, int np) {
  for (int i = 0; i < np; ++i) {
    uintptr_t a = (uintptr_t)f.acc[i] | (uintptr_t)f.out[i];
    if (f.base[i] && f.gal[i] == 1) a |= (uintptr_t)f.base[i];
    if (a & 15) return false;
  }
  return true;
}

// ModDown and rescale merged (reading C21) on the accumulators of nv outputs:
// o_c = round((acc_c + P base_c) / (P q_l)) - u over q_0..q_{l-1}.
static int ks_merged_tail(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *z, const int *mods,
                          const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1) {
  const u32 n = c->n;
  const int l = level, nl = level + 1, K = c->n_p, ext = nl + K, ns = K + 1;
  if (l < 1 || ns > MAXS || !base0 || !base1) return CKKS_E_PARAM;
  const MdrLayout L(c->conv.mdr_off[l], K, l);
  const u64 *hc = c->h_conv.data();
  int rc;
  {  // the tensor term P d joins the top limb (P d vanishes modulo P)
    FoldArgs f;
    f.n = n;
    f.ext = ext;
    f.l = l;
    f.q = c->mod[l];
    f.pm = hc[L.pmod];
    f.pm_s = hc[L.pmod + 1];
    for (int i = 0; i < nv; ++i) {
      f.acc[i] = acc[i];
      f.d0[i] = base0[i];
      f.d1[i] = base1[i];
    }
    dim3 g((n + TPB - 1) / TPB, nv, 2);
    PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nv * 2, (k_fold_top<<<g, TPB, 0, c->stream>>>(f)));
    if (cudaGetLastError() != cudaSuccess) return CKKS_E_CUDA;
  }
  // the sources q_l, p_0..p_{K-1} are adjacent in the accumulator: to coefficients
  std::vector<const u64 *> ps(2 * nv);
  std::vector<u64 *> pd(2 * nv);
  for (int i = 0; i < nv; ++i)
    for (int cc = 0; cc < 2; ++cc) {
      pd[2 * i + cc] = acc[i] + ((size_t)cc * ext + l) * n;
      ps[2 * i + cc] = pd[2 * i + cc];
    }
  if (c->use_fused && conv_fused_supported(c)) {
    rc = launch_ntt_part(c, ps.data(), pd.data(), 2 * nv, ns, mods + l, true, NTT_ROWS);
    if (rc) return rc;
    FusedConv f;
    f.ndig = 1;
    FusedConv::Digit &g = f.dig[0];
    g.ns = ns;
    g.nt = l;
    g.gap_lo = g.gap_hi = l;
    g.src_mod[0] = l;
    for (int k = 0; k < K; ++k) g.src_mod[1 + k] = c->n_q + k;
    g.inv = c->d_conv + L.inv;
    g.tab = c->d_conv + L.tab;
    for (int t = 0; t < l; ++t) f.pos_mod[t] = t;
    f.src_add = c->d_conv + L.src_add;
    f.dst_sub = c->d_conv + L.dst_sub;
    f.rdiv = c->d_conv + L.rdiv;
    f.negs = c->d_conv + L.negs;
    std::vector<u64 *> pz(2 * nv);
    for (int i = 0; i < nv; ++i)
      for (int cc = 0; cc < 2; ++cc) pz[2 * i + cc] = z[i] + (size_t)cc * l * n;
    for (int p0 = 0; p0 < 2 * nv; p0 += MAX_CTS) {
      const int cnt = std::min(MAX_CTS, 2 * nv - p0);
      rc = launch_conv_fused(c, f, ps.data() + p0, pz.data() + p0, cnt);
      if (rc) return rc;
    }
    return finish_rescale(c, level, nv, acc, z, base0, base1, o0, o1, L, NTT_ROWS);
  }
  rc = launch_ntt(c, ps.data(), pd.data(), 2 * nv, ns, mods + l, true);
  if (rc) return rc;
  for (int p0 = 0; p0 < 2 * nv; p0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, 2 * nv - p0);
    BConvArgs a;
    a.inv = c->d_conv + L.inv;
    a.tab = c->d_conv + L.tab;
    a.src_add = c->d_conv + L.src_add;
    a.dst_sub = c->d_conv + L.dst_sub;
    a.rdiv = c->d_conv + L.rdiv;
    a.negs = c->d_conv + L.negs;
    a.nt = l;
    a.src_mod[0] = (unsigned char)l;
    for (int k = 0; k < K; ++k) a.src_mod[1 + k] = (unsigned char)(c->n_q + k);
    for (int t = 0; t < l; ++t) {
      a.dst_mod[t] = (unsigned char)t;
      a.dst_pos[t] = (unsigned char)t;
    }
    for (int x = 0; x < cnt; ++x) {
      const int pp = p0 + x, i = pp / 2, cc = pp % 2;
      a.src[x] = pd[pp];
      a.dst[x] = z[i] + (size_t)cc * l * n;
    }
    if (c->use_tc) {
      int sm[MAXS], dm[MAX_MODS], dp[MAX_MODS];
      for (int i = 0; i < ns; ++i) sm[i] = a.src_mod[i];
      for (int t = 0; t < l; ++t) dm[t] = t, dp[t] = t;
      rc = launch_bconv_tc(c, L.inv << 8 | (size_t)l, hc + L.inv, hc + L.tab, ns, l, sm, dm, dp, a.src, a.dst, cnt,
                           hc + L.src_add, hc + L.dst_sub, hc + L.rdiv, hc + L.negs);
    } else {
      rc = launch_bconv(c, a, ns, cnt);
    }
    if (rc) return rc;
  }
  return finish_rescale(c, level, nv, acc, z, base0, base1, o0, o1, L, NTT_BOTH);
}

// The forward transform of the converted limbs z (the row pass alone after a
// fused column pass: part NTT_ROWS), then the merged finish: in the row pass's
// output stage (fuse_finish) or by k_combine_rescale after it.
static int finish_rescale(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *z,
                          const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1,
                          const MdrLayout &L, int part) {
  const u32 n = c->n;
  const int l = level, ext = level + 1 + c->n_p;
  int mods[MAX_MODS];
  for (int t = 0; t < l; ++t) mods[t] = c->ext_mod(level, t);
  std::vector<u64 *> pz(2 * nv);
  std::vector<const u64 *> pzc(2 * nv);
  for (int i = 0; i < nv; ++i)
    for (int cc = 0; cc < 2; ++cc) pz[2 * i + cc] = z[i] + (size_t)cc * l * n, pzc[2 * i + cc] = pz[2 * i + cc];
  if (c->fuse_finish) {
    RowFinish f;
    f.w = c->d_conv + L.sinv;
    f.wb = c->d_conv + L.qlinv;
    for (int i = 0; i < nv; ++i)
      for (int cc = 0; cc < 2; ++cc) {
        const int pp = 2 * i + cc;
        f.acc[pp] = acc[i] + (size_t)cc * ext * n;
        f.base[pp] = cc ? base1[i] : base0[i];
        f.gal[pp] = 1u;
        f.out[pp] = cc ? o1[i] : o0[i];
      }
    if (finish_aligned(f, 2 * nv)) return launch_ntt_fwd_finish(c, pzc.data(), pz.data(), 2 * nv, l, mods, part, f);
  }
  const int rc = launch_ntt_part(c, pzc.data(), pz.data(), 2 * nv, l, mods, false, part);
  if (rc) return rc;
  return combine_rescale(c, level, nv, acc, z, base0, base1, o0, o1, L);
}

// out_c = (acc_c - z_c) S^-1 + d_c q_l^-1 over q_0..q_{l-1} (the merged finish)
static int combine_rescale(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *z,
                           const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1,
                           const MdrLayout &L) {
  const u32 n = c->n;
  const int l = level, ext = level + 1 + c->n_p;
  CombineRArgs r;
  r.mods = c->d_mods;
  r.n = n;
  r.ext = ext;
  r.l = l;
  r.sinv = c->d_conv + L.sinv;
  r.qlinv = c->d_conv + L.qlinv;
  for (int i = 0; i < nv; ++i) {
    r.acc[i] = acc[i];
    r.z[i] = z[i];
    r.d0[i] = base0[i];
    r.d1[i] = base1[i];
    r.o0[i] = o0[i];
    r.o1[i] = o1[i];
  }
  dim3 g((n + TPB - 1) / TPB, l, nv);
  PROF_LAUNCH(c, PK_COMBINE, (u64)nv * l, (k_combine_rescale<<<g, TPB, 0, c->stream>>>(r)));
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

// C9 ModDown of nv accumulators acc[i] ([2][l+1+K][N], NTT domain; their
// special limbs are consumed) plus the optional base: o_c = base_c +
// (acc_c[Q] - z_c) P^-1, base0 read through sigma_g (base0_gal) when given.
static int moddown_tail(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *z, const int *mods,
                        const u64 *const *base0, const u32 *base0_gal, const u64 *const *base1, u64 *const *o0,
                        u64 *const *o1) {
  const u32 n = c->n;
  const int nl = level + 1, K = c->n_p, ext = nl + K;
  int rc;
  std::vector<const u64 *> ps(2 * nv);
  std::vector<u64 *> pd(2 * nv);
  for (int i = 0; i < nv; ++i)
    for (int cc = 0; cc < 2; ++cc) {
      pd[2 * i + cc] = acc[i] + ((size_t)cc * ext + nl) * n;
      ps[2 * i + cc] = pd[2 * i + cc];
    }
  const bool fused = c->use_fused && conv_fused_supported(c);
  rc = launch_ntt_part(c, ps.data(), pd.data(), 2 * nv, K, mods + nl, true, fused ? NTT_ROWS : NTT_BOTH);
  if (rc) return rc;
  if (fused) {
    FusedConv f;
    f.ndig = 1;
    FusedConv::Digit &g = f.dig[0];
    g.ns = K;
    g.nt = nl;
    g.gap_lo = g.gap_hi = nl;
    for (int k = 0; k < K; ++k) g.src_mod[k] = c->n_q + k;
    g.inv = c->d_conv + c->conv.moddown_phat_inv;
    g.tab = c->d_conv + c->conv.moddown_phat_mod;
    for (int t = 0; t < nl; ++t) f.pos_mod[t] = t;
    std::vector<u64 *> pz(2 * nv);
    for (int i = 0; i < nv; ++i)
      for (int cc = 0; cc < 2; ++cc) pz[2 * i + cc] = z[i] + (size_t)cc * nl * n;
    for (int p0 = 0; p0 < 2 * nv; p0 += MAX_CTS) {
      const int cnt = std::min(MAX_CTS, 2 * nv - p0);
      rc = launch_conv_fused(c, f, ps.data() + p0, pz.data() + p0, cnt);
      if (rc) return rc;
    }
  }
  for (int p0 = 0; !fused && p0 < 2 * nv; p0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, 2 * nv - p0);
    BConvArgs a;
    a.inv = c->d_conv + c->conv.moddown_phat_inv;
    a.tab = c->d_conv + c->conv.moddown_phat_mod;
    a.nt = nl;
    for (int i = 0; i < K; ++i) a.src_mod[i] = (unsigned char)(c->n_q + i);
    for (int t = 0; t < nl; ++t) {
      a.dst_mod[t] = (unsigned char)t;
      a.dst_pos[t] = (unsigned char)t;
    }
    for (int x = 0; x < cnt; ++x) {
      const int pp = p0 + x, i = pp / 2, cc = pp % 2;
      a.src[x] = pd[pp];
      a.dst[x] = z[i] + (size_t)cc * nl * n;
    }
    if (c->use_tc) {
      int sm[MAXS], dm[MAX_MODS], dp[MAX_MODS];
      for (int i = 0; i < K; ++i) sm[i] = a.src_mod[i];
      for (int t = 0; t < nl; ++t) dm[t] = t, dp[t] = t;
      rc = launch_bconv_tc(c, c->conv.moddown_phat_mod << 8 | (size_t)nl, c->h_conv.data() + c->conv.moddown_phat_inv,
                           c->h_conv.data() + c->conv.moddown_phat_mod, K, nl, sm, dm, dp, a.src, a.dst, cnt,
                           nullptr, nullptr, nullptr, nullptr);
    } else {
      rc = launch_bconv(c, a, K, cnt);
    }
    if (rc) return rc;
  }
  for (int i = 0; i < nv; ++i)
    for (int cc = 0; cc < 2; ++cc) {
      pd[2 * i + cc] = z[i] + (size_t)cc * nl * n;
      ps[2 * i + cc] = pd[2 * i + cc];
    }
  if (c->fuse_finish) {
    RowFinish f;
    f.w = c->d_conv + c->conv.moddown_pinv;
    for (int i = 0; i < nv; ++i)
      for (int cc = 0; cc < 2; ++cc) {
        const int pp = 2 * i + cc;
        f.acc[pp] = acc[i] + (size_t)cc * ext * n;
        f.base[pp] = cc ? (base1 ? base1[i] : nullptr) : (base0 ? base0[i] : nullptr);
        f.gal[pp] = (!cc && base0_gal) ? base0_gal[i] : 1u;
        f.out[pp] = cc ? o1[i] : o0[i];
      }
    if (finish_aligned(f, 2 * nv))
      return launch_ntt_fwd_finish(c, ps.data(), pd.data(), 2 * nv, nl, mods, fused ? NTT_ROWS : NTT_BOTH, f);
  }
  rc = launch_ntt_part(c, ps.data(), pd.data(), 2 * nv, nl, mods, false, fused ? NTT_ROWS : NTT_BOTH);
  if (rc) return rc;
  CombineArgs a;
  a.mods = c->d_mods;
  a.n = n;
  a.log_n = c->log_n;
  a.ext = ext;
  a.pinv = c->d_conv + c->conv.moddown_pinv;
  for (int i = 0; i < nv; ++i) {
    a.acc[i] = acc[i];
    a.z[i] = z[i];
    a.base0[i] = base0 ? base0[i] : nullptr;
    a.base0_gal[i] = base0_gal ? base0_gal[i] : 1u;
    a.base1[i] = base1 ? base1[i] : nullptr;
    a.o0[i] = o0[i];
    a.o1[i] = o1[i];
  }
  dim3 g((n + TPB - 1) / TPB, nl, nv);
  PROF_LAUNCH(c, PK_COMBINE, (u64)nv * nl, (k_combine<<<g, TPB, 0, c->stream>>>(a, nl)));
  if (cudaGetLastError() != cudaSuccess) return CKKS_E_CUDA;
  return CKKS_OK;
}


int ks_tail(ckks_ctx *c, int level, int nv, const u64 *const *d, const u64 *const *ext_digits,
            const u64 *const *keys, const u32 *gal, const u64 *const *base0, const u32 *base0_gal,
            const u64 *const *base1, u64 *const *o0, u64 *const *o1, u64 *ws, bool merged) {
  if (nv <= 0) return CKKS_OK;
  if (nv > MAX_CTS) return CKKS_E_PARAM;
  int rc = check_shape(c, level);
  if (rc) return rc;
  if (merged && (base0_gal || level < 1)) return CKKS_E_PARAM;
  const u32 n = c->n;
  const int nl = level + 1, K = c->n_p, ext = nl + K;
  const size_t per = ks_tail_words(c, level, 1);
  std::vector<u64 *> acc(nv), z(nv);
  for (int i = 0; i < nv; ++i) {
    acc[i] = ws + per * i;
    z[i] = acc[i] + (size_t)2 * ext * n;
  }
  int mods[MAX_MODS];
  for (int t = 0; t < ext; ++t) mods[t] = c->ext_mod(level, t);
  rc = launch_inner(c, level, nv, d, ext_digits, keys, gal, acc.data(), false);
  if (rc) return rc;
  if (merged) return ks_merged_tail(c, level, nv, acc.data(), z.data(), mods, base0, base1, o0, o1);
  return moddown_tail(c, level, nv, acc.data(), z.data(), mods, base0, base0_gal, base1, o0, o1);
}

int ks_accumulate(ckks_ctx *c, int level, int nv, const u64 *const *d, const u64 *const *ext_digits,
                  const u64 *const *keys, const u32 *gal, u64 *const *acc, bool accumulate,
                  const u64 *const *pbase0) {
  if (nv <= 0) return CKKS_OK;
  if (nv > MAX_CTS || level + 1 > CKKS_MAX_Q) return CKKS_E_PARAM;
  int rc = check_shape(c, level);
  if (rc) return rc;
  return launch_inner(c, level, nv, d, ext_digits, keys, gal, acc, accumulate, pbase0);
}

size_t ks_merged_words(const ckks_ctx *c, int level, int nv) { return (size_t)2 * level * c->n * nv; }

int ks_moddown_finish(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *o0, u64 *const *o1, u64 *ws) {
  if (nv <= 0) return CKKS_OK;
  if (nv > MAX_CTS) return CKKS_E_PARAM;
  int rc = check_shape(c, level);
  if (rc) return rc;
  const int ext = level + 1 + c->n_p;
  std::vector<u64 *> z(nv);
  for (int i = 0; i < nv; ++i) z[i] = ws + (size_t)2 * (level + 1) * c->n * i;
  int mods[MAX_MODS];
  for (int t = 0; t < ext; ++t) mods[t] = c->ext_mod(level, t);
  return moddown_tail(c, level, nv, acc, z.data(), mods, nullptr, nullptr, nullptr, o0, o1);
}

int ks_merged_finish(ckks_ctx *c, int level, int nv, u64 *const *acc, const u64 *const *base0,
                     const u64 *const *base1, u64 *const *o0, u64 *const *o1, u64 *ws) {
  if (nv <= 0) return CKKS_OK;
  if (nv > MAX_CTS || level < 1) return CKKS_E_PARAM;
  int rc = check_shape(c, level);
  if (rc) return rc;
  const int ext = level + 1 + c->n_p;
  std::vector<u64 *> z(nv);
  for (int i = 0; i < nv; ++i) z[i] = ws + (size_t)2 * level * c->n * i;
  int mods[MAX_MODS];
  for (int t = 0; t < ext; ++t) mods[t] = c->ext_mod(level, t);
  return ks_merged_tail(c, level, nv, acc, z.data(), mods, base0, base1, o0, o1);
}

int ks_batch(ckks_ctx *c, int level, int np, const u64 *const *d, const u64 *const *keys,
             const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1,
             u64 *ws, bool merged) {
  if (np <= 0) return CKKS_OK;
  if (np > MAX_CTS) return CKKS_E_PARAM;
  std::vector<u64 *> eb(np);
  int rc = ks_modup(c, level, np, d, ws, eb.data());
  if (rc) return rc;
  std::vector<const u64 *> ebc(eb.begin(), eb.end());
  return ks_tail(c, level, np, d, ebc.data(), keys, nullptr, base0, nullptr, base1, o0, o1,
                 ws + ks_modup_words(c, level, np), merged);
}
