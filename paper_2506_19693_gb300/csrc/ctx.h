// Internal (host-side) context of the GB300 RNS-CKKS core.
#pragma once

#include <map>
#include <vector>

#include "common.cuh"
#include "prof.h"

// A Galois or relinearisation key resident in HBM:
// uint64[n_digits][2][n_q + n_p][N] (b_j, a_j), NTT domain.
struct DevKey {
  u64 *data = nullptr;
};
// A compressed switching key stores KEY_HDR header words (the uniform
// generator's state for each digit's a row) and the b rows [n_digits][ext][N];
// the key inner product regenerates a from the header (reading C22).
constexpr int KEY_HDR = 16;

// Per-level basis-conversion constants for ModUp of digit j at level l and for
// ModDown / rescale.  All live in one device buffer; these are host offsets.
struct ConvTables {
  // ModUp(level l, digit j): source limbs [lo, hi), hi <= l+1.
  //   qhat_inv[i], qhat_inv_s[i]        (i < hi-lo)      : [Qhat_i^-1]_{q_i} and Shoup
  //   qhat_mod[t * n_src + i]                             : Qhat_i mod target t
  // targets t enumerate (q_0..q_l minus [lo,hi)) then p_0..p_{K-1}.
  std::vector<size_t> modup_off;   // index l * n_digits + j -> offset (u64 words)
  // ModDown to level l: phat_inv[k] (Shoup pair), phat_mod[i * K + k], pinv[i] (Shoup pair)
  size_t moddown_phat_inv = 0;     // [K] pairs
  size_t moddown_phat_mod = 0;     // [n_q][K]
  size_t moddown_pinv = 0;         // [n_q] pairs
  // rescale from level l: qlinv[l * n_q + i] (Shoup pair) = q_l^-1 mod q_i
  size_t rescale_qlinv = 0;
  // ModDown and rescale merged at level l >= 1 (reading C21): S = P q_l,
  // sources (q_l, p_0..p_{K-1}), targets q_0..q_{l-1}.  At mdr_off[l]:
  //   inv[K+1] pairs   [Shat_i^-1]_{s_i}                 (Shat_i = S / s_i)
  //   tab[l][K+1]      Shat_i mod q_t
  //   src_add[K+1]     [((s_i - 1)/2) Shat_i^-1]_{s_i}    (adds H = (S-1)/2 to each source)
  //   dst_sub[l]       [H]_{q_t}
  //   sinv[l] pairs    S^-1 mod q_t
  //   qlinv[l] pairs   q_l^-1 mod q_t
  //   pmod pair        [P]_{q_l}
  //   rdiv[2][K+1]     R_i = floor(2^96 / s_i) as low words, then high words
  //                    (R_i >= 2^64 only for s_i < 2^32): y_i / s_i in 32.32
  //                    fixed point is y_i R_hi + floor(y_i R_lo / 2^64), exact
  //   negs[l]          -S mod q_t (removes the overflow estimate v S)
  std::vector<size_t> mdr_off;     // index l (0 unused)
  // decode: Garner constants inv(q_j) mod q_i  [n_q][n_q] and half-Q digits per level
  size_t garner_inv = 0;
  size_t halfq_digits = 0;         // [n_q][n_q]: digits of (Q_l - 1)/2 for level l
  size_t total = 0;
};

struct BootState;  // boot.cu

struct ckks_ctx {
  BootState *boot = nullptr;
  u32 boot_slots = 0;                // bootstrapping slot count (0: N/2; reading B13 below that)
  int device = 0;
  cudaStream_t stream = nullptr;
  int log_n = 0;
  u32 n = 0;
  int n_q = 0, n_p = 0, dnum = 0, alpha = 0, n_digits = 0, h = 0;
  double sigma = 3.2, default_scale = 1.0;
  i64 e_bound = 19;
  u64 mod[MAX_MODS] = {0};
  u64 psi[MAX_MODS] = {0};

  // device tables
  ModInfo *d_mods = nullptr;         // [n_q + n_p]
  ulonglong2 *d_tw_fwd = nullptr;    // [n_q + n_p][N]: (psi^brv(k), Shoup)
  ulonglong2 *d_tw_inv = nullptr;    // [n_q + n_p][N]: (psi^-brv(k), Shoup)
  // the row pass's per-thread twiddles (second register phase) regrouped so
  // that a warp's load is contiguous: [n_q + n_p][s < 4][i < 2^s][N/16] holds
  // tw[((N/16 + m) << s) + i] at m (forward and inverse tables)
  ulonglong2 *d_tw_row_fwd = nullptr;
  ulonglong2 *d_tw_row_inv = nullptr;
  u64 *d_conv = nullptr;             // ConvTables payload
  ConvTables conv;
  std::vector<u64> h_conv;           // host copy of the payload

  // secret
  bool have_secret = false;
  std::vector<int8_t> s_host;        // [N]
  u64 *d_s_ntt = nullptr;            // [n_q + n_p][N]
  u64 *d_pk = nullptr;               // [2][n_q][N] public key (b, a), NTT domain, or null
  u64 key_seed = 0;
  DevKey relin;
  std::map<u64, DevKey> galois;
  bool key_compressed = false;       // keys generated with a regenerated from its seed (C22)

  // scratch (grown on demand, owned)
  u64 *scratch = nullptr;
  size_t scratch_words = 0;
  double *fscratch = nullptr;
  size_t fscratch_words = 0;
  void *pinned = nullptr;            // pinned host staging
  size_t pinned_bytes = 0;
  size_t table_bytes = 0;
  Profiler prof;
  int ip_group = 8;                  // key inner product: outputs per thread (ckks_tune)
  int ntt_rows = 16;                 // NTT row pass: rows per CTA, 16 or 8 (ckks_tune_ntt)
  bool ntt_cluster = false;          // forward NTT at N = 2^16 in one pass on an 8-CTA cluster
  bool use_tc = false;               // basis conversion on the tensor cores (ckks_ctx_set_form)
  bool use_fused = false;            // conversion fused with the transforms' column passes (N <= 2^16)
  bool fuse_finish = true;           // key-switch finish in the forward row pass (ckks_ctx_set_fused_finish)
  int fin_rows = 0;                  // row tile of that row pass: 16 or 8 (0: as ntt_rows)
  std::map<size_t, void *> tc_bmats; // byte-plane constants per conversion
  int *tc_err = nullptr;             // device flag: a bounded wait expired
  // host-streamed batches (ckks_mul_relin_host): copy streams, staging slots, events
  cudaStream_t h2d = nullptr, d2h = nullptr;
  u64 *stage = nullptr;
  size_t stage_words = 0;
  cudaEvent_t ev_in[3] = {nullptr, nullptr, nullptr}, ev_comp[3] = {nullptr, nullptr, nullptr},
              ev_out[3] = {nullptr, nullptr, nullptr};
  bool capturing = false;            // inside a CUDA-graph capture: no allocation, no sync

  size_t limb_words() const { return (size_t)n; }
  int ext_limbs(int level) const { return level + 1 + n_p; }
  // index into the key's limb axis for extended-basis position t at level l
  int key_limb(int level, int t) const { return t <= level ? t : n_q + (t - level - 1); }
  // modulus index of extended-basis position t at level l
  int ext_mod(int level, int t) const { return t <= level ? t : n_q + (t - level - 1); }
};

// ---- host parameter derivation (params_host.cpp) ----
int host_gen_primes(int count, const unsigned *bits, int log_step, u64 *out);
u64 host_find_psi(u64 q, u64 n);
u64 host_powmod(u64 b, u64 e, u64 q);
u64 host_mulmod(u64 a, u64 b, u64 q);
u64 host_invmod(u64 a, u64 q);
u64 host_shoup(u64 w, u64 q);
u64 host_bitrev(u64 x, int bits);
int build_tables(ckks_ctx *c);

// ---- host sampling (sampling_host.cpp) ----
u64 sm_draw(u64 key, u64 ctr);
u64 sm_stream(u64 seed, u64 tag, u64 idx);
enum { TAG_SECRET = 1, TAG_KEY_A = 2, TAG_KEY_E = 3, TAG_ENC_A = 4, TAG_ENC_E = 5,
       TAG_PK_A = 6, TAG_PK_E = 7, TAG_PKENC_V = 8, TAG_PKENC_E0 = 9, TAG_PKENC_E1 = 10 };
void sample_secret(u64 seed, u32 n, int h, int8_t *s);
void sample_gaussian(u64 key, u32 n, double sigma, i64 bound, i64 *e);
// public-key encryption's mask: 0 with probability 1/2, +1 and -1 with 1/4 each
void sample_pk_mask(u64 key, u32 n, i64 *v);
u64 sample_uniform(u64 key, u64 idx, u64 q);

// ---- scratch ----
int ensure_scratch(ckks_ctx *c, size_t words);
int ensure_fscratch(ckks_ctx *c, size_t words);

// ---- NTT launchers (ntt.cu) ----
// Transform `npoly` polynomials of `nl` limbs each.  Limb l of poly p is at
// src.p[p] + l*N (read) and dst.p[p] + l*N (written); its modulus index is
// mods[l].  src may equal dst.
int launch_ntt(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl,
               const int *mods, bool inverse);
// One pass only: NTT_ROWS runs the row pass alone (the inverse's first pass,
// src -> dst; the forward's last pass, src -> dst) around a fused column pass.
enum { NTT_COLS = 1, NTT_ROWS = 2, NTT_BOTH = 3 };
int launch_ntt_part(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl,
                    const int *mods, bool inverse, int part);
// The key-switch finish in the forward row pass's output stage (reading C9 and
// C21; the rescale's last step, C10, has the same form): for limb t of
// polynomial p, with v the transform's fully reduced output, out[p][t] =
// (acc[p][t] - v) w_t + b, where b = base[p][t] read through sigma_gal[p] (wb
// null) or b = base[p][t] wb_t (wb set, gal 1), and b = 0 without a base.  v
// itself is not stored.  acc, base (with gal 1) and out are 16-byte aligned;
// out may equal acc, and may alias base only with gal 1.
struct RowFinish {
  const u64 *w = nullptr;          // device [nl] pairs: w_t and its Shoup companion
  const u64 *wb = nullptr;         // device [nl] pairs, or null
  const u64 *acc[MAX_POLYS];       // limb 0 of each polynomial's accumulator
  const u64 *base[MAX_POLYS];      // limb 0, or null
  u32 gal[MAX_POLYS];
  u64 *out[MAX_POLYS];
};
// The forward transform (NTT_BOTH, or its row pass alone after a fused column
// pass: NTT_ROWS) of npoly <= MAX_POLYS polynomials, finished by `f` instead of
// storing the result in dst (which then holds the column pass's output only).
// Always the two-pass form.
int launch_ntt_fwd_finish(ckks_ctx *c, const u64 *const *src, u64 *const *dst, int npoly, int nl,
                          const int *mods, int part, const RowFinish &f);
// The one-pass forward transform on an 8-CTA cluster (N = 2^16 only): opt in
// its shared memory and count the clusters the device holds at once.
int ntt_cluster_prepare(const ckks_ctx *c, int *max_clusters);

// ---- fused conversion column pass (ntt.cu) ----
// A basis conversion between NTT domains with its transforms' column passes
// fused in one kernel: the sources have had the inverse row pass
// (launch_ntt_part NTT_ROWS), the targets get the forward row pass after.
struct FusedConv {
  struct Digit {
    int ns = 0, nt = 0, gap_lo = 0, gap_hi = 0;  // targets tt -> limb tt (< gap_lo) or tt + gap_hi - gap_lo
    size_t src_off = 0, dst_off = 0;            // words from a polynomial's src / dst pointer
    int src_mod[16] = {0};
    const u64 *inv = nullptr;                   // device [ns] Shoup pairs
    const u64 *tab = nullptr;                   // device [nt][ns]
  };
  int ndig = 0;
  Digit dig[8];
  int pos_mod[MAX_MODS] = {0};                  // modulus of each target limb position
  const u64 *src_add = nullptr, *dst_sub = nullptr, *rdiv = nullptr, *negs = nullptr;  // reading C21
};
bool conv_fused_supported(const ckks_ctx *c);
int launch_conv_fused(ckks_ctx *c, const FusedConv &f, const u64 *const *src, u64 *const *dst, int np);

// ---- packed wire format (ops.cu) ----
// A ciphertext at level l on the wire: polynomial 0 then polynomial 1, each
// the limbs t = 0..l in order, limb t packed as N residues of bits(q_t) bits
// (little-endian bit order within 64-bit words).  off[t] = byte offset of
// limb t in one polynomial, off[l+1] = the polynomial's size.
struct WireLayout {
  int nl = 0;
  unsigned char bits[MAX_MODS];
  u32 off[MAX_MODS + 1];
};
WireLayout wire_layout(const ckks_ctx *c, int level);
// unpack (to_wire false) or pack ncts ciphertexts between wire[i] and ct[i]
// ([2][n_limbs[i]][N] limb-major); ncts <= MAX_CTS.
int ew_wire(ckks_ctx *c, const WireLayout &L, unsigned char *const *wire, u64 *const *ct, const u32 *n_limbs,
            int ncts, bool to_wire);

// ---- element-wise and key-switch launchers (ops.cu / keyswitch.cu) ----
// ---- tensor-core basis conversion (bconv_tc.cu) ----
// src_add_host [ns] / dst_sub_host [nt] (or null): constants added to y_i
// mod b_i before the products / subtracted from the result mod t.
// rdiv_host [2][ns] / negs_host [nt] (or null): overflow removal, y_t += v negs_t
// with v = floor(sum_i floor(y_i R_i / 2^64) / 2^32), R_i = rdiv_host[ns + i] 2^64
// + rdiv_host[i] = floor(2^96 / b_i).
int launch_bconv_tc(ckks_ctx *c, size_t key, const u64 *inv_host, const u64 *tab_host, int ns, int nt,
                    const int *src_mod, const int *dst_mod, const int *dst_pos, const u64 *const *src,
                    u64 *const *dst, int np, const u64 *src_add_host, const u64 *dst_sub_host,
                    const u64 *rdiv_host, const u64 *negs_host);

// the same on a strided view of n_virt coefficients per source / target limb
int launch_bconv_tc_view(ckks_ctx *c, size_t key, const u64 *inv_host, const u64 *tab_host, int ns, int nt,
                         const int *src_mod, const int *dst_mod, const int *dst_pos, const u64 *const *src,
                         u64 *const *dst, int np, u32 n_virt);

// ---- batched ciphertext operations (capi.cu); n <= 128, all at one level ----
int rescale_chunk(ckks_ctx *c, ckks_ct *cts, int n);
// merged: ModDown and rescale in one step (reading C21), output at level - 1
int mul_relin_chunk(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n, bool merged = false);
int automorph_chunk(ckks_ctx *c, const ckks_ct *in, const u64 *g, ckks_ct *out, int n);
int rotate_hoisted_internal(ckks_ctx *c, const ckks_ct *in, int n, const u64 *g, int m, ckks_ct *out);
// the switching key of Galois element g (device), or null when absent
const u64 *galois_key_data(ckks_ctx *c, u64 g);
// giant step of a merged linear level: acc (=/+=) KS accumulator of sigma_g(c1)
// over Q_l P, base0 += sigma_g(c0)
int rotate_accumulate_chunk(ckks_ctx *c, const ckks_ct *in, u64 g, int n, u64 *const *acc, u64 *const *base0,
                            bool accumulate);
int galois_key_for(ckks_ctx *c, u64 g);
// encode.cu: N/2 device slots -> NTT plaintext over q_0..q_level at `scale`
int encode_device_z(ckks_ctx *c, const double2 *z_dev, uint32_t level, double scale, u64 *pt_dev, int *flag_dev);
// the same over q_0..q_level, then p_0..p_{K-1} (pt_dev holds level + 1 + K limbs)
int encode_device_z_ext(ckks_ctx *c, const double2 *z_dev, uint32_t level, double scale, u64 *pt_dev,
                        int *flag_dev);
// signed integer coefficients (host) -> NTT plaintext over q_0..q_level, p_0..p_{K-1}
extern "C" int pt_from_int_ext(ckks_ctx *c, const int64_t *m, uint32_t level, uint64_t *pt);
// boot.cu
void boot_free(ckks_ctx *c);
int boot_ensure_plan(ckks_ctx *c);
int boot_rotation_steps(ckks_ctx *c, std::vector<int> &steps);

// Key switching of np <= 128 NTT-domain polynomials at `level`, one key per
// polynomial: o_c = base_c + u_c (base may be null) with u0 + u1 s ~ d s'.
// merged: instead o_c = round((acc_c + P base_c) / (P q_l)) - u over
// q_0..q_{l-1} (reading C21; base required, not read through sigma_g).
// ws: device workspace of ks_ws_words(level, np) words.
size_t ks_ws_words(const ckks_ctx *c, int level, int np);
size_t ks_modup_words(const ckks_ctx *c, int level, int np);
size_t ks_tail_words(const ckks_ctx *c, int level, int nv);
int ks_modup(ckks_ctx *c, int level, int np, const u64 *const *d, u64 *ws, u64 **ext_out);
int ks_tail(ckks_ctx *c, int level, int nv, const u64 *const *d, const u64 *const *ext_digits,
            const u64 *const *keys, const u32 *gal, const u64 *const *base0, const u32 *base0_gal,
            const u64 *const *base1, u64 *const *o0, u64 *const *o1, u64 *ws, bool merged = false);
int ks_batch(ckks_ctx *c, int level, int np, const u64 *const *d, const u64 *const *keys,
             const u64 *const *base0, const u64 *const *base1, u64 *const *o0, u64 *const *o1,
             u64 *ws, bool merged = false);
// The key inner product alone: acc[i] ([2][level+1+K][N], NTT domain) = or +=
// sum_j sigma_gal_i(ModUp_j(d_i)) key_j_i, from ks_modup's digits (gal null:
// no automorphism); with pbase0, poly 0's q-limbs also get [P]_{q_t}
// sigma_gal_i(pbase0_i)[t] (the P sigma(c0) of a rotation kept over Q P).
int ks_accumulate(ckks_ctx *c, int level, int nv, const u64 *const *d, const u64 *const *ext_digits,
                  const u64 *const *keys, const u32 *gal, u64 *const *acc, bool accumulate,
                  const u64 *const *pbase0 = nullptr);
// Merged ModDown and rescale (reading C21) of caller-built sums acc + P base:
// o_c = round((acc_c + P base_c) / (P q_l)) - u.  acc is overwritten (its top
// and special limbs); ws: ks_merged_words(level, nv) words.
size_t ks_merged_words(const ckks_ctx *c, int level, int nv);
// C9 ModDown of caller-built accumulators acc ([2][level+1+K][N], NTT
// domain; the special limbs are consumed): o_c = (acc_c[Q] - z_c) P^-1.
// ws: 2 (level + 1) N words per accumulator.
int ks_moddown_finish(ckks_ctx *c, int level, int nv, u64 *const *acc, u64 *const *o0, u64 *const *o1, u64 *ws);
int ks_merged_finish(ckks_ctx *c, int level, int nv, u64 *const *acc, const u64 *const *base0,
                     const u64 *const *base1, u64 *const *o0, u64 *const *o1, u64 *ws);
