// Launch arguments of the element-wise kernels (ops.cu).
#pragma once

#include "ctx.h"

#define MAX_CTS 128  // ciphertexts per element-wise launch

// Per-ciphertext pointers to poly 0 / poly 1 of inputs x, y and output o.
struct EwArgs {
  const ModInfo *mods;
  u32 n;
  const u64 *x0[MAX_CTS], *x1[MAX_CTS];
  const u64 *y0[MAX_CTS], *y1[MAX_CTS];
  u64 *o0[MAX_CTS], *o1[MAX_CTS];
};

struct RescaleArgs {
  const ModInfo *mods;
  u32 n;
  int level;                         // level being dropped (q_level)
  const u64 *qlinv;                  // [level] Shoup pairs of q_level^-1 mod q_i
  u64 *c0[MAX_CTS], *c1[MAX_CTS];    // ciphertext polys (NTT domain), in place
  const u64 *last[MAX_CTS];          // [2][N] coefficient-domain top limbs
  u64 *lift[MAX_CTS];                // [2][level][N] scratch
};

struct EncArgs {
  const ModInfo *mods;
  u32 n;
  const u64 *s_ntt;
  u64 key_a[MAX_CTS];
  const u64 *pt[MAX_CTS];
  const u64 *err[MAX_CTS];
  u64 *c0[MAX_CTS], *c1[MAX_CTS];
};

// public-key encryption (C5, pk form): c0 = v b + pt + e0, c1 = v a + e1
struct EncPkArgs {
  const ModInfo *mods;
  u32 n;
  const u64 *b, *a;                  // the public key's limbs q_0..
  const u64 *v, *e0, *e1;            // NTT-domain mask and errors [nl][N]
  const u64 *pt;
  u64 *c0, *c1;
};

struct KeyArgs {
  const ModInfo *mods;
  u32 n;
  const u64 *s_ntt;
  const u64 *sp_ntt;                 // s' over all n_q + n_p limbs
  const u64 *err;                    // NTT-domain error over all limbs
  u64 key_a;
  int lo, hi;                        // q-limbs of this digit
  u64 p_mod[MAX_MODS];               // [P]_{q_t}
  u64 *b, *a;                        // outputs [n_q + n_p][N]
};

int ew_addsub(ckks_ctx *c, EwArgs &a, int nl, int ncts, bool sub);
int ew_plain(ckks_ctx *c, EwArgs &a, int nl, int ncts, int mode);  // 0 mul, 1 add
int ew_mul_int(ckks_ctx *c, EwArgs &a, int nl, int ncts, i64 k);
int ew_tensor(ckks_ctx *c, EwArgs &a, u64 *const *d2, int nl, int ncts);
// g[i]: Galois element applied to ciphertext i
int ew_automorph(ckks_ctx *c, EwArgs &a, const u32 *g, int nl, int ncts, bool both_polys);
int ew_decrypt(ckks_ctx *c, EwArgs &a, int nl, int ncts);
int ew_rescale_lift(ckks_ctx *c, RescaleArgs &r, int ncts);
int ew_rescale_finish(ckks_ctx *c, RescaleArgs &r, int ncts);
int ew_encrypt(ckks_ctx *c, EncArgs &e, int nl, int ncts);
int ew_encrypt_pk(ckks_ctx *c, EncPkArgs &e, int nl);
int ew_signed_to_res(ckks_ctx *c, const i64 *v, u64 *out, int first_mod, int nl);
int ew_keyrow(ckks_ctx *c, KeyArgs &k, int nl);
int ew_square(ckks_ctx *c, u64 *out, const u64 *in, int nl);
