/*
 * Plain CPU oracle for RNS-CKKS.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the bench
 * may load this code.  It shares nothing with the CUDA library: primes, roots,
 * transforms, basis conversion, key switching, rescale and automorphisms are
 * all re-derived here from their textbook definitions, as slowly and plainly
 * as possible (every modular product is a 128-bit product followed by `%`).
 *
 * What the paper fixes (ReBoot, Sec. 3): the parameter set {N, q, Delta}, that
 * a multiplication costs one level, dropping the top prime of the modulus
 * chain, batching of N/2 complex slots through the canonical embedding,
 * element-wise +, -, x on slots (Eq. add/sub/mult), left rotation Rot(a, k)
 * with one key per k, and bootstrapping (Sec. 3, last paragraph).  Everything
 * inside the scheme is a reading of the textbook RNS-CKKS definitions; each
 * reading is named in a comment where it is used:
 *   C1 primes, C2 roots and transform order, C4 seeded randomness,
 *   C5 encryption (secret- and public-key forms), C6 tensor/relinearisation, C7 hybrid key-switch gadget,
 *   C8 ModUp, C9 ModDown, C10 rescale, C11 automorphisms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

#define OC_MAXMOD 96

/* ------------------------------------------------------------------ */
/* Modular arithmetic: plain 128-bit products and remainders.          */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - (b % q)) % q); }
static u64 powmod(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
    e >>= 1;
  }
  return r;
}
/* q is prime everywhere this is used: Fermat inverse. */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }
/* signed integer -> residue in [0, q) */
static u64 smod(i64 v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 m = ((u64)(-(v + 1)) % q + 1) % q; /* |v| mod q without overflow */
  return m ? q - m : 0;
}

/* Miller-Rabin with the first twelve prime bases: deterministic below 2^64. */
static int is_prime_u64(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n % bases[i] == 0) return n == bases[i];
  }
  u64 d = n - 1;
  int r = 0;
  while ((d & 1) == 0) { d >>= 1; r++; }
  for (int i = 0; i < 12; i++) {
    u64 x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int witness = 1;
    for (int k = 1; k < r; k++) {
      x = mulmod(x, x, n);
      if (x == n - 1) { witness = 0; break; }
    }
    if (witness) return 0;
  }
  return 1;
}

static u64 bitrev(u64 x, int bits) {
  u64 r = 0;
  for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

/* ------------------------------------------------------------------ */
/* C4: counter-based SplitMix64 (Steele, Lea, Flood 2014).             */
/* draw(key, c) is output number c+1 of SplitMix64 started at `key`.   */
/* ------------------------------------------------------------------ */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL
static u64 sm_mix(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static u64 sm_draw(u64 key, u64 c) { return sm_mix(key + (c + 1) * SM_GAMMA); }
static u64 sm_stream(u64 seed, u64 tag, u64 idx) { return sm_draw(sm_draw(seed, tag), idx); }

enum { TAG_SECRET = 1, TAG_KEY_A = 2, TAG_KEY_E = 3, TAG_ENC_A = 4, TAG_ENC_E = 5,
       TAG_PK_A = 6, TAG_PK_E = 7, TAG_PKENC_V = 8, TAG_PKENC_E0 = 9, TAG_PKENC_E1 = 10 };

u64 oc_splitmix_draw(u64 key, u64 c) { return sm_draw(key, c); }

/* Rounded Gaussian (Box-Muller, cosine branch), tail-cut at |e| <= bound,
 * up to 16 tries per sample, then 0. */
static i64 gauss_sample(u64 key, u64 j, double sigma, i64 bound) {
  for (u64 k = 0; k < 16; k++) {
    u64 c = 2 * (j * 16 + k);
    double u1 = (double)((sm_draw(key, c) >> 11) + 1) * 0x1p-53;
    double u2 = (double)(sm_draw(key, c + 1) >> 11) * 0x1p-53;
    double g = sigma * sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    i64 e = (i64)llround(g);
    if (e >= -bound && e <= bound) return e;
  }
  return 0;
}

/* uniform residue mod q from two 64-bit words: (hi * 2^64 + lo) mod q */
static u64 uniform_mod(u64 key, u64 idx, u64 q) {
  u128 x = ((u128)sm_draw(key, 2 * idx) << 64) | (u128)sm_draw(key, 2 * idx + 1);
  return (u64)(x % q);
}

/* ------------------------------------------------------------------ */
/* Context                                                             */
/* ------------------------------------------------------------------ */
typedef struct okey {
  u64 galois;  /* 0 = relinearisation key (s^2 -> s), else Galois element g */
  u64 *data;   /* [n_digits][2][n_q + n_p][N]: (b_j, a_j), NTT domain      */
  struct okey *next;
} okey;

typedef struct {
  int log_n;
  u64 n;
  int n_q, n_p, dnum, alpha, n_digits;
  int h;
  double sigma;
  i64 e_bound;
  u64 mod[OC_MAXMOD]; /* q_0..q_{n_q-1}, p_0..p_{n_p-1} */
  u64 psi[OC_MAXMOD]; /* primitive 2N-th root per modulus */
  int have_secret;
  i64 *s_coeff;       /* [N] ternary secret */
  u64 *s_ntt;         /* [n_q + n_p][N] */
  u64 key_seed;
  okey *keys;
  u64 *pk;            /* [2][n_q][N] public key (b, a), NTT domain, or NULL */
} oc_ctx;

/* C1: for each bit size b scan t = 2^b + 1 - m * 2^e, m = 1, 2, ..., with
 * e = max(17, log2(2N)) (2N divides q - 1, so the 2N-th roots exist), keep
 * primes; the chain q_0..q_{n_q-1}, p_0..p_{n_p-1} takes, in order, the next
 * unused prime of its bit size.  Returns 0 or -1. */
int oc_gen_primes(int count, const unsigned *bits, int log_step, u64 *out) {
  u64 next_m[64];
  if (log_step < 17 || log_step > 40) return -1;
  for (int b = 0; b < 64; b++) next_m[b] = 1;
  for (int i = 0; i < count; i++) {
    unsigned b = bits[i];
    if (b < 20 || b > 62) return -1;
    for (;;) {
      u64 m = next_m[b]++;
      u64 step = m << log_step;
      if (step >= ((u64)1 << b)) return -1;
      u64 t = ((u64)1 << b) + 1 - step;
      if (is_prime_u64(t)) { out[i] = t; break; }
    }
  }
  return 0;
}

/* C2: g = smallest integer >= 2 that is a quadratic non-residue mod q;
 * psi = g^((q-1)/2N) is then a primitive 2N-th root of unity. */
u64 oc_find_psi(u64 q, u64 n) {
  u64 g = 2;
  while (powmod(g, (q - 1) / 2, q) != q - 1) g++;
  return powmod(g, (q - 1) / (2 * n), q);
}

oc_ctx *oc_create(int log_n, int n_q, int n_p, int dnum, const unsigned *q_bits,
                  const unsigned *p_bits, int h, double sigma) {
  if (log_n < 2 || log_n > 17 || n_q < 1 || n_p < 1 || dnum < 1 || n_q + n_p > OC_MAXMOD)
    return NULL;
  oc_ctx *c = (oc_ctx *)calloc(1, sizeof(oc_ctx));
  c->log_n = log_n;
  c->n = (u64)1 << log_n;
  c->n_q = n_q;
  c->n_p = n_p;
  c->dnum = dnum;
  c->alpha = (n_q + dnum - 1) / dnum;
  c->n_digits = (n_q + c->alpha - 1) / c->alpha;
  c->h = h;
  c->sigma = sigma;
  c->e_bound = (i64)floor(6.0 * sigma);
  unsigned bits[OC_MAXMOD];
  for (int i = 0; i < n_q; i++) bits[i] = q_bits[i];
  for (int i = 0; i < n_p; i++) bits[n_q + i] = p_bits[i];
  if (oc_gen_primes(n_q + n_p, bits, log_n + 1 > 17 ? log_n + 1 : 17, c->mod) != 0) { free(c); return NULL; }
  for (int i = 0; i < n_q + n_p; i++) c->psi[i] = oc_find_psi(c->mod[i], c->n);
  return c;
}

void oc_destroy(oc_ctx *c) {
  if (!c) return;
  okey *k = c->keys;
  while (k) { okey *nx = k->next; free(k->data); free(k); k = nx; }
  free(c->s_coeff);
  free(c->s_ntt);
  free(c->pk);
  free(c);
}

int oc_n_digits(const oc_ctx *c) { return c->n_digits; }
int oc_alpha(const oc_ctx *c) { return c->alpha; }
void oc_moduli(const oc_ctx *c, u64 *out) { memcpy(out, c->mod, sizeof(u64) * (c->n_q + c->n_p)); }
void oc_psis(const oc_ctx *c, u64 *out) { memcpy(out, c->psi, sizeof(u64) * (c->n_q + c->n_p)); }

/* ------------------------------------------------------------------ */
/* C2: negacyclic transform.  Canonical NTT-domain order:              */
/*   A[j] = a(psi^(2*brv(j)+1)) mod q, brv over log2 N bits.           */
/* Computed as twist (b_k = a_k psi^k), a textbook cyclic radix-2 DFT   */
/* with omega = psi^2 (B[i] = a(psi^(2i+1))), then A[j] = B[brv(j)].    */
/* ------------------------------------------------------------------ */
static void cyclic_dft(u64 *b, u64 n, int log_n, u64 omega, u64 q) {
  for (u64 i = 0; i < n; i++) {
    u64 r = bitrev(i, log_n);
    if (i < r) { u64 t = b[i]; b[i] = b[r]; b[r] = t; }
  }
  for (u64 len = 2; len <= n; len <<= 1) {
    u64 wl = powmod(omega, n / len, q);
    for (u64 st = 0; st < n; st += len) {
      u64 w = 1;
      for (u64 j = 0; j < len / 2; j++) {
        u64 u = b[st + j];
        u64 v = mulmod(b[st + j + len / 2], w, q);
        b[st + j] = addmod(u, v, q);
        b[st + j + len / 2] = submod(u, v, q);
        w = mulmod(w, wl, q);
      }
    }
  }
}

static void ntt_one(const oc_ctx *c, int mi, u64 *a) {
  u64 n = c->n, q = c->mod[mi], psi = c->psi[mi];
  u64 *b = (u64 *)malloc(sizeof(u64) * n);
  u64 pk = 1;
  for (u64 k = 0; k < n; k++) { b[k] = mulmod(a[k] % q, pk, q); pk = mulmod(pk, psi, q); }
  cyclic_dft(b, n, c->log_n, mulmod(psi, psi, q), q);
  for (u64 j = 0; j < n; j++) a[j] = b[bitrev(j, c->log_n)];
  free(b);
}

static void intt_one(const oc_ctx *c, int mi, u64 *a) {
  u64 n = c->n, q = c->mod[mi], psi_inv = invmod(c->psi[mi], q);
  u64 *b = (u64 *)malloc(sizeof(u64) * n);
  for (u64 i = 0; i < n; i++) b[i] = a[bitrev(i, c->log_n)] % q;
  cyclic_dft(b, n, c->log_n, mulmod(psi_inv, psi_inv, q), q);
  u64 ninv = invmod(n % q, q), pk = 1;
  for (u64 k = 0; k < n; k++) { a[k] = mulmod(mulmod(b[k], ninv, q), pk, q); pk = mulmod(pk, psi_inv, q); }
  free(b);
}

/* limb l of `a` uses modulus mods[l] */
void oc_ntt(const oc_ctx *c, u64 *a, int n_limbs, const int *mods) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < n_limbs; l++) ntt_one(c, mods[l], a + (u64)l * c->n);
}
void oc_intt(const oc_ctx *c, u64 *a, int n_limbs, const int *mods) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < n_limbs; l++) intt_one(c, mods[l], a + (u64)l * c->n);
}

/* O(N^2) definition of the transform: A[j] = sum_k a_k psi^((2 brv(j)+1) k). */
void oc_ntt_direct(const oc_ctx *c, int mi, const u64 *a, u64 *out) {
  u64 n = c->n, q = c->mod[mi];
  for (u64 j = 0; j < n; j++) {
    u64 x = powmod(c->psi[mi], 2 * bitrev(j, c->log_n) + 1, q), xp = 1, acc = 0;
    for (u64 k = 0; k < n; k++) { acc = addmod(acc, mulmod(a[k] % q, xp, q), q); xp = mulmod(xp, x, q); }
    out[j] = acc;
  }
}

/* Schoolbook product in Z_q[X]/(X^N + 1). */
void oc_negacyclic_schoolbook(const oc_ctx *c, int mi, const u64 *a, const u64 *b, u64 *out) {
  u64 n = c->n, q = c->mod[mi];
  for (u64 i = 0; i < n; i++) out[i] = 0;
  for (u64 i = 0; i < n; i++)
    for (u64 j = 0; j < n; j++) {
      u64 p = mulmod(a[i], b[j], q);
      u64 k = i + j;
      if (k < n) out[k] = addmod(out[k], p, q);
      else out[k - n] = submod(out[k - n], p, q);
    }
}

/* ------------------------------------------------------------------ */
/* Limb helpers.  A polynomial over "basis" = list of modulus indices. */
/* ------------------------------------------------------------------ */
static void q_basis(int n_limbs, int *mods) { for (int i = 0; i < n_limbs; i++) mods[i] = i; }

/* signed integer coefficients -> residues (coefficient domain) */
static void from_signed(const oc_ctx *c, const i64 *v, int n_limbs, const int *mods, u64 *out) {
  for (int l = 0; l < n_limbs; l++)
    for (u64 k = 0; k < c->n; k++) out[(u64)l * c->n + k] = smod(v[k], c->mod[mods[l]]);
}

/* C11: sigma_g on signed coefficients: X^i -> X^(i g mod 2N). */
static void automorph_signed(const oc_ctx *c, const i64 *in, u64 g, i64 *out) {
  u64 n = c->n;
  for (u64 i = 0; i < n; i++) {
    u64 e = (i * g) % (2 * n);
    if (e < n) out[e] = in[i];
    else out[e - n] = -in[i];
  }
}

/* sigma_g on residues (coefficient domain), one limb */
static void automorph_limb(const oc_ctx *c, const u64 *in, u64 g, u64 q, u64 *out) {
  u64 n = c->n;
  for (u64 i = 0; i < n; i++) {
    u64 e = (i * g) % (2 * n);
    if (e < n) out[e] = in[i];
    else out[e - n] = (q - in[i]) % q;
  }
}

/* ------------------------------------------------------------------ */
/* C4/C7: secret and key generation                                    */
/* ------------------------------------------------------------------ */
static void sample_secret(const oc_ctx *c, u64 seed, i64 *s) {
  u64 n = c->n, key = sm_stream(seed, TAG_SECRET, 0);
  u64 *perm = (u64 *)malloc(sizeof(u64) * n);
  for (u64 i = 0; i < n; i++) { perm[i] = i; s[i] = 0; }
  for (u64 i = 0; i < (u64)c->h; i++) {
    u64 r = sm_draw(key, i) % (n - i);
    u64 t = perm[i]; perm[i] = perm[i + r]; perm[i + r] = t;
    s[perm[i]] = (sm_draw(key, (u64)c->h + i) & 1) ? -1 : 1;
  }
  free(perm);
}

/* Build one switching key from s' (given as NTT-domain residues over all
 * n_q + n_p moduli) to s.  C7: digit j = q-primes [j*alpha, min((j+1)*alpha, n_q));
 * b_j = -a_j s + e_j + P * g_j * s' with g_j = Qhat_j [Qhat_j^-1]_{Q_j}, which is
 * 1 mod every prime of digit j and 0 mod every other q-prime; P = 0 mod p. */
static okey *make_key(oc_ctx *c, u64 galois, const u64 *sp_ntt) {
  int ext = c->n_q + c->n_p;
  u64 n = c->n;
  okey *k = (okey *)calloc(1, sizeof(okey));
  k->galois = galois;
  k->data = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * 2 * ext * n);
  int mods[OC_MAXMOD];
  for (int i = 0; i < ext; i++) mods[i] = i;
  u64 key_id = galois;
  i64 *e = (i64 *)malloc(sizeof(i64) * n);
  u64 *e_res = (u64 *)malloc(sizeof(u64) * (u64)ext * n);
  for (int j = 0; j < c->n_digits; j++) {
    u64 ka = sm_stream(c->key_seed, TAG_KEY_A, key_id * 256 + (u64)j);
    u64 ke = sm_stream(c->key_seed, TAG_KEY_E, key_id * 256 + (u64)j);
    for (u64 x = 0; x < n; x++) e[x] = gauss_sample(ke, x, c->sigma, c->e_bound);
    from_signed(c, e, ext, mods, e_res);
    oc_ntt(c, e_res, ext, mods);
    u64 *bj = k->data + ((u64)j * 2 + 0) * ext * n;
    u64 *aj = k->data + ((u64)j * 2 + 1) * ext * n;
    int lo = j * c->alpha, hi = (j + 1) * c->alpha < c->n_q ? (j + 1) * c->alpha : c->n_q;
    for (int t = 0; t < ext; t++) {
      u64 q = c->mod[t];
      u64 p_mod_q = 1 % q;
      for (int pi = 0; pi < c->n_p; pi++) p_mod_q = mulmod(p_mod_q, c->mod[c->n_q + pi], q);
      int in_digit = (t >= lo && t < hi);
      for (u64 x = 0; x < n; x++) {
        u64 idx = (u64)t * n + x;
        u64 a = uniform_mod(ka, idx, q);
        u64 v = submod(e_res[idx], mulmod(a, c->s_ntt[idx], q), q);
        if (in_digit) v = addmod(v, mulmod(p_mod_q, sp_ntt[idx], q), q);
        aj[idx] = a;
        bj[idx] = v;
      }
    }
  }
  free(e);
  free(e_res);
  k->next = c->keys;
  c->keys = k;
  return k;
}

static okey *find_key(const oc_ctx *c, u64 galois) {
  for (okey *k = c->keys; k; k = k->next)
    if (k->galois == galois) return k;
  return NULL;
}

/* Draw s from `seed` and build the relinearisation key (s^2 -> s). */
int oc_keygen(oc_ctx *c, u64 seed) {
  int ext = c->n_q + c->n_p;
  u64 n = c->n;
  okey *k = c->keys;
  while (k) { okey *nx = k->next; free(k->data); free(k); k = nx; }
  c->keys = NULL;
  free(c->s_coeff);
  free(c->s_ntt);
  free(c->pk);
  c->pk = NULL;
  c->key_seed = seed;
  c->s_coeff = (i64 *)malloc(sizeof(i64) * n);
  c->s_ntt = (u64 *)malloc(sizeof(u64) * (u64)ext * n);
  sample_secret(c, seed, c->s_coeff);
  int mods[OC_MAXMOD];
  for (int i = 0; i < ext; i++) mods[i] = i;
  from_signed(c, c->s_coeff, ext, mods, c->s_ntt);
  oc_ntt(c, c->s_ntt, ext, mods);
  c->have_secret = 1;
  u64 *s2 = (u64 *)malloc(sizeof(u64) * (u64)ext * n);
  for (int t = 0; t < ext; t++)
    for (u64 x = 0; x < n; x++) {
      u64 idx = (u64)t * n + x;
      s2[idx] = mulmod(c->s_ntt[idx], c->s_ntt[idx], c->mod[t]);
    }
  make_key(c, 0, s2);
  free(s2);
  return 0;
}

/* Galois key for element g (odd, < 2N): s' = sigma_g(s). */
int oc_gen_galois_key(oc_ctx *c, u64 g) {
  if (!c->have_secret || (g & 1) == 0 || g >= 2 * c->n) return -1;
  if (find_key(c, g)) return 0;
  int ext = c->n_q + c->n_p;
  u64 n = c->n;
  i64 *sg = (i64 *)malloc(sizeof(i64) * n);
  automorph_signed(c, c->s_coeff, g, sg);
  u64 *sp = (u64 *)malloc(sizeof(u64) * (u64)ext * n);
  int mods[OC_MAXMOD];
  for (int i = 0; i < ext; i++) mods[i] = i;
  from_signed(c, sg, ext, mods, sp);
  oc_ntt(c, sp, ext, mods);
  make_key(c, g, sp);
  free(sg);
  free(sp);
  return 0;
}

void oc_secret(const oc_ctx *c, i64 *out) { memcpy(out, c->s_coeff, sizeof(i64) * c->n); }

/* copy a key out: [n_digits][2][n_q+n_p][N] */
int oc_key_data(const oc_ctx *c, u64 galois, u64 *out) {
  okey *k = find_key(c, galois);
  if (!k) return -1;
  memcpy(out, k->data, sizeof(u64) * (u64)c->n_digits * 2 * (c->n_q + c->n_p) * c->n);
  return 0;
}

/* Rotation by k slots to the left (C11): g = 5^(k mod N/2) mod 2N. */
u64 oc_galois_elt(const oc_ctx *c, i64 k) {
  i64 half = (i64)(c->n / 2);
  i64 r = ((k % half) + half) % half;
  return powmod(5, (u64)r, 2 * c->n);
}

/* ------------------------------------------------------------------ */
/* Plaintexts, encryption, decryption (C5)                             */
/* ------------------------------------------------------------------ */
/* signed integer coefficients m -> NTT-domain residues over q_0..q_level */
void oc_pt_from_signed(const oc_ctx *c, const i64 *m, int level, u64 *pt) {
  int mods[OC_MAXMOD];
  q_basis(level + 1, mods);
  from_signed(c, m, level + 1, mods, pt);
  oc_ntt(c, pt, level + 1, mods);
}

/* Secret-key encryption (Sec. 3: "encrypted using the secret key"):
 * ct = ([-a s + m + e]_Q, a), a uniform (drawn in the NTT domain), e Gaussian. */
int oc_encrypt(const oc_ctx *c, const u64 *pt, int level, u64 enc_seed, u64 *ct) {
  if (!c->have_secret || level < 0 || level >= c->n_q) return -1;
  u64 n = c->n;
  int nl = level + 1;
  u64 ka = sm_stream(enc_seed, TAG_ENC_A, 0), ke = sm_stream(enc_seed, TAG_ENC_E, 0);
  i64 *e = (i64 *)malloc(sizeof(i64) * n);
  for (u64 x = 0; x < n; x++) e[x] = gauss_sample(ke, x, c->sigma, c->e_bound);
  u64 *er = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  int mods[OC_MAXMOD];
  q_basis(nl, mods);
  from_signed(c, e, nl, mods, er);
  oc_ntt(c, er, nl, mods);
  u64 *c0 = ct, *c1 = ct + (u64)nl * n;
  for (int t = 0; t < nl; t++) {
    u64 q = c->mod[t];
    for (u64 x = 0; x < n; x++) {
      u64 idx = (u64)t * n + x;
      u64 a = uniform_mod(ka, idx, q);
      c1[idx] = a;
      c0[idx] = submod(addmod(pt[idx], er[idx], q), mulmod(a, c->s_ntt[idx], q), q);
    }
  }
  free(e);
  free(er);
  return 0;
}

/* the error polynomial that oc_encrypt adds for enc_seed (signed) */
void oc_enc_error(const oc_ctx *c, u64 enc_seed, i64 *e) {
  u64 ke = sm_stream(enc_seed, TAG_ENC_E, 0);
  for (u64 x = 0; x < c->n; x++) e[x] = gauss_sample(ke, x, c->sigma, c->e_bound);
}

/* Public key (C5, pk form; Sec. 3 writes encryption as E(pk, .)): the
 * secret-key encryption of 0 at the top level, drawn from the key seed's own
 * streams: pk = ([-a s + e]_Q, a) over q_0..q_{n_q-1}. */
int oc_gen_public_key(oc_ctx *c) {
  if (!c->have_secret) return -1;
  u64 n = c->n;
  int nl = c->n_q;
  u64 *pk = (u64 *)malloc(sizeof(u64) * 2 * (u64)nl * n);
  u64 ka = sm_stream(c->key_seed, TAG_PK_A, 0), ke = sm_stream(c->key_seed, TAG_PK_E, 0);
  i64 *e = (i64 *)malloc(sizeof(i64) * n);
  for (u64 x = 0; x < n; x++) e[x] = gauss_sample(ke, x, c->sigma, c->e_bound);
  u64 *er = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  int mods[OC_MAXMOD];
  q_basis(nl, mods);
  from_signed(c, e, nl, mods, er);
  oc_ntt(c, er, nl, mods);
  u64 *b = pk, *a = pk + (u64)nl * n;
  for (int t = 0; t < nl; t++) {
    u64 q = c->mod[t];
    for (u64 x = 0; x < n; x++) {
      u64 idx = (u64)t * n + x;
      u64 av = uniform_mod(ka, idx, q);
      a[idx] = av;
      b[idx] = submod(er[idx], mulmod(av, c->s_ntt[idx], q), q);
    }
  }
  free(e);
  free(er);
  free(c->pk);
  c->pk = pk;
  return 0;
}

int oc_public_key(const oc_ctx *c, u64 *out) {
  if (!c->pk) return -1;
  memcpy(out, c->pk, sizeof(u64) * 2 * (u64)c->n_q * c->n);
  return 0;
}

/* The masking polynomial of public-key encryption: each coefficient 0 with
 * probability 1/2 and +1, -1 with probability 1/4 each, from the low two bits
 * of one draw (0, 1 -> 0; 2 -> +1; 3 -> -1). */
void oc_pk_mask(u64 enc_seed, u64 n, i64 *v) {
  u64 kv = sm_stream(enc_seed, TAG_PKENC_V, 0);
  for (u64 x = 0; x < n; x++) {
    u64 r = sm_draw(kv, x) & 3;
    v[x] = r < 2 ? 0 : (r == 2 ? 1 : -1);
  }
}

/* Public-key encryption (C5, pk form): v the mask above, e0 and e1 Gaussian,
 * ct = ([v b + m + e0]_Q, [v a + e1]_Q) over q_0..q_level, with (b, a) = pk
 * restricted to those primes; the products are negacyclic, taken as
 * point-wise products of NTT-domain residues. */
int oc_encrypt_pk(const oc_ctx *c, const u64 *pt, int level, u64 enc_seed, u64 *ct) {
  if (!c->pk || level < 0 || level >= c->n_q) return -1;
  u64 n = c->n;
  int nl = level + 1;
  int mods[OC_MAXMOD];
  q_basis(nl, mods);
  i64 *w = (i64 *)malloc(sizeof(i64) * n);
  u64 *vr = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *e0r = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *e1r = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  oc_pk_mask(enc_seed, n, w);
  from_signed(c, w, nl, mods, vr);
  oc_ntt(c, vr, nl, mods);
  u64 k0 = sm_stream(enc_seed, TAG_PKENC_E0, 0), k1 = sm_stream(enc_seed, TAG_PKENC_E1, 0);
  for (u64 x = 0; x < n; x++) w[x] = gauss_sample(k0, x, c->sigma, c->e_bound);
  from_signed(c, w, nl, mods, e0r);
  oc_ntt(c, e0r, nl, mods);
  for (u64 x = 0; x < n; x++) w[x] = gauss_sample(k1, x, c->sigma, c->e_bound);
  from_signed(c, w, nl, mods, e1r);
  oc_ntt(c, e1r, nl, mods);
  const u64 *b = c->pk, *a = c->pk + (u64)c->n_q * n;
  u64 *c0 = ct, *c1 = ct + (u64)nl * n;
  for (int t = 0; t < nl; t++) {
    u64 q = c->mod[t];
    for (u64 x = 0; x < n; x++) {
      u64 idx = (u64)t * n + x;
      c0[idx] = addmod(addmod(mulmod(vr[idx], b[idx], q), pt[idx], q), e0r[idx], q);
      c1[idx] = addmod(mulmod(vr[idx], a[idx], q), e1r[idx], q);
    }
  }
  free(w);
  free(vr);
  free(e0r);
  free(e1r);
  return 0;
}

/* m' = c0 + c1 s (NTT domain) over q_0..q_level */
int oc_decrypt(const oc_ctx *c, const u64 *ct, int level, u64 *pt) {
  if (!c->have_secret) return -1;
  u64 n = c->n;
  int nl = level + 1;
  const u64 *c0 = ct, *c1 = ct + (u64)nl * n;
  for (int t = 0; t < nl; t++)
    for (u64 x = 0; x < n; x++) {
      u64 idx = (u64)t * n + x;
      pt[idx] = addmod(c0[idx], mulmod(c1[idx], c->s_ntt[idx], c->mod[t]), c->mod[t]);
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Element-wise operations (Eq. add, sub, mult; plaintext variants)    */
/* ------------------------------------------------------------------ */
void oc_add(const oc_ctx *c, const u64 *a, const u64 *b, int level, u64 *out) {
  u64 n = c->n;
  int nl = level + 1;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < nl; t++)
      for (u64 x = 0; x < n; x++) {
        u64 idx = ((u64)p * nl + t) * n + x;
        out[idx] = addmod(a[idx], b[idx], c->mod[t]);
      }
}
void oc_sub(const oc_ctx *c, const u64 *a, const u64 *b, int level, u64 *out) {
  u64 n = c->n;
  int nl = level + 1;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < nl; t++)
      for (u64 x = 0; x < n; x++) {
        u64 idx = ((u64)p * nl + t) * n + x;
        out[idx] = submod(a[idx], b[idx], c->mod[t]);
      }
}
/* (c0, c1) * pt */
void oc_mul_plain(const oc_ctx *c, const u64 *a, const u64 *pt, int level, u64 *out) {
  u64 n = c->n;
  int nl = level + 1;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < nl; t++)
      for (u64 x = 0; x < n; x++) {
        u64 idx = ((u64)p * nl + t) * n + x;
        out[idx] = mulmod(a[idx], pt[(u64)t * n + x], c->mod[t]);
      }
}
/* (c0 + pt, c1) */
void oc_add_plain(const oc_ctx *c, const u64 *a, const u64 *pt, int level, u64 *out) {
  u64 n = c->n;
  int nl = level + 1;
  memcpy(out, a, sizeof(u64) * 2 * nl * n);
  for (int t = 0; t < nl; t++)
    for (u64 x = 0; x < n; x++) {
      u64 idx = (u64)t * n + x;
      out[idx] = addmod(a[idx], pt[idx], c->mod[t]);
    }
}
/* multiply every coefficient by a signed integer constant (no level used) */
void oc_mul_int(const oc_ctx *c, const u64 *a, i64 k, int level, u64 *out) {
  u64 n = c->n;
  int nl = level + 1;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < nl; t++) {
      u64 kk = smod(k, c->mod[t]);
      for (u64 x = 0; x < n; x++) {
        u64 idx = ((u64)p * nl + t) * n + x;
        out[idx] = mulmod(a[idx], kk, c->mod[t]);
      }
    }
}

/* C6: tensor product d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 (NTT domain) */
void oc_tensor(const oc_ctx *c, const u64 *a, const u64 *b, int level, u64 *d0, u64 *d1, u64 *d2) {
  u64 n = c->n;
  int nl = level + 1;
  const u64 *a0 = a, *a1 = a + (u64)nl * n, *b0 = b, *b1 = b + (u64)nl * n;
  for (int t = 0; t < nl; t++) {
    u64 q = c->mod[t];
    for (u64 x = 0; x < n; x++) {
      u64 i = (u64)t * n + x;
      d0[i] = mulmod(a0[i], b0[i], q);
      d1[i] = addmod(mulmod(a0[i], b1[i], q), mulmod(a1[i], b0[i], q), q);
      d2[i] = mulmod(a1[i], b1[i], q);
    }
  }
}

/* ------------------------------------------------------------------ */
/* C8: fast basis conversion (uncentred).                              */
/*   y_t = sum_{i in src} [x_i * (Bhat_i)^-1]_{b_i} * (Bhat_i mod m_t) mod m_t  */
/* with Bhat_i = prod_{i' in src, i' != i} b_i'.  Coefficient domain.  */
/* ------------------------------------------------------------------ */
void oc_bconv(const oc_ctx *c, const u64 *x, int n_src, const int *src, u64 *y, int n_dst,
              const int *dst) {
  u64 n = c->n;
  u64 bhat_inv[OC_MAXMOD];
  for (int i = 0; i < n_src; i++) {
    u64 bi = c->mod[src[i]], v = 1;
    for (int k = 0; k < n_src; k++)
      if (k != i) v = mulmod(v, c->mod[src[k]] % bi, bi);
    bhat_inv[i] = invmod(v, bi);
  }
#pragma omp parallel for schedule(static)
  for (int t = 0; t < n_dst; t++) {
    u64 mt = c->mod[dst[t]];
    u64 bhat_mod_t[OC_MAXMOD];
    for (int i = 0; i < n_src; i++) {
      u64 v = 1;
      for (int k = 0; k < n_src; k++)
        if (k != i) v = mulmod(v, c->mod[src[k]] % mt, mt);
      bhat_mod_t[i] = v;
    }
    for (u64 k = 0; k < n; k++) {
      u64 acc = 0;
      for (int i = 0; i < n_src; i++) {
        u64 bi = c->mod[src[i]];
        u64 yi = mulmod(x[(u64)i * n + k], bhat_inv[i], bi);
        acc = addmod(acc, mulmod(yi, bhat_mod_t[i], mt), mt);
      }
      y[(u64)t * n + k] = acc;
    }
  }
}

/* ------------------------------------------------------------------ */
/* C7-C9: hybrid key switching.                                        */
/* d: NTT-domain polynomial over q_0..q_level; key: [n_digits][2][n_q+n_p][N].   */
/* out0/out1: NTT domain over q_0..q_level, with out0 + out1 s ~ d s'. */
/* ------------------------------------------------------------------ */
static void ext_basis(const oc_ctx *c, int level, int *ext_mods) {
  for (int t = 0; t <= level; t++) ext_mods[t] = t;
  for (int t = 0; t < c->n_p; t++) ext_mods[level + 1 + t] = c->n_q + t;
}

/* C7/C8 ModUp: digits[j] = NTT-domain lift of digit j of d to q_0..q_level, P;
 * its own limbs are d's, the others come from BConv.  Returns the number of
 * active digits; digits is [n_digits][level+1+n_p][N]. */
static int modup(const oc_ctx *c, const u64 *d, int level, u64 *digits) {
  u64 n = c->n;
  int nl = level + 1, ext = nl + c->n_p, nact = 0;
  int ext_mods[OC_MAXMOD];
  ext_basis(c, level, ext_mods);
  u64 *dc = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  memcpy(dc, d, sizeof(u64) * (u64)nl * n);
  oc_intt(c, dc, nl, ext_mods);
  for (int j = 0; j < c->n_digits; j++) {
    int lo = j * c->alpha, hi = (j + 1) * c->alpha;
    if (hi > nl) hi = nl;
    if (lo >= hi) break;
    u64 *dig = digits + (u64)j * ext * n;
    int src[OC_MAXMOD], dst[OC_MAXMOD], dst_pos[OC_MAXMOD], n_src = hi - lo, n_dst = 0;
    for (int i = lo; i < hi; i++) src[i - lo] = i;
    for (int t = 0; t < ext; t++)
      if (t < lo || t >= hi) { dst[n_dst] = ext_mods[t]; dst_pos[n_dst] = t; n_dst++; }
    u64 *conv = (u64 *)malloc(sizeof(u64) * (u64)n_dst * n);
    oc_bconv(c, dc + (u64)lo * n, n_src, src, conv, n_dst, dst);
    oc_ntt(c, conv, n_dst, dst);
    for (int i = lo; i < hi; i++) memcpy(dig + (u64)i * n, d + (u64)i * n, sizeof(u64) * n);
    for (int k = 0; k < n_dst; k++) memcpy(dig + (u64)dst_pos[k] * n, conv + (u64)k * n, sizeof(u64) * n);
    free(conv);
    nact++;
  }
  free(dc);
  return nact;
}

/* inner product of the lifted digits with evk = (b_j, a_j): acc = [2][ext][N]
 * over q_0..q_level, P (NTT domain) */
static void inner(const oc_ctx *c, const u64 *digits, int nact, int level, const u64 *key, u64 *acc) {
  u64 n = c->n;
  int nl = level + 1, np = c->n_p, ext = nl + np, key_ext = c->n_q + c->n_p;
  int ext_mods[OC_MAXMOD];
  ext_basis(c, level, ext_mods);
  memset(acc, 0, sizeof(u64) * (u64)2 * ext * n);
  for (int j = 0; j < nact; j++) {
    const u64 *dig = digits + (u64)j * ext * n;
    /* key limbs above the level are skipped */
    const u64 *bj = key + ((u64)j * 2 + 0) * key_ext * n;
    const u64 *aj = key + ((u64)j * 2 + 1) * key_ext * n;
    for (int t = 0; t < ext; t++) {
      u64 q = c->mod[ext_mods[t]];
      const u64 *kb = bj + (u64)ext_mods[t] * n, *ka = aj + (u64)ext_mods[t] * n;
      for (u64 x = 0; x < n; x++) {
        u64 v = dig[(u64)t * n + x];
        acc[(u64)t * n + x] = addmod(acc[(u64)t * n + x], mulmod(v, kb[x], q), q);
        acc[((u64)ext + t) * n + x] = addmod(acc[((u64)ext + t) * n + x], mulmod(v, ka[x], q), q);
      }
    }
  }
}

/* inner product, then ModDown (C9) */
static void inner_moddown(const oc_ctx *c, const u64 *digits, int nact, int level, const u64 *key, u64 *out0,
                          u64 *out1) {
  u64 n = c->n;
  int nl = level + 1, np = c->n_p, ext = nl + np;
  u64 *acc = (u64 *)malloc(sizeof(u64) * (u64)2 * ext * n);
  inner(c, digits, nact, level, key, acc);
  /* C9: ModDown, out_i = (x_i - BConv_{P->Q}(x_P)_i) * P^-1 mod q_i */
  int psrc[OC_MAXMOD], qdst[OC_MAXMOD];
  for (int t = 0; t < np; t++) psrc[t] = c->n_q + t;
  for (int t = 0; t < nl; t++) qdst[t] = t;
  u64 *xp = (u64 *)malloc(sizeof(u64) * (u64)np * n);
  u64 *z = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  for (int pol = 0; pol < 2; pol++) {
    u64 *a = acc + (u64)pol * ext * n;
    u64 *out = pol == 0 ? out0 : out1;
    memcpy(xp, a + (u64)nl * n, sizeof(u64) * (u64)np * n);
    oc_intt(c, xp, np, psrc);
    oc_bconv(c, xp, np, psrc, z, nl, qdst);
    oc_ntt(c, z, nl, qdst);
    for (int t = 0; t < nl; t++) {
      u64 q = c->mod[t], pinv = 1;
      for (int pi = 0; pi < np; pi++) pinv = mulmod(pinv, c->mod[c->n_q + pi] % q, q);
      pinv = invmod(pinv, q);
      for (u64 x = 0; x < n; x++) {
        u64 i = (u64)t * n + x;
        out[i] = mulmod(submod(a[i], z[i], q), pinv, q);
      }
    }
  }
  free(xp);
  free(z);
  free(acc);
}

static void keyswitch(const oc_ctx *c, const u64 *d, int level, const u64 *key, u64 *out0, u64 *out1) {
  int ext = level + 1 + c->n_p;
  u64 *digits = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * c->n);
  int nact = modup(c, d, level, digits);
  inner_moddown(c, digits, nact, level, key, out0, out1);
  free(digits);
}

/* sigma_g of NTT-domain limbs: back to coefficients, X^i -> X^(ig), forward again */
static void automorph_ntt_limbs(const oc_ctx *c, const u64 *in, int n_limbs, const int *mods, u64 g, u64 *out) {
  u64 n = c->n;
  u64 *tmp = (u64 *)malloc(sizeof(u64) * (u64)n_limbs * n);
  memcpy(tmp, in, sizeof(u64) * (u64)n_limbs * n);
  oc_intt(c, tmp, n_limbs, mods);
  for (int l = 0; l < n_limbs; l++) automorph_limb(c, tmp + (u64)l * n, g, c->mod[mods[l]], out + (u64)l * n);
  oc_ntt(c, out, n_limbs, mods);
  free(tmp);
}

/* Hoisted rotations (Halevi-Shoup): one ModUp of c1 serves every Galois
 * element g in gs.  For each g the lifted digits are mapped by sigma_g, then
 * inner product with the key of g and ModDown: out_g = (sigma_g(c0) + u0, u1).
 * outs: [n_g][2][level+1][N]. */
int oc_rotate_hoisted(const oc_ctx *c, const u64 *in, int level, int n_g, const u64 *gs, u64 *outs) {
  for (int i = 0; i < n_g; i++)
    if (!find_key(c, gs[i])) return -1;
  u64 n = c->n;
  int nl = level + 1, ext = nl + c->n_p;
  int ext_mods[OC_MAXMOD];
  ext_basis(c, level, ext_mods);
  u64 *digits = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * n);
  u64 *pdig = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * n);
  u64 *u0 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *u1 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *s0 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  int nact = modup(c, in + (u64)nl * n, level, digits);
  for (int i = 0; i < n_g; i++) {
    for (int j = 0; j < nact; j++)
      automorph_ntt_limbs(c, digits + (u64)j * ext * n, ext, ext_mods, gs[i], pdig + (u64)j * ext * n);
    inner_moddown(c, pdig, nact, level, find_key(c, gs[i])->data, u0, u1);
    automorph_ntt_limbs(c, in, nl, ext_mods, gs[i], s0);
    u64 *o = outs + (u64)i * 2 * nl * n;
    for (int t = 0; t < nl; t++)
      for (u64 x = 0; x < n; x++) {
        u64 k = (u64)t * n + x;
        o[k] = addmod(s0[k], u0[k], c->mod[t]);
        o[(u64)nl * n + k] = u1[k];
      }
  }
  free(digits);
  free(pdig);
  free(u0);
  free(u1);
  free(s0);
  return 0;
}

/* Hoisted rotations stopped before ModDown (the baby steps of reading B11):
 * out_g = (P sigma_g(c0) + acc0, acc1) over q_0..q_level, P, with acc the key
 * inner product of the sigma_g-mapped digits of ModUp(c1).
 * outs: [n_g][2][level+1+K][N]. */
int oc_rotate_hoisted_ext(const oc_ctx *c, const u64 *in, int level, int n_g, const u64 *gs, u64 *outs) {
  for (int i = 0; i < n_g; i++)
    if (!find_key(c, gs[i])) return -1;
  u64 n = c->n;
  int nl = level + 1, ext = nl + c->n_p;
  int ext_mods[OC_MAXMOD];
  ext_basis(c, level, ext_mods);
  u64 *digits = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * n);
  u64 *pdig = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * n);
  u64 *s0 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  int nact = modup(c, in + (u64)nl * n, level, digits);
  for (int i = 0; i < n_g; i++) {
    for (int j = 0; j < nact; j++)
      automorph_ntt_limbs(c, digits + (u64)j * ext * n, ext, ext_mods, gs[i], pdig + (u64)j * ext * n);
    u64 *o = outs + (u64)i * 2 * ext * n;
    inner(c, pdig, nact, level, find_key(c, gs[i])->data, o);
    automorph_ntt_limbs(c, in, nl, ext_mods, gs[i], s0);
    for (int t = 0; t < nl; t++) {
      u64 q = c->mod[t], pm = 1;
      for (int k = 0; k < c->n_p; k++) pm = mulmod(pm, c->mod[c->n_q + k] % q, q);
      for (u64 x = 0; x < n; x++) o[(u64)t * n + x] = addmod(o[(u64)t * n + x], mulmod(pm, s0[(u64)t * n + x], q), q);
    }
  }
  free(digits);
  free(pdig);
  free(s0);
  return 0;
}

/* C9 ModDown of one polynomial x over q_0..q_level, P (NTT domain):
 * out = (x_Q - BConv_{P->Q}(x_P)) * P^-1 over q_0..q_level. */
int oc_moddown(const oc_ctx *c, const u64 *x, int level, u64 *out) {
  u64 n = c->n;
  int nl = level + 1, np = c->n_p;
  int psrc[OC_MAXMOD], qdst[OC_MAXMOD];
  for (int t = 0; t < np; t++) psrc[t] = c->n_q + t;
  for (int t = 0; t < nl; t++) qdst[t] = t;
  u64 *xp = (u64 *)malloc(sizeof(u64) * (u64)np * n);
  u64 *z = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  memcpy(xp, x + (u64)nl * n, sizeof(u64) * (u64)np * n);
  oc_intt(c, xp, np, psrc);
  oc_bconv(c, xp, np, psrc, z, nl, qdst);
  oc_ntt(c, z, nl, qdst);
  for (int t = 0; t < nl; t++) {
    u64 q = c->mod[t], pinv = 1;
    for (int pi = 0; pi < np; pi++) pinv = mulmod(pinv, c->mod[c->n_q + pi] % q, q);
    pinv = invmod(pinv, q);
    for (u64 k = 0; k < n; k++) {
      u64 i = (u64)t * n + k;
      out[i] = mulmod(submod(x[i], z[i], q), pinv, q);
    }
  }
  free(xp);
  free(z);
  return 0;
}

/* out[t][k] = x[t][k] * y[t][k] mod m_t */
void oc_mul_elem(const oc_ctx *c, const u64 *x, const u64 *y, int n_limbs, const int *mods, u64 *out) {
  for (int t = 0; t < n_limbs; t++) {
    u64 q = c->mod[mods[t]];
    for (u64 k = 0; k < c->n; k++) out[(u64)t * c->n + k] = mulmod(x[(u64)t * c->n + k], y[(u64)t * c->n + k], q);
  }
}

/* expose key switching for tests: galois = 0 selects the relinearisation key */
/* The key switch of d stopped before ModDown: acc = sum_j ModUp_j(d) * key_j
 * over q_0..q_level, P (NTT domain), [2][level+1+K][N]. */
int oc_keyswitch_ext(const oc_ctx *c, const u64 *d, int level, u64 galois, u64 *acc) {
  okey *k = find_key(c, galois);
  if (!k) return -1;
  int ext = level + 1 + c->n_p;
  u64 *digits = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * c->n);
  int nact = modup(c, d, level, digits);
  inner(c, digits, nact, level, k->data, acc);
  free(digits);
  return 0;
}

/* out[t][k] = x[t][k] * w[t] mod m_t: one scalar per limb */
void oc_mul_scalars(const oc_ctx *c, const u64 *x, int n_limbs, const int *mods, const u64 *w, u64 *out) {
  for (int t = 0; t < n_limbs; t++) {
    u64 q = c->mod[mods[t]];
    for (u64 k = 0; k < c->n; k++) out[(u64)t * c->n + k] = mulmod(x[(u64)t * c->n + k], w[t] % q, q);
  }
}

int oc_keyswitch(const oc_ctx *c, const u64 *d, int level, u64 galois, u64 *out0, u64 *out1) {
  okey *k = find_key(c, galois);
  if (!k) return -1;
  keyswitch(c, d, level, k->data, out0, out1);
  return 0;
}

/* C6: relinearised product (d0, d1) + KS_{s^2 -> s}(d2); levels must match. */
int oc_mul_relin(const oc_ctx *c, const u64 *a, const u64 *b, int level, u64 *out) {
  okey *k = find_key(c, 0);
  if (!k) return -1;
  u64 n = c->n;
  int nl = level + 1;
  u64 *d2 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *u0 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *u1 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *o0 = out, *o1 = out + (u64)nl * n;
  oc_tensor(c, a, b, level, o0, o1, d2);
  keyswitch(c, d2, level, k->data, u0, u1);
  for (int t = 0; t < nl; t++)
    for (u64 x = 0; x < n; x++) {
      u64 i = (u64)t * n + x;
      o0[i] = addmod(o0[i], u0[i], c->mod[t]);
      o1[i] = addmod(o1[i], u1[i], c->mod[t]);
    }
  free(d2);
  free(u0);
  free(u1);
  return 0;
}

/* C10: rescale.  c'_i = (c_i - [c_l]_centred mod q_i) * q_l^-1 mod q_i.
 * in: level `level` (level+1 limbs per poly); out: level-1 (level limbs per poly). */
int oc_rescale(const oc_ctx *c, const u64 *in, int level, u64 *out) {
  if (level < 1) return -1;
  u64 n = c->n, ql = c->mod[level];
  int nl = level + 1;
  u64 *last = (u64 *)malloc(sizeof(u64) * n);
  u64 *lift = (u64 *)malloc(sizeof(u64) * n);
  int ml = level;
  for (int pol = 0; pol < 2; pol++) {
    const u64 *src = in + (u64)pol * nl * n;
    u64 *dst = out + (u64)pol * (nl - 1) * n;
    memcpy(last, src + (u64)level * n, sizeof(u64) * n);
    oc_intt(c, last, 1, &ml);
    for (int t = 0; t < level; t++) {
      u64 q = c->mod[t];
      for (u64 x = 0; x < n; x++) {
        i64 v = last[x] > (ql - 1) / 2 ? -(i64)(ql - last[x]) : (i64)last[x];
        lift[x] = smod(v, q);
      }
      oc_ntt(c, lift, 1, &t);
      u64 qinv = invmod(ql % q, q);
      for (u64 x = 0; x < n; x++) {
        u64 i = (u64)t * n + x;
        dst[i] = mulmod(submod(src[i], lift[x], q), qinv, q);
      }
    }
  }
  free(last);
  free(lift);
  return 0;
}

/* Multi-word unsigned integers (little-endian 64-bit words), just enough for
 * the exact division below: a word times a number, sums, comparisons,
 * differences and the remainder by one word. */
static void mw_mul_word(const u64 *a, int w, u64 b, u64 *out) {
  u128 carry = 0;
  for (int i = 0; i < w; i++) {
    u128 t = (u128)a[i] * b + carry;
    out[i] = (u64)t;
    carry = t >> 64;
  }
}
static void mw_add(u64 *acc, const u64 *b, int w) {
  u128 carry = 0;
  for (int i = 0; i < w; i++) {
    u128 t = (u128)acc[i] + b[i] + carry;
    acc[i] = (u64)t;
    carry = t >> 64;
  }
}
static void mw_sub(u64 *acc, const u64 *b, int w) { /* acc >= b */
  u64 borrow = 0;
  for (int i = 0; i < w; i++) {
    u128 t = (u128)acc[i] - b[i] - borrow;
    acc[i] = (u64)t;
    borrow = (u64)(t >> 64) ? 1 : 0;
  }
}
static int mw_cmp(const u64 *a, const u64 *b, int w) {
  for (int i = w - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  return 0;
}
static u64 mw_mod(const u64 *a, int w, u64 q) {
  u128 r = 0;
  for (int i = w - 1; i >= 0; i--) r = ((r << 64) | a[i]) % q;
  return (u64)r;
}

/* C21: ModDown and rescale merged, written as its definition.  x (NTT domain,
 * [ext][N] over q_0..q_l, p_0..p_{K-1}) represents the integer polynomial X
 * with coefficients in [0, Q_l P); the result is round(X / S), S = P q_l,
 * over q_0..q_{l-1}.  Per coefficient: the exact residue V = X mod S by the
 * CRT over the sources {q_l, p_0..p_{K-1}} in multi-word integers
 * (V = sum_i y_i Shat_i minus the multiple of S that brings it below S), its
 * centred form r in (-S/2, S/2) (S is odd: no ties), and then
 *   out_t = (x_t - r) S^-1 mod q_t,
 * which is the integer (X - r) / S = round(X / S) reduced mod q_t.
 * out: [level][N], NTT domain. */
int oc_moddown_rescale(const oc_ctx *c, const u64 *x, int level, u64 *out) {
  if (level < 1) return -1;
  u64 n = c->n;
  int nl = level + 1, np = c->n_p, ns = np + 1, w = ns + 1;
  int src[OC_MAXMOD], dst[OC_MAXMOD];
  src[0] = level;
  for (int k = 0; k < np; k++) src[1 + k] = c->n_q + k;
  for (int t = 0; t < level; t++) dst[t] = t;
  /* the sources to coefficients */
  u64 *xs = (u64 *)malloc(sizeof(u64) * (u64)ns * n);
  memcpy(xs, x + (u64)level * n, sizeof(u64) * n);
  memcpy(xs + n, x + (u64)nl * n, sizeof(u64) * (u64)np * n);
  oc_intt(c, xs, ns, src);
  /* S, Shat_i = S / s_i and [Shat_i^-1]_{s_i} */
  u64 *big = (u64 *)calloc((u64)(ns + 2) * w, sizeof(u64));
  u64 *S = big, *half = big + w, *shat = big + 2 * w;
  u64 *shat_inv = (u64 *)malloc(sizeof(u64) * ns);
  S[0] = 1;
  for (int i = 0; i < ns; i++) {
    u64 tmp[OC_MAXMOD];
    mw_mul_word(S, w, c->mod[src[i]], tmp);
    memcpy(S, tmp, sizeof(u64) * w);
  }
  for (int i = 0; i < w; i++) half[i] = (S[i] >> 1) | (i + 1 < w ? S[i + 1] << 63 : 0); /* (S - 1) / 2 */
  for (int i = 0; i < ns; i++) {
    u64 *h = shat + (u64)i * w, tmp[OC_MAXMOD];
    memset(h, 0, sizeof(u64) * w);
    h[0] = 1;
    for (int k = 0; k < ns; k++)
      if (k != i) {
        mw_mul_word(h, w, c->mod[src[k]], tmp);
        memcpy(h, tmp, sizeof(u64) * w);
      }
    shat_inv[i] = invmod(mw_mod(h, w, c->mod[src[i]]), c->mod[src[i]]);
  }
  /* r mod q_t per coefficient (coefficient domain) */
  u64 *z = (u64 *)malloc(sizeof(u64) * (u64)level * n);
  u64 smod_t[OC_MAXMOD];
  for (int t = 0; t < level; t++) smod_t[t] = mw_mod(S, w, c->mod[t]);
#pragma omp parallel for schedule(static)
  for (u64 k = 0; k < n; k++) {
    u64 v[OC_MAXMOD], tmp[OC_MAXMOD];
    memset(v, 0, sizeof(u64) * w);
    for (int i = 0; i < ns; i++) {
      u64 si = c->mod[src[i]];
      u64 y = mulmod(xs[(u64)i * n + k], shat_inv[i], si);
      mw_mul_word(shat + (u64)i * w, w, y, tmp);
      mw_add(v, tmp, w);
    }
    while (mw_cmp(v, S, w) >= 0) mw_sub(v, S, w); /* V = X mod S */
    int neg = mw_cmp(v, half, w) > 0;               /* r = V - S when V > (S - 1)/2 */
    for (int t = 0; t < level; t++) {
      u64 q = c->mod[t], vm = mw_mod(v, w, q);
      z[(u64)t * n + k] = neg ? submod(vm, smod_t[t], q) : vm;
    }
  }
  oc_ntt(c, z, level, dst);
  for (int t = 0; t < level; t++) {
    u64 q = c->mod[t], sinv = invmod(smod_t[t], q);
    for (u64 k = 0; k < n; k++) {
      u64 i = (u64)t * n + k;
      out[i] = mulmod(submod(x[i], z[i], q), sinv, q);
    }
  }
  free(xs);
  free(z);
  free(big);
  free(shat_inv);
  return 0;
}

/* C6 + C21: relinearised product divided by P q_l in the merged step.  The
 * tensor's (d0, d1) join the key-switch accumulator as P d (which vanishes
 * modulo the special primes), so out = round((acc + P d) / (P q_l)).
 * out: [2][level][N], level - 1, NTT domain. */
int oc_mul_relin_rescale(const oc_ctx *c, const u64 *a, const u64 *b, int level, u64 *out) {
  okey *k = find_key(c, 0);
  if (!k || level < 1) return -1;
  u64 n = c->n;
  int nl = level + 1, np = c->n_p, ext = nl + np;
  u64 *d = (u64 *)malloc(sizeof(u64) * (u64)3 * nl * n);
  u64 *d0 = d, *d1 = d + (u64)nl * n, *d2 = d + (u64)2 * nl * n;
  oc_tensor(c, a, b, level, d0, d1, d2);
  u64 *digits = (u64 *)malloc(sizeof(u64) * (u64)c->n_digits * ext * n);
  int nact = modup(c, d2, level, digits);
  u64 *acc = (u64 *)malloc(sizeof(u64) * (u64)2 * ext * n);
  inner(c, digits, nact, level, k->data, acc);
  for (int pol = 0; pol < 2; pol++) {
    u64 *x = acc + (u64)pol * ext * n;
    const u64 *dp = pol == 0 ? d0 : d1;
    for (int t = 0; t < nl; t++) {
      u64 q = c->mod[t], pm = 1;
      for (int kk = 0; kk < np; kk++) pm = mulmod(pm, c->mod[c->n_q + kk] % q, q);
      for (u64 i = 0; i < n; i++) x[(u64)t * n + i] = addmod(x[(u64)t * n + i], mulmod(pm, dp[(u64)t * n + i], q), q);
    }
    oc_moddown_rescale(c, x, level, out + (u64)pol * level * n);
  }
  free(d);
  free(digits);
  free(acc);
  return 0;
}

/* C11: sigma_g on a ciphertext followed by key switching from sigma_g(s) to s. */
int oc_automorph(const oc_ctx *c, const u64 *in, int level, u64 g, u64 *out) {
  okey *k = find_key(c, g);
  if (!k) return -1;
  u64 n = c->n;
  int nl = level + 1;
  int mods[OC_MAXMOD];
  q_basis(nl, mods);
  u64 *tmp = (u64 *)malloc(sizeof(u64) * (u64)2 * nl * n);
  u64 *coef = (u64 *)malloc(sizeof(u64) * (u64)2 * nl * n);
  memcpy(coef, in, sizeof(u64) * (u64)2 * nl * n);
  oc_intt(c, coef, nl, mods);
  oc_intt(c, coef + (u64)nl * n, nl, mods);
  for (int pol = 0; pol < 2; pol++)
    for (int t = 0; t < nl; t++)
      automorph_limb(c, coef + ((u64)pol * nl + t) * n, g, c->mod[t], tmp + ((u64)pol * nl + t) * n);
  oc_ntt(c, tmp, nl, mods);
  oc_ntt(c, tmp + (u64)nl * n, nl, mods);
  u64 *u0 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  u64 *u1 = (u64 *)malloc(sizeof(u64) * (u64)nl * n);
  keyswitch(c, tmp + (u64)nl * n, level, k->data, u0, u1);
  for (int t = 0; t < nl; t++)
    for (u64 x = 0; x < n; x++) {
      u64 i = (u64)t * n + x;
      out[i] = addmod(tmp[i], u0[i], c->mod[t]);
      out[(u64)nl * n + i] = u1[i];
    }
  free(u0);
  free(u1);
  free(tmp);
  free(coef);
  return 0;
}

/* sigma_g applied to each limb of a coefficient-domain polynomial (no key switch) */
void oc_automorph_coeff(const oc_ctx *c, const u64 *in, int n_limbs, const int *mods, u64 g, u64 *out) {
  for (int l = 0; l < n_limbs; l++)
    automorph_limb(c, in + (u64)l * c->n, g, c->mod[mods[l]], out + (u64)l * c->n);
}
