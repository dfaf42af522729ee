/*
 * ckks.h -- C ABI of the GB300 RNS-CKKS evaluation core.
 *
 * The operations follow the statement of CKKS in ReBoot (arXiv 2506.19693),
 * Sec. 3: a parameter set {N, q, Delta} (N the ring degree, q the prime chain,
 * Delta the scale); batching of up to N/2 complex values into one plaintext
 * through the complex canonical embedding; secret-key encryption; slot-wise
 * homomorphic +, -, x (Eq. add, sub, mult) and their plaintext variants;
 * dropping the chain's top prime after a multiplication; Rot(a, k), a cyclic left
 * shift by k slots with one key per k; and bootstrapping.  The scheme's
 * internals (prime chain, NTT order, hybrid key switching, rescale rounding)
 * are the textbook RNS-CKKS readings listed in the design notes as C1..C12.
 *
 * Conventions for every entry point:
 *  - Return value: CKKS_OK (0) or a negative CKKS_E_* status.  Nothing aborts,
 *    nothing throws; ckks_status_str() names a status.
 *  - Device pointers ("_dev") are CUDA global-memory addresses on the device
 *    that was current when the context was created; the caller owns them and
 *    keeps them alive until the work enqueued on the context's stream is done.
 *    Host pointers ("_host" or plain host arrays) are read or written before
 *    the call returns.
 *  - All device work is enqueued on the context's stream (stream order); calls
 *    that return host data synchronise that stream.
 *  - Layout: a polynomial over limbs q_0..q_l is uint64[l+1][N], limb-major,
 *    each limb contiguous, residues in [0, q_i).  A ciphertext buffer is
 *    uint64[2][n_limbs][N]: poly 0 at data, poly 1 at data + n_limbs*N; only
 *    limbs 0..level of each poly are meaningful (n_limbs >= level + 1 is the
 *    capacity, so rescale can work in place).  Ciphertexts and plaintexts live
 *    in the NTT domain, canonical order A[j] = a(psi^(2*brv(j)+1)) mod q_i.
 *  - The context is not thread-safe; use one context per host thread.
 */
#ifndef CKKS_H
#define CKKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CKKS_OK 0
#define CKKS_E_PARAM (-1)   /* invalid argument or parameter set               */
#define CKKS_E_LEVEL (-2)   /* level mismatch, level out of range, level 0 rescale */
#define CKKS_E_SCALE (-3)   /* scaled plaintext >= 2^62 or scale mismatch       */
#define CKKS_E_NOKEY (-4)   /* secret, relinearisation or Galois key missing    */
#define CKKS_E_OOM (-5)     /* device or host allocation failed                 */
#define CKKS_E_CUDA (-6)    /* a CUDA runtime call failed                       */
#define CKKS_E_TIMEOUT (-7) /* a bounded device-side wait ran out               */
#define CKKS_E_STATE (-8)   /* call made in the wrong state                      */

#define CKKS_MAX_Q 60
#define CKKS_MAX_P 16

typedef struct ckks_ctx ckks_ctx;

/* Parameter set Theta = {N, q, Delta} (Sec. 3).  N = 2^log_n (2^12..2^17;
 * Table 3 uses 2^16 and 2^17).  The chain q_0..q_{n_q-1} and the special
 * primes p_0..p_{n_p-1} are the largest primes = 1 mod 2^max(17, log_n + 1)
 * below 2^bits, taken in chain order per bit size (reading C1).  dnum = number of key-switching digits: alpha = ceil(n_q/dnum)
 * q-primes per digit (reading C7).  h = Hamming weight of the ternary secret,
 * sigma = standard deviation of the rounded Gaussian error (tail cut at
 * floor(6 sigma)).  log2_scale is the default scale used by ckks_encode when
 * it is passed scale <= 0. */
typedef struct {
  uint32_t log_n, n_q, n_p, dnum, h;
  uint32_t q_bits[CKKS_MAX_Q], p_bits[CKKS_MAX_P];
  double log2_scale, sigma;
  uint64_t seed; /* unused by ckks_ctx_create; kept for presets */
} ckks_params;

/* A ciphertext handle.  data: device, uint64[2][n_limbs][N], NTT domain.
 * level: index of the top active prime (level + 1 active limbs).
 * scale: Delta of the encrypted message, tracked exactly as a double. */
typedef struct {
  uint64_t *data;
  uint32_t log_n, level, n_limbs, is_ntt;
  double scale;
} ckks_ct;

/* ---- context ------------------------------------------------------------ */

/* Create a context for `params` on the current CUDA device; all its work goes
 * to `cuda_stream` (a cudaStream_t, or NULL for the legacy default stream).
 * Derives primes, roots and all tables and uploads them.  *out owns them. */
int ckks_ctx_create(const ckks_params *params, void *cuda_stream, ckks_ctx **out);
int ckks_ctx_destroy(ckks_ctx *ctx);
/* Change the stream later calls enqueue on. */
int ckks_ctx_set_stream(ckks_ctx *ctx, void *cuda_stream);
/* Host copy of the moduli q_0..q_{n_q-1}, p_0..p_{n_p-1} (cap entries max). */
int ckks_ctx_moduli(const ckks_ctx *ctx, uint64_t *out_host, int cap);
/* Host copy of the primitive 2N-th roots psi_i (reading C2). */
int ckks_ctx_roots(const ckks_ctx *ctx, uint64_t *out_host, int cap);
/* Digits actually used (ceil(n_q / alpha)) and alpha. */
int ckks_ctx_digits(const ckks_ctx *ctx, int *n_digits, int *alpha);
/* Bytes of device memory the context holds (tables, keys, scratch). */
int ckks_ctx_device_bytes(const ckks_ctx *ctx, uint64_t *bytes);

/* ---- launch accounting (no paper counterpart: measurement support) ----- */

/* Enable (1) or disable (0) per-kernel-class device timing: when on, every
 * kernel launch on the context stream is bracketed by a CUDA event pair.
 * Enabling clears earlier records. */
int ckks_ctx_profile(ckks_ctx *ctx, int enable);
/* Fold the recorded event pairs (synchronises them) and copy, per kernel class
 * k < min(cap, ckks_profile_kinds()), the summed device milliseconds, the
 * launch count and the limbs processed since the last reset; then reset.
 * Any of the three arrays may be NULL.  Returns the number of classes. */
int ckks_ctx_profile_read(ckks_ctx *ctx, double *ms, uint64_t *launches, uint64_t *limbs, int cap);
/* Key switches by level since the last ckks_ctx_profile_read or
 * ckks_ctx_profile call (counted whether timing is on or not): counts[l] =
 * outputs of key inner products at level l (each reads one switching key),
 * for l < min(cap, 64).  Call it before ckks_ctx_profile_read, which resets
 * it.  Returns 64. */
int ckks_ctx_ks_histogram(ckks_ctx *ctx, uint64_t *counts, int cap);
/* Number of kernel classes and the name of class k. */
int ckks_profile_kinds(void);
const char *ckks_profile_kind_name(int k);
/* Total kernels this context has launched since creation. */
int ckks_ctx_launch_count(const ckks_ctx *ctx, uint64_t *count);
/* Integer-pipe roofs measured on this GPU by register-only kernels that run
 * the production instruction sequences themselves: out[0] = 128-bit
 * multiply-accumulates per second (the basis conversion's and the key inner
 * product's MAC), out[1] = loose forward NTT butterflies per second (primes
 * with 65 q < 2^64), out[2] = strict forward butterflies, out[3] = inverse
 * butterflies with the approximate quotient (primes below 2^61), out[4] =
 * inverse butterflies with the exact quotient.  Writes min(cap, 5) values and
 * returns 5 (or a negative status).  Synchronises the context stream; uses the
 * context's scratch memory. */
int ckks_alu_peaks(ckks_ctx *ctx, double *out, int cap);

/* ---- arithmetic form --------------------------------------------------- */

#define CKKS_FORM_UINT64 0 /* basis conversion as 64x64->128 MACs on the CUDA cores (default) */
#define CKKS_FORM_TENSOR 1 /* basis conversion as an exact byte-split fp16 GEMM on tcgen05   */
#define CKKS_FORM_FUSED 2  /* uint64 conversion fused with the NTTs' column passes          */

/* Select how ModUp / ModDown basis conversion (reading C8/C9) runs.  All forms
 * give identical limbs.  The tensor form splits each residue into bytes and the
 * constants into byte planes, multiplies on tcgen05 tensor cores with exact fp32
 * accumulation in tensor memory, and recombines modularly.  The fused form runs
 * the key-switch pipeline iNTT -> conversion -> NTT with the middle in one
 * kernel per column tile: the inverse transform's column stages, the
 * conversion (64x64->128 multiply-accumulates on the CUDA cores) and the
 * forward transform's column stages on shared-memory tiles, so the
 * coefficient-domain digits and conversion targets never reach HBM (rings up
 * to 2^16; the 2^17 ring runs the uint64 form's kernels). */
int ckks_ctx_set_form(ckks_ctx *ctx, int form);
/* CKKS_E_TIMEOUT if a bounded device-side wait of a tensor-core kernel expired
 * since the last call (the affected outputs are invalid; no matrix multiply was
 * left running), CKKS_E_CUDA if, in addition, multiplies committed by the
 * expired kernel had still not completed after a second, longer bounded wait
 * when it released its tensor memory (destroy the context), else CKKS_OK.
 * Synchronises the context stream and clears the flag. */
int ckks_ctx_device_error(ckks_ctx *ctx);
/* TEST ONLY (no paper counterpart): run the tensor-core conversion kernel once
 * on a scratch polynomial with its CTAs made to wait, before issuing any
 * matrix multiply, on a barrier that nothing arrives on.  The wait gives up
 * after wait_ns (clamped to 1 ms .. 1 s), so the kernel takes its failure
 * path: it records the error and frees its tensor memory, and the next
 * ckks_ctx_device_error returns CKKS_E_TIMEOUT.  Nothing faults and the
 * context stays usable.  CKKS_E_STATE during graph capture. */
int ckks_debug_tc_expire(ckks_ctx *ctx, uint64_t wait_ns);

/* ---- keys (Sec. 3: one Galois key per rotation step) -------------------- */

/* Draw the ternary secret from `seed` and build the relinearisation key
 * (s^2 -> s) plus one Galois key per rotation step in rot_steps[0..n_rot)
 * (left rotation by k, g = 5^(k mod N/2) mod 2N), the conjugation key when
 * want_conj, and, when want_boot, the conjugation key and every rotation key
 * the bootstrapping circuit uses (ckks_boot_rotation_steps).  Randomness:
 * counter-based SplitMix64 keyed by seed (reading C4).  Replaces earlier keys,
 * the public key included. */
int ckks_keygen_from_seed(ckks_ctx *ctx, uint64_t seed, const int32_t *rot_steps, int n_rot,
                          int want_conj, int want_boot);
/* Key compression (reading C22; no paper counterpart).  With on = 1, keys
 * generated afterwards keep only their b rows and, per digit, the state of
 * the counter-based generator that drew a_j; the key inner product
 * regenerates a_j.  The keys' values are unchanged, so every result is
 * bit-identical; device key memory and key reads halve.  CKKS_E_STATE once a
 * key exists (call it before the first keygen). */
int ckks_set_key_compression(ckks_ctx *ctx, int on);
/* Add the Galois key for element g (odd, < 2N) to the current key set. */
int ckks_keygen_galois(ckks_ctx *ctx, uint64_t galois_elt);
/* Galois element of a left rotation by k. */
uint64_t ckks_galois_elt(const ckks_ctx *ctx, int32_t k);
/* TEST ONLY: host copy of the ternary secret (int8[N]). */
int ckks_debug_secret(const ckks_ctx *ctx, int8_t *out_host);
/* TEST ONLY: host copy of one switching key, uint64[n_digits][2][n_q+n_p][N]
 * (b_j, a_j per digit, NTT domain, residues in [0, q)); galois_elt 0 selects
 * relinearisation.  The device keeps keys in Montgomery form (x 2^64 mod q);
 * this call converts them back. */
int ckks_debug_key(const ckks_ctx *ctx, uint64_t galois_elt, uint64_t *out_host);

/* ---- plaintexts (Sec. 3 batching) --------------------------------------- */

/* Encode n_slots <= N/2 complex values (re/im host arrays; missing slots are 0)
 * at `scale` (<= 0 selects the default) into an NTT-domain plaintext over
 * q_0..q_level: pt_dev is uint64[level+1][N].  Coefficients are
 * round-half-away(scale * tau^-1(z)) computed in FP64 on the GPU; CKKS_E_SCALE
 * if any reaches 2^62. */
int ckks_encode(ckks_ctx *ctx, const double *re, const double *im, int n_slots, uint32_t level,
                double scale, uint64_t *pt_dev);
/* Decode an NTT-domain plaintext over q_0..q_level: centred CRT to FP64, then
 * the forward embedding, divided by `scale`.  Writes n_slots values to re/im. */
int ckks_decode(ckks_ctx *ctx, const uint64_t *pt_dev, uint32_t level, double scale, double *re,
                double *im, int n_slots);
/* Signed integer coefficients (host int64[N], |m| < 2^62) -> NTT-domain
 * residues over q_0..q_level in pt_dev. */
int ckks_pt_from_int(ckks_ctx *ctx, const int64_t *m_host, uint32_t level, uint64_t *pt_dev);
/* Forward (inverse != 0: inverse) negacyclic NTT, in place, of n_limbs limbs
 * at data_dev; limb l uses modulus index first_mod + l (0..n_q-1 are q_i,
 * n_q.. are p_j).  Residues in [0, modulus) in and out. */
int ckks_ntt(ckks_ctx *ctx, uint64_t *data_dev, uint32_t n_limbs, uint32_t first_mod, int inverse);
/* Forward NTT of n_polys (1..128) polynomials stored back to back
 * (uint64[n_polys][n_limbs][N], limb t under modulus t), in place, with the
 * first four column stages on the tensor cores (no paper counterpart: the
 * byte-split tensor-core form of an NTT stage group, measured against the
 * butterflies).  Those stages map every 16-point block by one 16 x 16 matrix
 * over Z_q, applied to the limb's 16-row slabs as an exact byte-split fp16
 * GEMM on tcgen05 with fp32 accumulation and modular recombination; the other
 * twelve stages run as in ckks_ntt.  Same residues as ckks_ntt.  N = 2^15 or
 * 2^16 (else CKKS_E_PARAM); uses the context scratch (n_polys N words). */
int ckks_ntt_tc(ckks_ctx *ctx, uint64_t *data_dev, uint32_t n_polys, uint32_t n_limbs);
/* Key-switch inner product (reading C7: the products of the lifted digits with
 * the key, summed over digits) for a batch sharing one key, in two forms with
 * identical outputs, for comparison:
 *   out[p][o][t][k] = sum_j d[p][j][t][k] key[j][o][t][k]  mod q_t,  o = 0, 1,
 * all device arrays of plain residues: d uint64[n_cts][n_digits][n_limbs][N],
 * key uint64[n_digits][2][n_limbs][N], out uint64[n_cts][2][n_limbs][N]
 * (16-byte aligned); limb t is reduced mod the context's modulus t.
 * n_digits 1..4, n_limbs <= min(40, n_q + n_p) (else CKKS_E_PARAM); CKKS_E_STATE
 * during graph capture.
 * _tc: a byte-split fp16 GEMM on tcgen05 per coefficient, M = 128 ciphertexts
 * (n_cts must be 128), N = 16 (2 outputs x 8 byte planes of 2^(8a) key mod q),
 * K = 8 n_digits, fp32 accumulation in tensor memory, modular recombination;
 * bounded waits as the tensor-core conversion (ckks_ctx_device_error).
 * _u64: 128-bit multiply-accumulates on the CUDA cores, any n_cts >= 1. */
int ckks_ks_inner_tc(ckks_ctx *ctx, const uint64_t *d_dev, const uint64_t *key_dev, uint32_t n_cts,
                     uint32_t n_digits, uint32_t n_limbs, uint64_t *out_dev);
int ckks_ks_inner_u64(ckks_ctx *ctx, const uint64_t *d_dev, const uint64_t *key_dev, uint32_t n_cts,
                      uint32_t n_digits, uint32_t n_limbs, uint64_t *out_dev);

/* ---- encryption (Sec. 3, reading C5) ------------------------------------ */

/* ct = ([-a s + m + e], a) over q_0..q_level; a uniform (drawn in the NTT
 * domain), e rounded Gaussian, both from enc_seed.  out->data must hold
 * out->n_limbs >= level + 1 limbs per poly; level/scale/is_ntt are set. */
int ckks_encrypt(ckks_ctx *ctx, const uint64_t *pt_dev, uint32_t level, double scale,
                 uint64_t enc_seed, ckks_ct *out);
/* pt_dev (uint64[level+1][N]) = c0 + c1 s, NTT domain. */
int ckks_decrypt(ckks_ctx *ctx, const ckks_ct *ct, uint64_t *pt_dev);

/* Public key (Sec. 3 writes encryption as E(pk, .); reading C5, pk form):
 * pk = ([-a s + e]_Q, a) over q_0..q_{n_q-1}, NTT domain, the secret-key
 * encryption of 0 with a and e drawn from the key seed's own streams.  Needs
 * the secret (CKKS_E_NOKEY before ckks_keygen_from_seed); CKKS_E_STATE during
 * graph capture.  Kept on the device until the next key generation. */
int ckks_keygen_public(ckks_ctx *ctx);
/* Copy the public key to host memory: out_host uint64[2][n_q][N] (b, then a),
 * NTT domain.  CKKS_E_NOKEY before ckks_keygen_public. */
int ckks_public_key_export(ckks_ctx *ctx, uint64_t *out_host);
/* Public-key encryption (reading C5, pk form): with the mask v (each
 * coefficient 0 with probability 1/2, +1 and -1 with 1/4 each) and rounded
 * Gaussian e0, e1, all from enc_seed's streams,
 *   ct = ([v b + m + e0], [v a + e1]) over q_0..q_level,
 * products negacyclic (point-wise in the NTT domain).  Arguments as
 * ckks_encrypt; CKKS_E_NOKEY without a public key. */
int ckks_encrypt_pk(ckks_ctx *ctx, const uint64_t *pt_dev, uint32_t level, double scale,
                    uint64_t enc_seed, ckks_ct *out);

/* ---- evaluation (Eq. add, sub, mult; Sec. 3) ----------------------------- */

/* Slot-wise sum / difference; levels must match (CKKS_E_LEVEL).  out may alias. */
int ckks_add(ckks_ctx *ctx, const ckks_ct *a, const ckks_ct *b, ckks_ct *out);
int ckks_sub(ckks_ctx *ctx, const ckks_ct *a, const ckks_ct *b, ckks_ct *out);
/* (c0 * pt, c1 * pt); out->scale = a->scale * pt_scale. */
int ckks_mul_plain(ckks_ctx *ctx, const ckks_ct *a, const uint64_t *pt_dev, double pt_scale,
                   ckks_ct *out);
/* (c0 + pt, c1); the plaintext must be at a's scale. */
int ckks_add_plain(ckks_ctx *ctx, const ckks_ct *a, const uint64_t *pt_dev, ckks_ct *out);
/* Multiply by a signed integer constant; consumes no level (reading C14). */
int ckks_mul_int(ckks_ctx *ctx, const ckks_ct *a, int64_t k, ckks_ct *out);
/* Relinearised product (reading C6): (d0, d1) + KeySwitch_{s^2->s}(d2) with
 * d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.  out->scale = a->scale*b->scale. */
int ckks_mul_relin(ckks_ctx *ctx, const ckks_ct *a, const ckks_ct *b, ckks_ct *out);
/* Drop the top prime q_l: c'_i = (c_i - [c_l]_centred) * q_l^-1 mod q_i
 * (reading C10); level -1, scale / q_l.  In place; CKKS_E_LEVEL at level 0. */
int ckks_rescale(ckks_ctx *ctx, ckks_ct *inout);
/* Rot(a, k): left cyclic shift of the slots by k (Sec. 3), via
 * X -> X^(5^k mod 2N) and key switching (reading C11). */
int ckks_rotate(ckks_ctx *ctx, const ckks_ct *a, int32_t k, ckks_ct *out);
/* Rescale that allocates nothing.  The paper has no counterpart: this exists
 * for callers that cannot let the library call cudaMalloc -- a process whose
 * device memory is capped or handed out by its own pool allocator, or a
 * latency-bound path that cannot accept an allocation's implicit
 * synchronisation.  ckks_rescale may grow the context's scratch buffer; this
 * variant gives the same limbs (same arithmetic) using a fixed 5 MiB
 * workspace in a file-scope device array that every GPU loading the library
 * holds until exit.  Limit: N <= 2^17 (larger rings return CKKS_E_PARAM); any
 * level.  At N = 2^17 the array holds one lifted limb of each polynomial per
 * pass, at N = 2^16 four.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current -- make that
 * first call before any stream capture; a failed lookup returns CKKS_E_CUDA
 * and is retried by the next call.  All calls share the array, so calls whose GPU
 * work overlaps (other streams or threads) race; nothing in it must start at
 * zero.  The current device must be the context's.  In place, like
 * ckks_rescale; CKKS_E_LEVEL at level 0.  Allocates no device memory as long
 * as event profiling (ckks_ctx_profile) is off. */
int ckks_rescale_noalloc(ckks_ctx *ctx, ckks_ct *inout);
/* Complex conjugation of every slot (X -> X^(2N-1)). */
int ckks_conjugate(ckks_ctx *ctx, const ckks_ct *a, ckks_ct *out);
/* Apply the automorphism X -> X^g (g odd, < 2N) and switch back to s. */
int ckks_automorph(ckks_ctx *ctx, const ckks_ct *a, uint64_t galois_elt, ckks_ct *out);

/* ---- bootstrapping (Sec. 3 last paragraph; Alg. 1; Sec. 5.1: tau_bs = 16) --- */

/* Build the bootstrapping circuit for this parameter set (needs n_q >= 17)
 * and generate its constants on the GPU in FP64: the diagonals of the three
 * CoeffToSlot and three SlotToCoeff levels of the special DFT (readings
 * B2-B4), encoded at the scale of the prime each level drops, and the
 * degree-60 Chebyshev coefficients of EvalMod (B6).  Run once per context,
 * before ckks_bootstrap; keys come from ckks_keygen_from_seed(want_boot=1). */
int ckks_boot_setup(ckks_ctx *ctx);
/* Sparse slots (reading B13): bootstrap messages of n_slots (a power of two,
 * 2 .. N/2) complex slots, each stored as the full-slot vector repeated with
 * period n_slots (ckks_encode of the repeated vector).  The circuit adds the
 * sub-sum rotations by n_slots 2^i after ModRaise and runs n_slots-point
 * transforms.  Call before ckks_keygen_from_seed(want_boot=1) and
 * ckks_boot_setup; CKKS_E_STATE once a plan with another count exists. */
int ckks_boot_set_slots(ckks_ctx *ctx, uint32_t n_slots);
/* Left-rotation steps the circuit uses (sorted); returns their count and
 * writes up to cap of them to out (NULL allowed). */
int ckks_boot_rotation_steps(ckks_ctx *ctx, int32_t *out, int cap);
/* Number of diagonal plaintexts of the circuit. */
int ckks_boot_constant_count(ckks_ctx *ctx);
/* Replace the circuit's constants: count = ckks_boot_constant_count integer
 * coefficient vectors (host int64[count][N], plan order: CoeffToSlot levels
 * then SlotToCoeff levels; per level ascending giant step, then ascending
 * baby step) and the n_cheb = 61 Chebyshev coefficients.  Used to run the
 * circuit on constants produced elsewhere (e.g. an independent oracle). */
int ckks_boot_import(ckks_ctx *ctx, const int64_t *coeffs, int count, const double *cheb, int n_cheb);
/* Copy the current constants out in the same layout (centred integer
 * coefficients) and the Chebyshev coefficients; either array may be NULL. */
int ckks_boot_export(ckks_ctx *ctx, int64_t *coeffs, int count, double *cheb, int n_cheb);
/* Refresh ciphertexts whose modulus is exhausted: ModRaise, CoeffToSlot,
 * EvalMod, SlotToCoeff (B1-B8).  Inputs are read at level 0 (limb q_0 only);
 * outputs come back at level n_q - 1 - 16 with scale Delta_in * S / q_0
 * (S ~ q_0), decrypting to the input slots within about 2^-12.  out[i] needs
 * n_limbs >= n_q - 16.  Needs the relinearisation, conjugation and rotation
 * keys of ckks_keygen_from_seed(want_boot=1) (CKKS_E_NOKEY) and
 * ckks_boot_setup or ckks_boot_import (CKKS_E_STATE). */
int ckks_bootstrap(ckks_ctx *ctx, const ckks_ct *in, ckks_ct *out);
int ckks_bootstrap_batch(ckks_ctx *ctx, const ckks_ct *in, ckks_ct *out, int n);
/* One merged level of the circuit's special DFT on its own (readings B3,
 * B10, B11; the linear transforms of the bootstrapping Sec. 3 cites): plan
 * level `index`, 0..2 the CoeffToSlot levels and 3..5 the SlotToCoeff levels
 * in circuit order, applied to n ciphertexts exactly as ckks_bootstrap applies
 * it (same constants, same launches).  Inputs at a level >= the plan level's
 * (ckks_boot_export gives the plan's constants; CKKS_E_LEVEL below), all at
 * one scale (CKKS_E_SCALE); outputs one level below the plan level with the
 * input scale (the diagonals are encoded at the dropped prime).  Needs
 * ckks_boot_setup or ckks_boot_import (CKKS_E_STATE) and the level's
 * rotation keys. */
int ckks_boot_linear(ckks_ctx *ctx, int index, const ckks_ct *in, ckks_ct *out, int n);
/* Iterative bootstrapping (Sec. 5.1 sizes tau_bs for it, citing Bae et al.
 * 2022; reading B12): ct1 = Bootstrap(ct); the level-0 difference
 * align(ct1, 0, Delta_in) - ct is multiplied by 2^log2_k and bootstrapped
 * again (ct2); out = 2^log2_k ct1 - ct2 at the same level n_q - 1 - 16, with
 * scale 2^log2_k * Delta_in * S / q_0.  Twice the work of ckks_bootstrap for
 * an error about 2^log2_k times smaller, down to the inputs' own noise.
 * All n inputs share one scale (CKKS_E_SCALE); 1 <= log2_k <= 30
 * (CKKS_E_PARAM); log2_k must keep 2^log2_k times the first pass's error
 * inside the sine's range (about 2^-22 at N = 2^16: log2_k <= 20).  Other
 * requirements and errors as ckks_bootstrap_batch. */
int ckks_bootstrap_iterative_batch(ckks_ctx *ctx, const ckks_ct *in, ckks_ct *out, int n, int log2_k);

/* ---- batched variants: n independent ciphertexts in one set of launches -- */

#define CKKS_RESCALE_NONE 0     /* out at the inputs' level                                   */
#define CKKS_RESCALE_SEPARATE 1 /* ModDown (C9) then rescale (C10): the limbs of ckks_rescale */
#define CKKS_RESCALE_MERGED 2   /* ModDown and rescale merged (no paper counterpart; an
                                 * implementation choice the paper leaves open, reading C21):
                                 * the key-switch accumulator plus P (d0, d1) is divided by
                                 * P q_l in one fast basis conversion from {q_l, p_0..p_{K-1}}
                                 * to q_0..q_{l-1} whose overflow is estimated in fixed point
                                 * and removed, rounding to nearest: out = round(x / (P q_l))
                                 * + e, e in {0, 1} and almost always 0.  Saves ModDown's NTT
                                 * of 2(l+1) limbs and the rescale's own transforms; limbs
                                 * differ from SEPARATE by at most 2 per coefficient. */

/* out[i] = mul_relin(a[i], b[i]), rescaled per do_rescale (CKKS_RESCALE_*;
 * another value: CKKS_E_PARAM; a rescale at level 0: CKKS_E_LEVEL).
 * All a[i], b[i] at one level. */
int ckks_mul_relin_batch(ckks_ctx *ctx, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n,
                         int do_rescale);
/* out[i] = rotate(in[i], k[i]). */
int ckks_rotate_batch(ckks_ctx *ctx, const ckks_ct *in, const int32_t *k, ckks_ct *out, int n);
/* Hoisted rotations (one ModUp of each input's c1 shared by all steps):
 * out[j*n + i] = Rot(in[i], k[j]) for i < n, j < n_k.  The lifted digits are
 * mapped by the automorphism before the key inner product, so the limbs
 * differ from n_k separate ckks_rotate calls (by multiples of the digit
 * moduli, absorbed by the gadget) while decrypting to the same slots.
 * Outputs must not alias inputs (CKKS_E_PARAM). */
int ckks_rotate_hoisted(ckks_ctx *ctx, const ckks_ct *in, int n, const int32_t *k, int n_k, ckks_ct *out);
/* Element-wise batches (Eq. add/sub; plaintext and integer variants):
 * out[i] = a[i] +- b[i]; out[i] = k * a[i]; out[i] = a[i] * pt (same
 * plaintext for all, scale a.scale * pt_scale); out[i] = a[i] + pt.
 * All inputs at one level; out may alias a. */
int ckks_add_batch(ckks_ctx *ctx, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n, int subtract);
int ckks_mul_int_batch(ckks_ctx *ctx, const ckks_ct *a, int64_t k, ckks_ct *out, int n);
int ckks_mul_plain_batch(ckks_ctx *ctx, const ckks_ct *a, const uint64_t *pt_dev, double pt_scale, ckks_ct *out,
                         int n);
int ckks_add_plain_batch(ckks_ctx *ctx, const ckks_ct *a, const uint64_t *pt_dev, ckks_ct *out, int n);
/* In-place rescale of n ciphertexts at one level. */
int ckks_rescale_batch(ckks_ctx *ctx, ckks_ct *inout, int n);

/* Relinearised products of n ciphertext pairs that live in HOST memory (no
 * paper counterpart: the batched multiply of Eq. mult fed from the host).
 * a_host, b_host: n x uint64[2][level+1][N] (NTT domain, the layout of
 * ckks_ct_export_ntt), scales scale_a, scale_b; out_host: n x
 * uint64[2][level'+1][N] with level' = level - (do_rescale != NONE);
 * *out_scale (may be NULL) receives the products' scale.  The batch is cut
 * into chunks of `chunk` (1..128) pairs: the host->device copy of chunk i+1,
 * the products of chunk i (on the context stream) and the device->host copy
 * of chunk i-1 overlap on two non-blocking copy streams and three staging
 * slots owned by the context.  Copies are asynchronous only from page-locked
 * host memory (otherwise they serialise but stay correct).  Returns when
 * out_host is complete; CKKS_E_STATE during graph capture. */
int ckks_mul_relin_host(ckks_ctx *ctx, const uint64_t *a_host, const uint64_t *b_host, double scale_a,
                        double scale_b, uint32_t level, int n, int do_rescale, int chunk, uint64_t *out_host,
                        double *out_scale);

/* Packed wire format (no paper counterpart): a ciphertext at level l is its
 * polynomial 0 then polynomial 1, each the limbs t = 0..l in order, limb t
 * holding the N residues in bits(q_t) bits each, residue k at bits
 * [k b, k b + b) of the limb's little-endian 64-bit words.  With 55-bit
 * primes that is 14% fewer bytes than uint64 limbs.  ckks_wire_bytes gives the
 * size of one ciphertext at `level`.  export/import pack / unpack on the GPU
 * (ct's level and capacity as for ckks_ct_export/import); host buffers must
 * be 8-byte aligned (CKKS_E_PARAM). */
int ckks_wire_bytes(const ckks_ctx *ctx, uint32_t level, uint64_t *bytes);
int ckks_ct_export_packed(ckks_ctx *ctx, const ckks_ct *ct, uint8_t *out_host);
int ckks_ct_import_packed(ckks_ctx *ctx, const uint8_t *in_host, ckks_ct *ct);
/* ckks_mul_relin_host with packed host buffers: a_host, b_host hold n
 * ciphertexts of ckks_wire_bytes(level) bytes each, out_host n of
 * ckks_wire_bytes(level') bytes; the GPU unpacks each chunk after its copy-in
 * and packs the products before their copy-out. */
int ckks_mul_relin_host_packed(ckks_ctx *ctx, const uint8_t *a_host, const uint8_t *b_host, double scale_a,
                               double scale_b, uint32_t level, int n, int do_rescale, int chunk, uint8_t *out_host,
                               double *out_scale);

/* ---- uneven batches: executor, graph capture, tuning ------------------- */

#define CKKS_OP_MUL_RELIN 1 /* out = a * b relinearised (rescaled when rescale != 0) */
#define CKKS_OP_ROTATE 2    /* out = Rot(a, k)                                         */
#define CKKS_OP_RESCALE 3   /* out = rescale(a), a left unchanged                      */

/* One operation of an uneven batch.  a, b, out point to caller-owned handles;
 * out must not alias a or b.  Operations of one batch are independent (none
 * reads another's output); each may use its own context (ring degree). */
typedef struct {
  int op;
  ckks_ctx *ctx;
  const ckks_ct *a;
  const ckks_ct *b;
  ckks_ct *out;
  int32_t k;
  int rescale;         /* CKKS_OP_MUL_RELIN: a CKKS_RESCALE_* mode */
} ckks_op_desc;

typedef struct ckks_graph ckks_graph;

/* Run n independent operations, grouped by (context, operation, level) so each
 * group is one batched launch set on its context's stream; the out handles'
 * level and scale are updated. */
int ckks_exec(const ckks_op_desc *ops, int n);
/* Run the batch once (sizing every scratch buffer), then capture the same
 * grouped launches on `stream` into a CUDA graph; *out replays the whole
 * batch with one cudaGraphLaunch.  The graph reads and writes the buffers the
 * handles pointed to at capture time.  `cuda_stream` must be a created
 * stream (not the legacy or per-thread default stream: CKKS_E_PARAM). */
int ckks_exec_capture(const ckks_op_desc *ops, int n, void *cuda_stream, ckks_graph **out);
int ckks_graph_launch(ckks_graph *graph, void *cuda_stream);
int ckks_graph_destroy(ckks_graph *graph);
/* Autotune the key inner product for this context: time outputs-per-thread
 * groups of 2..32 on a batch of `batch` key switches at `level` and keep the
 * fastest for later calls; *chosen (may be NULL) receives it. */
int ckks_tune(ckks_ctx *ctx, int level, int batch, int *chosen);
/* Autotune the NTT's row pass for this context: time forward + inverse
 * transforms of n_polys (1..64) polynomials over all ciphertext primes with
 * 16 and 8 rows per CTA and keep the faster; *rows (may be NULL) receives it.
 * At N = 2^16 it then times the forward transform in one pass on clusters
 * (ckks_ctx_set_ntt_cluster) against the two passes and keeps the faster.
 * Last it times the row pass that carries the key-switch finish with 16 and 8
 * rows per CTA (ckks_ctx_set_finish_rows) and keeps the faster.
 * Needs the relinearisation key (its limbs are the timing input);
 * CKKS_E_STATE during graph capture. */
int ckks_tune_ntt(ckks_ctx *ctx, int n_polys, int *rows);
/* Set the NTT row-pass tile directly: 16 or 8 rows per CTA (else CKKS_E_PARAM). */
int ckks_ctx_set_ntt_rows(ckks_ctx *ctx, int rows);
/* Forward NTT in one pass (Sec. 2.2's negacyclic transform, the same
 * butterflies and the same residues as the two-pass form): on = 1 runs each
 * limb of a full forward transform on a cluster of 8 CTAs that hold the whole
 * limb in distributed shared memory, so it is read from and written to HBM
 * once; on = 0 restores the two passes.  N = 2^16 only (else CKKS_E_PARAM when
 * on = 1).  *max_clusters (may be NULL) receives how many such clusters the
 * device runs at once; CKKS_E_CUDA when it runs none.  The inverse and the
 * fused conversion's column passes are unchanged. */
int ckks_ctx_set_ntt_cluster(ckks_ctx *ctx, int on, int *max_clusters);
/* The NTT launch choices in force: *rows (16 or 8 rows per row-pass CTA) and
 * *cluster (1 when the forward transform runs in one pass); either may be NULL. */
int ckks_ctx_ntt_config(const ckks_ctx *ctx, int *rows, int *cluster);
/* Key-switch finish in the forward NTT's row pass (ModDown, reading C9; the
 * merged ModDown-rescale, reading C21): on = 1 (the default) computes the last
 * step of every ModDown, (acc - [converted limbs]) P^-1 + base, and of every
 * merged ModDown-rescale in the output stage of the transform that brings the
 * converted limbs to the NTT domain, so those limbs are never stored; on = 0
 * runs the transform and then a separate element-wise kernel.  The rescale's
 * last step, (c - [lifted top limb]) q_l^-1 (reading C10), takes the same
 * route.  Both give the same residues.  The fused form always takes the
 * two-pass transform.  Pointers not 16-byte aligned take the separate kernel.
 * CKKS_E_PARAM unless on is 0 or 1. */
int ckks_ctx_set_fused_finish(ckks_ctx *ctx, int on);
/* The row tile of the forward row pass that carries the key-switch finish: 16
 * or 8 rows per CTA, or 0 to follow ckks_ctx_set_ntt_rows (the default); else
 * CKKS_E_PARAM.  ckks_tune_ntt times both and sets it. */
int ckks_ctx_set_finish_rows(ckks_ctx *ctx, int rows);
/* The row tile in force for that pass (16 or 8) in *rows. */
int ckks_ctx_finish_rows(const ckks_ctx *ctx, int *rows);
/* Autotune the gadget (reading C7) of a parameter set: for each candidate
 * dnum a context with alpha = ceil(n_q / dnum) special primes of p_bits[0]
 * bits (P spans one digit) is created on cuda_stream, its relinearisation key
 * generated from `seed`, and a batch of `batch` (1..128) HMult+relin with the
 * merged rescale timed at the top level, then destroyed.  *best receives the
 * fastest dnum; ms_per_op[i] (may be NULL) each candidate's milliseconds per
 * product (HUGE_VAL where it does not fit: alpha + 1 > 16 sources).  Allocates
 * and frees device memory; CKKS_E_PARAM when no candidate fits. */
int ckks_tune_dnum(const ckks_params *params, void *cuda_stream, const uint32_t *cands, int n_cands, int batch,
                   uint64_t seed, uint32_t *best, double *ms_per_op);

/* ---- ciphertext buffers and host exchange (Sec. 3: a ciphertext is a pair
 * of polynomials of R_q; these calls move one between HBM and the host) ---- */

/* Allocate a ciphertext buffer of n_limbs (1..n_q) limbs per polynomial on the
 * context's device (uint64[2][n_limbs][N], zero-filled on the context
 * stream) and fill *out: level = n_limbs - 1, is_ntt = 1, scale = the default
 * scale.  The buffer belongs to the caller, who releases it with
 * ckks_ct_free (not cudaFree).  For callers that do not wrap their own device
 * memory.  CKKS_E_OOM when the allocation fails, CKKS_E_STATE during graph
 * capture. */
int ckks_ct_alloc(ckks_ctx *ctx, uint32_t n_limbs, ckks_ct *out);
/* Release a buffer from ckks_ct_alloc after the context stream's work is
 * done (synchronises it); sets ct->data to NULL.  A NULL data is a no-op.
 * Passing a buffer not from ckks_ct_alloc is undefined. */
int ckks_ct_free(ckks_ctx *ctx, ckks_ct *ct);
/* Copy a ciphertext's active limbs to host memory as uint64[2][level+1][N]
 * in the COEFFICIENT domain: both polynomials c0, c1 of ct = (c0, c1) with
 * coefficient k of limb t in [0, q_t).  The inverse NTT runs on the GPU into
 * the context's scratch (which may grow); ct is unchanged.  Synchronises the
 * stream. */
int ckks_ct_export(ckks_ctx *ctx, const ckks_ct *ct, uint64_t *out_host);
/* The inverse: in_host (uint64[2][level+1][N], coefficient domain, residues
 * in [0, q_t), else CKKS_E_PARAM before anything is copied) fills ct's
 * active limbs (ct->level and n_limbs as set by the caller), transformed to
 * the NTT domain on the GPU.  Synchronises the stream. */
int ckks_ct_import(ckks_ctx *ctx, const uint64_t *in_host, ckks_ct *ct);
/* The same two copies without the transforms: the NTT-domain limbs as they
 * live in HBM (canonical order).  Used by checkpointing and by the tests'
 * limb-for-limb comparisons. */
int ckks_ct_export_ntt(ckks_ctx *ctx, const ckks_ct *ct, uint64_t *out_host);
int ckks_ct_import_ntt(ckks_ctx *ctx, const uint64_t *in_host, ckks_ct *ct);

const char *ckks_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* CKKS_H */
