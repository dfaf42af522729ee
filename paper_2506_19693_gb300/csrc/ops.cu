// Element-wise RNS-CKKS kernels: slot-wise add/sub (Eq. add, sub), plaintext
// multiply/add, integer-constant multiply, tensor product (reading C6),
// Galois automorphisms in the NTT domain (C11), rescale (C10), encryption and
// decryption (C5) and on-device uniform sampling (C4).  All of these are
// HBM-bound streams over limb-major uint64 data: one thread per coefficient,
// limbs on gridDim.y, ciphertexts on gridDim.z.
#include "ops.cuh"

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ u32 brv_dev(u32 x, int bits) { return __brev(x) >> (32 - bits); }

// signed 64-bit integer -> residue in [0, q)
__device__ __forceinline__ u64 signed_res(i64 x, const ModInfo &m) {
  if (x >= 0) return reduce128(0, (u64)x, m);
  const u64 mag = reduce128(0, (u64)(-(x + 1)) + 1, m);
  return mag ? m.q - mag : 0;
}

__global__ void k_addsub(EwArgs a, int sub) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const u64 q = a.mods[l].q;
  const size_t off = (size_t)l * a.n + k;
  const u64 x0 = a.x0[c][off], x1 = a.x1[c][off], y0 = a.y0[c][off], y1 = a.y1[c][off];
  a.o0[c][off] = sub ? submod(x0, y0, q) : addmod(x0, y0, q);
  a.o1[c][off] = sub ? submod(x1, y1, q) : addmod(x1, y1, q);
}

// mode 0: (c0 pt, c1 pt); mode 1: (c0 + pt, c1).  Plaintext pointer in y0.
__global__ void k_plain(EwArgs a, int mode) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[l];
  const size_t off = (size_t)l * a.n + k;
  const u64 pt = a.y0[c][off], x0 = a.x0[c][off], x1 = a.x1[c][off];
  if (mode == 0) {
    a.o0[c][off] = mulmod(x0, pt, m);
    a.o1[c][off] = mulmod(x1, pt, m);
  } else {
    a.o0[c][off] = addmod(x0, pt, m.q);
    a.o1[c][off] = x1;
  }
}

__global__ void k_mul_int(EwArgs a, i64 kconst) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[l];
  const u64 kk = signed_res(kconst, m);
  const size_t off = (size_t)l * a.n + k;
  const u64 x0 = a.x0[c][off], x1 = a.x1[c][off];
  a.o0[c][off] = mulmod(x0, kk, m);
  a.o1[c][off] = mulmod(x1, kk, m);
}

// tensor product (C6): d0 = a0 b0 -> o0, d1 = a0 b1 + a1 b0 -> o1, d2 = a1 b1 -> d2
struct D2Ptrs {
  u64 *p[MAX_CTS];
};
__global__ void k_tensor(EwArgs a, D2Ptrs d2) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[l];
  const size_t off = (size_t)l * a.n + k;
  const u64 a0 = a.x0[c][off], a1 = a.x1[c][off];
  const u64 b0 = a.y0[c][off], b1 = a.y1[c][off];
  u64 hi = 0, lo = 0;
  mac128(hi, lo, a0, b1);
  mac128(hi, lo, a1, b0);
  const u64 r0 = mulmod(a0, b0, m), r1 = reduce128(hi, lo, m), r2 = mulmod(a1, b1, m);
  a.o0[c][off] = r0;
  a.o1[c][off] = r1;
  d2.p[c][off] = r2;
}

// automorphism X -> X^g in the canonical NTT order (C11):
// out[j] = in[j'] with 2 brv(j') + 1 = g (2 brv(j) + 1) mod 2N.
struct Gal {
  u32 g[MAX_CTS];
};
__global__ void k_automorph(EwArgs a, Gal gal, int log_n, int both) {
  const u32 j = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y, c = blockIdx.z;
  if (j >= a.n) return;
  const u32 g = gal.g[c];
  const u32 mask = 2 * a.n - 1;
  const u32 e = (u32)(((u64)g * (2 * brv_dev(j, log_n) + 1)) & mask);
  const u32 jp = brv_dev((e - 1) >> 1, log_n);
  const size_t off = (size_t)l * a.n;
  a.o0[c][off + j] = a.x0[c][off + jp];
  if (both) a.o1[c][off + j] = a.x1[c][off + jp];
}

// rescale stage 1: lift_i = [last]_centred mod q_i (coefficient domain)
__global__ void k_rescale_lift(RescaleArgs r) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int i = blockIdx.y, c = blockIdx.z;
  if (k >= r.n) return;
  const u64 ql = r.mods[r.level].q;
  const ModInfo m = r.mods[i];
  for (int p = 0; p < 2; ++p) {
    const u64 v = r.last[c][(size_t)p * r.n + k];
    u64 res;
    if (v > (ql >> 1)) {
      const u64 mag = reduce128(0, ql - v, m);
      res = mag ? m.q - mag : 0;
    } else {
      res = reduce128(0, v, m);
    }
    r.lift[c][((size_t)p * r.level + i) * r.n + k] = res;
  }
}
// rescale stage 2: c_i = (c_i - lift_i) q_l^-1 (NTT domain), in place
__global__ void k_rescale_finish(RescaleArgs r) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int i = blockIdx.y, c = blockIdx.z;
  if (k >= r.n) return;
  const u64 q = r.mods[i].q;
  const u64 w = r.qlinv[2 * i], ws = r.qlinv[2 * i + 1];
  const size_t off = (size_t)i * r.n + k;
  const u64 l0 = r.lift[c][off], l1 = r.lift[c][(size_t)r.level * r.n + off];
  r.c0[c][off] = shoup(submod(r.c0[c][off], l0, q), w, ws, q);
  r.c1[c][off] = shoup(submod(r.c1[c][off], l1, q), w, ws, q);
}

// encryption (C5): c1 = a (uniform, NTT domain, key_a), c0 = pt + e - a s
__global__ void k_encrypt(EncArgs e) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y, c = blockIdx.z;
  if (k >= e.n) return;
  const ModInfo m = e.mods[t];
  const size_t off = (size_t)t * e.n + k;
  const u64 a = uniform_dev(e.key_a[c], (u64)t * e.n + k, m);
  const u64 as = mulmod(a, e.s_ntt[off], m);
  const u64 v = addmod(e.pt[c][off], e.err[c][off], m.q);
  e.c0[c][off] = submod(v, as, m.q);
  e.c1[c][off] = a;
}

// public-key encryption (C5, pk form): c0 = v b + pt + e0, c1 = v a + e1
__global__ void k_encrypt_pk(EncPkArgs e) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y;
  if (k >= e.n) return;
  const ModInfo m = e.mods[t];
  const size_t off = (size_t)t * e.n + k;
  const u64 v = e.v[off];
  e.c0[off] = addmod(addmod(mulmod(v, e.b[off], m), e.pt[off], m.q), e.e0[off], m.q);
  e.c1[off] = addmod(mulmod(v, e.a[off], m), e.e1[off], m.q);
}

__global__ void k_decrypt(EwArgs a, const u64 *s_ntt) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y, c = blockIdx.z;
  if (k >= a.n) return;
  const ModInfo m = a.mods[l];
  const size_t off = (size_t)l * a.n + k;
  a.o0[c][off] = addmod(a.x0[c][off], mulmod(a.x1[c][off], s_ntt[off], m), m.q);
}

__global__ void k_signed_to_res(const i64 *v, u64 *out, const ModInfo *mods, int first_mod, u32 n) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int l = blockIdx.y;
  if (k >= n) return;
  out[(size_t)l * n + k] = signed_res(v[k], mods[first_mod + l]);
}

// switching-key row for digit j: a uniform; b = -a s + e (+ [P]_{q_t} s' on the digit's limbs).
// Both are stored in Montgomery form (x 2^64 mod q_t), the form the key inner
// product's Montgomery reduction expects; ckks_debug_key converts back.
__global__ void k_keyrow(KeyArgs ka) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y;
  if (k >= ka.n) return;
  const ModInfo m = ka.mods[t];
  const size_t off = (size_t)t * ka.n + k;
  const u64 a = uniform_dev(ka.key_a, (u64)t * ka.n + k, m);
  u64 b = submod(ka.err[off], mulmod(a, ka.s_ntt[off], m), m.q);
  if (t >= ka.lo && t < ka.hi) b = addmod(b, mulmod(ka.p_mod[t], ka.sp_ntt[off], m), m.q);
  ka.b[off] = shoup(b, m.r64, m.r64_s, m.q);
  ka.a[off] = shoup(a, m.r64, m.r64_s, m.q);
}

__global__ void k_square(u64 *out, const u64 *in, const ModInfo *mods, u32 n) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int t = blockIdx.y;
  if (k >= n) return;
  const size_t off = (size_t)t * n + k;
  out[off] = mulmod(in[off], in[off], mods[t]);
}

struct WireArgs {
  u32 n;
  int nl;
  unsigned char bits[MAX_MODS];
  u32 off[MAX_MODS + 1];
  unsigned char *wire[MAX_CTS];
  u64 *ct[MAX_CTS];
  u32 n_limbs[MAX_CTS];
};

// A block takes one segment of WSEG residues of a limb.  WSEG is a multiple of
// 64, so the segment's bits [k0 b, (k0 + WSEG) b) start and end on 64-bit
// words: WSEG b / 64 words.  The segment is staged in shared memory with
// independent coalesced loads (WR per thread), then split or joined there.
constexpr int WR = 4;
constexpr int WSEG = TPB * WR;

// residue k of limb t: bits [k b, k b + b) of the limb's 64-bit words
__global__ void k_unpack(const WireArgs a) {
  __shared__ u64 sw[WSEG];
  const int t = blockIdx.y, i = blockIdx.z >> 1, pl = blockIdx.z & 1;
  const u32 b = a.bits[t];
  const u32 k0 = blockIdx.x * WSEG, nw = (WSEG / 64) * b;
  const u64 *src = reinterpret_cast<const u64 *>(a.wire[i] + (size_t)pl * a.off[a.nl] + a.off[t]) + (k0 / 64) * b;
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const u32 x = threadIdx.x + r * TPB;
    if (x < nw) sw[x] = __ldg(src + x);
  }
  __syncthreads();
  u64 *dst = a.ct[i] + ((size_t)pl * a.n_limbs[i] + t) * a.n + k0;
  const u64 mask = b < 64 ? (1ULL << b) - 1 : ~0ULL;
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const u32 k = threadIdx.x + r * TPB;
    const u32 o = k * b, w = o >> 6, sh = o & 63;  // w + 1 < nw whenever the residue straddles
    u64 v = sw[w] >> sh;
    if (sh + b > 64) v |= sw[w + 1] << (64 - sh);
    dst[k] = v & mask;
  }
}

// 64-bit word j of limb t: the residues overlapping bits [64 j, 64 j + 64)
__global__ void k_pack(const WireArgs a) {
  __shared__ u64 sr[WSEG];
  const int t = blockIdx.y, i = blockIdx.z >> 1, pl = blockIdx.z & 1;
  const u32 b = a.bits[t];
  const u32 k0 = blockIdx.x * WSEG, nw = (WSEG / 64) * b;
  const u64 *src = a.ct[i] + ((size_t)pl * a.n_limbs[i] + t) * a.n + k0;
#pragma unroll
  for (int r = 0; r < WR; ++r) sr[threadIdx.x + r * TPB] = __ldg(src + threadIdx.x + r * TPB);
  __syncthreads();
  u64 *dst = reinterpret_cast<u64 *>(a.wire[i] + (size_t)pl * a.off[a.nl] + a.off[t]) + (k0 / 64) * b;
  for (u32 j = threadIdx.x; j < nw; j += TPB) {
    const u32 lo_bit = j * 64u;  // segment-local bit offsets stay below WSEG * 64
    u64 acc = 0;
    for (u32 k = lo_bit / b; k < (u32)WSEG && k * b < lo_bit + 64u; ++k) {
      const int sft = (int)(k * b) - (int)lo_bit;
      const u64 v = sr[k];
      acc |= sft >= 0 ? v << sft : v >> (-sft);
    }
    dst[j] = acc;
  }
}

dim3 grid_for(u32 n, int limbs, int cts) { return dim3((n + TPB - 1) / TPB, limbs, cts); }
int last_status() { return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA; }

}  // namespace

WireLayout wire_layout(const ckks_ctx *c, int level) {
  WireLayout L;
  L.nl = level + 1;
  u32 off = 0;
  for (int t = 0; t < L.nl; ++t) {
    int b = 0;
    while (b < 64 && (c->mod[t] >> b)) ++b;
    L.bits[t] = (unsigned char)b;
    L.off[t] = off;
    off += (u32)((u64)c->n * b / 8);
  }
  L.off[L.nl] = off;
  return L;
}

int ew_wire(ckks_ctx *c, const WireLayout &L, unsigned char *const *wire, u64 *const *ct, const u32 *n_limbs,
            int ncts, bool to_wire) {
  if (ncts <= 0) return CKKS_OK;
  if (ncts > MAX_CTS || c->n % WSEG) return CKKS_E_PARAM;
  WireArgs a;
  a.n = c->n;
  a.nl = L.nl;
  for (int t = 0; t < L.nl; ++t) a.bits[t] = L.bits[t];
  for (int t = 0; t <= L.nl; ++t) a.off[t] = L.off[t];
  for (int i = 0; i < ncts; ++i) {
    if (((uintptr_t)wire[i] & 7) || n_limbs[i] < (u32)L.nl) return CKKS_E_PARAM;
    a.wire[i] = wire[i];
    a.ct[i] = ct[i];
    a.n_limbs[i] = n_limbs[i];
  }
  if (to_wire) {
    PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)L.nl * 2 * ncts,
                (k_pack<<<dim3(c->n / WSEG, L.nl, 2 * ncts), TPB, 0, c->stream>>>(a)));
  } else {
    PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)L.nl * 2 * ncts,
                (k_unpack<<<dim3(c->n / WSEG, L.nl, 2 * ncts), TPB, 0, c->stream>>>(a)));
  }
  return last_status();
}

int ew_addsub(ckks_ctx *c, EwArgs &a, int nl, int ncts, bool sub) {
  a.mods = c->d_mods;
  a.n = c->n;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl * ncts,
              (k_addsub<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(a, sub ? 1 : 0)));
  return last_status();
}
int ew_plain(ckks_ctx *c, EwArgs &a, int nl, int ncts, int mode) {
  a.mods = c->d_mods;
  a.n = c->n;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl * ncts,
              (k_plain<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(a, mode)));
  return last_status();
}
int ew_mul_int(ckks_ctx *c, EwArgs &a, int nl, int ncts, i64 k) {
  a.mods = c->d_mods;
  a.n = c->n;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl * ncts,
              (k_mul_int<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(a, k)));
  return last_status();
}
int ew_tensor(ckks_ctx *c, EwArgs &a, u64 *const *d2, int nl, int ncts) {
  a.mods = c->d_mods;
  a.n = c->n;
  D2Ptrs d;
  for (int i = 0; i < ncts; ++i) d.p[i] = d2[i];
  PROF_LAUNCH(c, PK_TENSOR, (u64)nl * ncts, (k_tensor<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(a, d)));
  return last_status();
}
int ew_automorph(ckks_ctx *c, EwArgs &a, const u32 *g, int nl, int ncts, bool both_polys) {
  a.mods = c->d_mods;
  a.n = c->n;
  Gal gal;
  for (int i = 0; i < ncts; ++i) gal.g[i] = g[i];
  PROF_LAUNCH(c, PK_AUTOMORPH, (u64)nl * ncts * (both_polys ? 2 : 1),
              (k_automorph<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(a, gal, c->log_n, both_polys ? 1 : 0)));
  return last_status();
}
int ew_decrypt(ckks_ctx *c, EwArgs &a, int nl, int ncts) {
  a.mods = c->d_mods;
  a.n = c->n;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl * ncts,
              (k_decrypt<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(a, c->d_s_ntt)));
  return last_status();
}
int ew_rescale_lift(ckks_ctx *c, RescaleArgs &r, int ncts) {
  r.mods = c->d_mods;
  r.n = c->n;
  PROF_LAUNCH(c, PK_RESCALE, (u64)r.level * ncts,
              (k_rescale_lift<<<grid_for(c->n, r.level, ncts), TPB, 0, c->stream>>>(r)));
  return last_status();
}
int ew_rescale_finish(ckks_ctx *c, RescaleArgs &r, int ncts) {
  r.mods = c->d_mods;
  r.n = c->n;
  PROF_LAUNCH(c, PK_RESCALE, (u64)r.level * ncts,
              (k_rescale_finish<<<grid_for(c->n, r.level, ncts), TPB, 0, c->stream>>>(r)));
  return last_status();
}
int ew_encrypt(ckks_ctx *c, EncArgs &e, int nl, int ncts) {
  e.mods = c->d_mods;
  e.n = c->n;
  e.s_ntt = c->d_s_ntt;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl * ncts, (k_encrypt<<<grid_for(c->n, nl, ncts), TPB, 0, c->stream>>>(e)));
  return last_status();
}
int ew_encrypt_pk(ckks_ctx *c, EncPkArgs &e, int nl) {
  e.mods = c->d_mods;
  e.n = c->n;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl, (k_encrypt_pk<<<grid_for(c->n, nl, 1), TPB, 0, c->stream>>>(e)));
  return last_status();
}
int ew_signed_to_res(ckks_ctx *c, const i64 *v, u64 *out, int first_mod, int nl) {
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl,
              (k_signed_to_res<<<grid_for(c->n, nl, 1), TPB, 0, c->stream>>>(v, out, c->d_mods, first_mod, c->n)));
  return last_status();
}
int ew_keyrow(ckks_ctx *c, KeyArgs &k, int nl) {
  k.mods = c->d_mods;
  k.n = c->n;
  k.s_ntt = c->d_s_ntt;
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl, (k_keyrow<<<grid_for(c->n, nl, 1), TPB, 0, c->stream>>>(k)));
  return last_status();
}
int ew_square(ckks_ctx *c, u64 *out, const u64 *in, int nl) {
  PROF_LAUNCH(c, PK_ELEMENTWISE, (u64)nl, (k_square<<<grid_for(c->n, nl, 1), TPB, 0, c->stream>>>(out, in, c->d_mods, c->n)));
  return last_status();
}
