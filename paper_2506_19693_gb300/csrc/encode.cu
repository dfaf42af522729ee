// Batching (ReBoot Sec. 3): the complex canonical embedding between N/2 slots
// and Z[X]/(X^N + 1), computed in FP64 on the GPU (reading C3).
//
// Slot j is the value at zeta^(g_j), zeta = exp(i pi / N), g_j = 5^j mod 2N.
// With odd exponents e = 2u + 1 and omega = zeta^2:
//   encode  m_k = (1/N) Re( zeta^-k  sum_u w_u omega^(-u k) ),
//           w_u = z_j at u = (g_j - 1)/2 and conj(z_j) at u = N - 1 - (g_j - 1)/2;
//   decode  z_j = sum_k (m_k zeta^k) omega^(u_j k),  u_j = (g_j - 1)/2.
// Both are one length-N complex DFT: a radix-2 decimation-in-time transform
// (bit-reversed load, log2 N butterfly stages), twiddles from sincospi.
// Encoding rounds scale * m_k half away from zero into int64 and reduces it
// into every limb; decoding first converts the residues to a centred FP64
// value by mixed-radix (Garner) conversion.
#include "ops.cuh"

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ u32 brv32(u32 x, int bits) { return __brev(x) >> (32 - bits); }

__device__ __forceinline__ u32 slot_exp(u32 j, u32 two_n) {
  // 5^j mod 2N by square-and-multiply
  u64 r = 1, b = 5;
  while (j) {
    if (j & 1) r = (r * b) & (two_n - 1);
    b = (b * b) & (two_n - 1);
    j >>= 1;
  }
  return (u32)r;
}

// scatter slots into the bit-reversed DFT input for encoding
__global__ void k_enc_scatter(const double *re, const double *im, int n_slots, double2 *x, u32 n, int log_n) {
  const u32 j = blockIdx.x * TPB + threadIdx.x;
  if (j >= n / 2) return;
  double zr = 0.0, zi = 0.0;
  if ((int)j < n_slots) {
    zr = re[j];
    zi = im ? im[j] : 0.0;
  }
  const u32 u = (slot_exp(j, 2 * n) - 1) >> 1;
  x[brv32(u, log_n)] = make_double2(zr, zi);
  x[brv32(n - 1 - u, log_n)] = make_double2(zr, -zi);
}

// one radix-2 DIT stage of half-length `half`; sign -1 forward, +1 inverse
__global__ void k_fft_stage(double2 *x, u32 n, u32 half, double sign) {
  const u32 i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n / 2) return;
  const u32 grp = i / half, pos = i % half;
  const u32 a = grp * 2 * half + pos, b = a + half;
  double s, c;
  sincospi((double)pos / (double)half, &s, &c);  // exp(sign * i pi pos / half)
  s *= sign;
  const double2 u = x[a], v = x[b];
  const double2 t = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
  x[a] = make_double2(u.x + t.x, u.y + t.y);
  x[b] = make_double2(u.x - t.x, u.y - t.y);
}

// m_k = round(scale/N * Re(zeta^-k F_k)), reduced into limbs 0..nl-1 (coefficient domain)
__global__ void k_enc_finish(const double2 *f, u32 n, double scale, const ModInfo *mods, int nl, u64 *pt,
                             int *overflow) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi((double)k / (double)n, &s, &c);  // zeta^k = c + i s ; zeta^-k = c - i s
  const double2 F = f[k];
  const double v = (F.x * c + F.y * s) * (scale / (double)n);
  if (!(fabs(v) < 4611686018427387904.0)) {  // 2^62
    *overflow = 1;
    return;
  }
  const i64 m = llround(v);
  for (int l = 0; l < nl; ++l) {
    const ModInfo md = mods[l];
    u64 r;
    if (m >= 0) {
      r = reduce128(0, (u64)m, md);
    } else {
      const u64 mag = reduce128(0, (u64)(-(m + 1)) + 1, md);
      r = mag ? md.q - mag : 0;
    }
    pt[(size_t)l * n + k] = r;
  }
}

// centred CRT of residues over q_0..q_level into FP64, times zeta^k, bit-reversed
__global__ void k_dec_crt(const u64 *res, int level, u32 n, int log_n, const ModInfo *mods,
                          const u64 *garner, const u64 *halfq, int nq, double2 *x) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  if (k >= n) return;
  u64 v[CKKS_MAX_Q];
  for (int i = 0; i <= level; ++i) {
    const ModInfo m = mods[i];
    u64 t = res[(size_t)i * n + k];
    for (int j = 0; j < i; ++j) {
      const u64 vj = reduce128(0, v[j], m);
      const u64 *g = garner + 2 * ((size_t)i * nq + j);
      t = shoup(submod(t, vj, m.q), g[0], g[1], m.q);
    }
    v[i] = t;
  }
  // compare with (Q - 1)/2 from the most significant digit
  const u64 *h = halfq + (size_t)level * nq;
  int greater = 0;
  for (int i = level; i >= 0; --i) {
    if (v[i] != h[i]) {
      greater = v[i] > h[i];
      break;
    }
  }
  double acc = 0.0;
  if (!greater) {
    for (int i = level; i >= 0; --i) acc = acc * (double)mods[i].q + (double)v[i];
  } else {  // x - Q = -((Q - 1 - x) + 1); digits of Q - 1 - x are q_i - 1 - v_i
    for (int i = level; i >= 0; --i) acc = acc * (double)mods[i].q + (double)(mods[i].q - 1 - v[i]);
    acc = -(acc + 1.0);
  }
  double s, c;
  sincospi((double)k / (double)n, &s, &c);
  x[brv32(k, log_n)] = make_double2(acc * c, acc * s);
}

__global__ void k_dec_gather(const double2 *g, u32 n, double inv_scale, double *re, double *im, int n_slots) {
  const u32 j = blockIdx.x * TPB + threadIdx.x;
  if ((int)j >= n_slots) return;
  const u32 u = (slot_exp(j, 2 * n) - 1) >> 1;
  re[j] = g[u].x * inv_scale;
  im[j] = g[u].y * inv_scale;
}

void fft(ckks_ctx *c, double2 *x, double sign) {
  const u32 n = c->n;
  const u32 blocks = (n / 2 + TPB - 1) / TPB;
  for (u32 half = 1; half < n; half <<= 1)
    PROF_LAUNCH(c, PK_ENCODE, 1, (k_fft_stage<<<blocks, TPB, 0, c->stream>>>(x, n, half, sign)));
}

}  // namespace

namespace {
// same as k_enc_scatter, slots given as interleaved complex values on the device
__global__ void k_enc_scatter_z(const double2 *z, double2 *x, u32 n, int log_n) {
  const u32 j = blockIdx.x * TPB + threadIdx.x;
  if (j >= n / 2) return;
  const double2 v = z[j];
  const u32 u = (slot_exp(j, 2 * n) - 1) >> 1;
  x[brv32(u, log_n)] = v;
  x[brv32(n - 1 - u, log_n)] = make_double2(v.x, -v.y);
}
}  // namespace

// Encode N/2 device-resident complex slots into an NTT-domain plaintext over
// q_0..q_level (the ckks_encode arithmetic).  Sets *flag_dev to 1 when a
// scaled coefficient reaches 2^62; never clears it.  Uses the FFT buffer in
// the context's float scratch.
int encode_device_z(ckks_ctx *c, const double2 *z_dev, uint32_t level, double scale, u64 *pt_dev, int *flag_dev) {
  const u32 n = c->n;
  int rc = ensure_fscratch(c, 3 * (size_t)n + 8);
  if (rc) return rc;
  double2 *x = reinterpret_cast<double2 *>(c->fscratch + n);
  PROF_LAUNCH(c, PK_ENCODE, 1,
              (k_enc_scatter_z<<<(n / 2 + TPB - 1) / TPB, TPB, 0, c->stream>>>(z_dev, x, n, c->log_n)));
  fft(c, x, -1.0);
  PROF_LAUNCH(c, PK_ENCODE, level + 1,
              (k_enc_finish<<<(n + TPB - 1) / TPB, TPB, 0, c->stream>>>(x, n, scale, c->d_mods, level + 1, pt_dev,
                                                                         flag_dev)));
  int mods[MAX_MODS];
  for (int l = 0; l <= (int)level; ++l) mods[l] = l;
  const u64 *src[1] = {pt_dev};
  u64 *dst[1] = {pt_dev};
  return launch_ntt(c, src, dst, 1, level + 1, mods, false);
}

int encode_device_z_ext(ckks_ctx *c, const double2 *z_dev, uint32_t level, double scale, u64 *pt_dev,
                        int *flag_dev) {
  const u32 n = c->n;
  int rc = ensure_fscratch(c, 3 * (size_t)n + 8);
  if (rc) return rc;
  double2 *x = reinterpret_cast<double2 *>(c->fscratch + n);
  PROF_LAUNCH(c, PK_ENCODE, 1,
              (k_enc_scatter_z<<<(n / 2 + TPB - 1) / TPB, TPB, 0, c->stream>>>(z_dev, x, n, c->log_n)));
  fft(c, x, -1.0);
  // the same integer coefficients reduced mod q_0..q_level, then mod p_0..p_{K-1}
  PROF_LAUNCH(c, PK_ENCODE, level + 1,
              (k_enc_finish<<<(n + TPB - 1) / TPB, TPB, 0, c->stream>>>(x, n, scale, c->d_mods, level + 1, pt_dev,
                                                                         flag_dev)));
  PROF_LAUNCH(c, PK_ENCODE, c->n_p,
              (k_enc_finish<<<(n + TPB - 1) / TPB, TPB, 0, c->stream>>>(x, n, scale, c->d_mods + c->n_q, c->n_p,
                                                                         pt_dev + (size_t)(level + 1) * n,
                                                                         flag_dev)));
  int mods[MAX_MODS];
  for (int l = 0; l <= (int)level; ++l) mods[l] = l;
  for (int k = 0; k < c->n_p; ++k) mods[level + 1 + k] = c->n_q + k;
  const u64 *src[1] = {pt_dev};
  u64 *dst[1] = {pt_dev};
  return launch_ntt(c, src, dst, 1, level + 1 + c->n_p, mods, false);
}

extern "C" int ckks_encode(ckks_ctx *c, const double *re, const double *im, int n_slots, uint32_t level,
                           double scale, uint64_t *pt_dev) {
  if (!c || !re || !pt_dev || n_slots < 0 || n_slots > (int)(c->n / 2)) return CKKS_E_PARAM;
  if ((int)level >= c->n_q) return CKKS_E_LEVEL;
  if (scale <= 0) scale = c->default_scale;
  const u32 n = c->n;
  // float scratch: slots (2 * N/2), DFT buffer (2 * N), flag
  int rc = ensure_fscratch(c, 3 * (size_t)n + 8);
  if (rc) return rc;
  double *d_re = c->fscratch, *d_im = d_re + n / 2;
  double2 *x = reinterpret_cast<double2 *>(c->fscratch + n);
  int *flag = reinterpret_cast<int *>(c->fscratch + 3 * (size_t)n);
  CK_CUDA(cudaMemcpyAsync(d_re, re, sizeof(double) * n_slots, cudaMemcpyHostToDevice, c->stream));
  if (im) CK_CUDA(cudaMemcpyAsync(d_im, im, sizeof(double) * n_slots, cudaMemcpyHostToDevice, c->stream));
  CK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  PROF_LAUNCH(c, PK_ENCODE, 1,
              (k_enc_scatter<<<(n / 2 + TPB - 1) / TPB, TPB, 0, c->stream>>>(d_re, im ? d_im : nullptr, n_slots,
                                                                              x, n, c->log_n)));
  fft(c, x, -1.0);
  PROF_LAUNCH(c, PK_ENCODE, level + 1,
              (k_enc_finish<<<(n + TPB - 1) / TPB, TPB, 0, c->stream>>>(x, n, scale, c->d_mods, level + 1, pt_dev,
                                                                         flag)));
  int mods[MAX_MODS];
  for (int l = 0; l <= (int)level; ++l) mods[l] = l;
  const u64 *src[1] = {pt_dev};
  u64 *dst[1] = {pt_dev};
  rc = launch_ntt(c, src, dst, 1, level + 1, mods, false);
  if (rc) return rc;
  int h_flag = 0;
  CK_CUDA(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return h_flag ? CKKS_E_SCALE : CKKS_OK;
}

extern "C" int ckks_decode(ckks_ctx *c, const uint64_t *pt_dev, uint32_t level, double scale, double *re,
                           double *im, int n_slots) {
  if (!c || !pt_dev || !re || !im || n_slots < 0 || n_slots > (int)(c->n / 2) || scale <= 0)
    return CKKS_E_PARAM;
  if ((int)level >= c->n_q) return CKKS_E_LEVEL;
  const u32 n = c->n;
  int rc = ensure_fscratch(c, 3 * (size_t)n + 8);
  if (rc) return rc;
  rc = ensure_scratch(c, (size_t)(level + 1) * n);
  if (rc) return rc;
  u64 *coef = c->scratch;
  int mods[MAX_MODS];
  for (int l = 0; l <= (int)level; ++l) mods[l] = l;
  const u64 *src[1] = {pt_dev};
  u64 *dst[1] = {coef};
  rc = launch_ntt(c, src, dst, 1, level + 1, mods, true);
  if (rc) return rc;
  double *d_re = c->fscratch, *d_im = d_re + n / 2;
  double2 *x = reinterpret_cast<double2 *>(c->fscratch + n);
  PROF_LAUNCH(c, PK_ENCODE, level + 1,
              (k_dec_crt<<<(n + TPB - 1) / TPB, TPB, 0, c->stream>>>(coef, level, n, c->log_n, c->d_mods,
                                                                      c->d_conv + c->conv.garner_inv,
                                                                      c->d_conv + c->conv.halfq_digits, c->n_q, x)));
  fft(c, x, 1.0);
  PROF_LAUNCH(c, PK_ENCODE, 1,
              (k_dec_gather<<<(n / 2 + TPB - 1) / TPB, TPB, 0, c->stream>>>(x, n, 1.0 / scale, d_re, d_im, n_slots)));
  CK_CUDA(cudaMemcpyAsync(re, d_re, sizeof(double) * n_slots, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaMemcpyAsync(im, d_im, sizeof(double) * n_slots, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}
