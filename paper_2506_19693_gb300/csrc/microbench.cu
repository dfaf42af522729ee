// Integer-pipe roofs for the ALU-bound kernels, measured on this GPU with the
// production instruction sequences themselves (common.cuh): the 128-bit
// multiply-accumulate of the basis conversion and the key inner product
// (mac128, with a multiplicand that changes every iteration), and the NTT's
// butterflies (bfly_fwd_loose for primes with
// 65 q < 2^64, bfly_fwd_strict for the others, bfly_inv<true> for the inverse
// below 2^61).  Register-only kernels: eight independent chains per thread,
// 256-thread CTAs at the occupancy the sequence allows, several waves; no
// memory traffic, so the rate is the issue/ALU ceiling of that sequence.
#include "ctx.h"

namespace {

constexpr int TPB = 256;
constexpr int CHAINS = 8;

__global__ void __launch_bounds__(TPB) k_peak_mac(u64 *sink, u64 seed, int iters) {
  const u64 t = blockIdx.x * (u64)TPB + threadIdx.x;
  u64 a[CHAINS], b[CHAINS], hi[CHAINS], lo[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    a[c] = (seed ^ (t * 0x9E3779B97F4A7C15ULL)) + c;
    b[c] = (seed * (c + 3)) | 1;
    hi[c] = lo[c] = 0;
  }
  for (int it = 0; it < iters; ++it) {
    // a multiplicand that changes every iteration (both halves), so that no
    // partial product of the 64 x 64 multiply is loop-invariant; the XOR
    // stands in for the operand load each production MAC pays
    const u64 salt = (u64)it * 0x9E3779B97F4A7C15ULL;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) mac128(hi[c], lo[c], a[c] ^ salt, b[c]);
  }
  u64 r = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) r ^= hi[c] ^ lo[c];
  if (r == 0x123456789ULL) sink[t] = r;  // keeps the chains live
}

// kind 0: forward loose, 1: forward strict, 2: inverse (approximate quotient),
// 3: inverse (exact quotient)
template <int KIND>
__global__ void __launch_bounds__(TPB) k_peak_bfly(u64 *sink, u64 q, u64 w, u64 ws, int iters) {
  const u64 t = blockIdx.x * (u64)TPB + threadIdx.x;
  const u64 twoq = 2 * q, r4 = 4 * q;
  u64 x[CHAINS], y[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    x[c] = (t * 7 + c) % q;
    y[c] = (t * 13 + 5 * c) % q;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      if (KIND == 0) bfly_fwd_loose(x[c], y[c], w, ws, q, twoq);
      if (KIND == 1) bfly_fwd_strict(x[c], y[c], w, ws, q, twoq);
      if (KIND == 2) bfly_inv<true>(x[c], y[c], w, ws, q, r4);
      if (KIND == 3) bfly_inv<false>(x[c], y[c], w, ws, q, twoq);
    }
  }
  u64 r = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) r ^= x[c] ^ y[c];
  if (r == 0x123456789ULL) sink[t] = r;
}

template <class F>
int time_kernel(ckks_ctx *c, F launch, double units, double *out) {
  cudaEvent_t e0, e1;
  CK_CUDA(cudaEventCreate(&e0));
  CK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  for (int rep = 0; rep < 3; ++rep) {  // the first run warms up; keep the faster of the others
    cudaEventRecord(e0, c->stream);
    launch();
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 1 || (rep > 1 && ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out) *out = units / (best * 1e-3);
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

}  // namespace

extern "C" int ckks_alu_peaks(ckks_ctx *c, double *out, int cap) {
  if (!c || cap < 0 || (cap > 0 && !out)) return CKKS_E_PARAM;
  int dev = 0, sms = 0;
  CK_CUDA(cudaGetDevice(&dev));
  CK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8 * 4;  // 4 waves at 8 resident CTAs of 256 threads
  const int iters = 2048;
  int rc = ensure_scratch(c, (size_t)blocks * TPB);
  if (rc) return rc;
  const double units = (double)blocks * TPB * iters * CHAINS;
  u64 *sink = c->scratch;
  cudaStream_t st = c->stream;
  const u64 q = c->mod[c->n_q > 1 ? 1 : 0], w = q / 3, ws = host_shoup(w, q);
  double r[5] = {0, 0, 0, 0, 0};
  rc = time_kernel(c, [&] { k_peak_mac<<<blocks, TPB, 0, st>>>(sink, 0x1234567ULL, iters); }, units, &r[0]);
  if (!rc) rc = time_kernel(c, [&] { k_peak_bfly<0><<<blocks, TPB, 0, st>>>(sink, q, w, ws, iters); }, units, &r[1]);
  if (!rc) rc = time_kernel(c, [&] { k_peak_bfly<1><<<blocks, TPB, 0, st>>>(sink, q, w, ws, iters); }, units, &r[2]);
  if (!rc) rc = time_kernel(c, [&] { k_peak_bfly<2><<<blocks, TPB, 0, st>>>(sink, q, w, ws, iters); }, units, &r[3]);
  if (!rc) rc = time_kernel(c, [&] { k_peak_bfly<3><<<blocks, TPB, 0, st>>>(sink, q, w, ws, iters); }, units, &r[4]);
  if (rc) return rc;
  for (int i = 0; i < cap && i < 5; ++i) out[i] = r[i];
  return 5;
}
