// Integer-pipe peaks for the roofline of the ALU-bound kernels: the same
// 64x64->128 multiply-accumulate (basis conversion, key inner product) and the
// same Shoup butterfly (NTT) as the production kernels, in registers only, with
// eight independent chains per thread and a grid of several waves.
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
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      u64 pl = a[c] * b[c], ph = __umul64hi(a[c], b[c]);
      lo[c] += pl;
      hi[c] += ph + (lo[c] < pl ? 1 : 0);
      a[c] ^= lo[c];
    }
  }
  u64 r = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) r ^= hi[c] ^ lo[c];
  if (r == 0x123456789ULL) sink[t] = r;  // keeps the chains live
}

__global__ void __launch_bounds__(TPB) k_peak_bfly(u64 *sink, u64 q, u64 w, u64 ws, int iters) {
  const u64 t = blockIdx.x * (u64)TPB + threadIdx.x;
  const u64 twoq = 2 * q;
  u64 x[CHAINS], y[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    x[c] = (t * 7 + c) % q;
    y[c] = (t * 13 + 5 * c) % q;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      u64 xx = x[c];
      if (xx >= twoq) xx -= twoq;
      const u64 s = w * y[c] - __umul64hi(ws, y[c]) * q;
      x[c] = xx + s;
      y[c] = xx + twoq - s;
    }
  }
  u64 r = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) r ^= x[c] ^ y[c];
  if (r == 0x123456789ULL) sink[t] = r;
}

}  // namespace

extern "C" int ckks_alu_peaks(ckks_ctx *c, double *mac_per_s, double *bfly_per_s) {
  if (!c) return CKKS_E_PARAM;
  int dev = 0, sms = 0;
  CK_CUDA(cudaGetDevice(&dev));
  CK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8 * 4;  // 4 waves at 8 resident CTAs of 256 threads
  const int iters = 2048;
  int rc = ensure_scratch(c, (size_t)blocks * TPB);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  CK_CUDA(cudaEventCreate(&e0));
  CK_CUDA(cudaEventCreate(&e1));
  const u64 q = c->mod[0], w = c->mod[0] / 3, ws = host_shoup(w, q);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {  // first run warms up
    cudaEventRecord(e0, c->stream);
    k_peak_mac<<<blocks, TPB, 0, c->stream>>>(c->scratch, 0x1234567ULL + rep, iters);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
  }
  cudaEventElapsedTime(&ms, e0, e1);
  if (mac_per_s) *mac_per_s = (double)blocks * TPB * iters * CHAINS / (ms * 1e-3);
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0, c->stream);
    k_peak_bfly<<<blocks, TPB, 0, c->stream>>>(c->scratch, q, w, ws, iters);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
  }
  cudaEventElapsedTime(&ms, e0, e1);
  if (bfly_per_s) *bfly_per_s = (double)blocks * TPB * iters * CHAINS / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}
