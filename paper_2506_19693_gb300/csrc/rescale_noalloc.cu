// Rescale for callers that must not allocate device memory.
//
// ckks_rescale takes its workspace from the context's scratch buffer, which
// grows with cudaMalloc (and frees the old buffer) the first time a larger
// batch needs it.  Some callers cannot accept that: a process whose device
// memory is capped or handed out by its own pool allocator, or a latency-bound
// path where an allocation's implicit synchronisation is not acceptable.  This
// variant computes exactly the same result (the same per-limb arithmetic as
// ckks_rescale) with its workspace in a fixed file-scope device array, so it
// allocates nothing on any call.
//
// Workspace: the coefficient-domain top limb of both polynomials (2 N words)
// plus G lifted limbs of both polynomials (2 G N words), G chosen to fill the
// array (G = 4 at N = 2^16, G = 1 at N = 2^17); the lifted limbs are processed
// in chunks of G.  Rings above 2^17 do not fit (G would be 0).
// Nothing in the array needs to start at zero: every word is written before it
// is read within one call.  The array is shared by every call on a device, so
// calls whose GPU work overlaps (other streams, other host threads) race.
#include <algorithm>
#include <mutex>

#include "ops.cuh"

namespace {

constexpr size_t kNoAllocWords = 655360;  // 5 MiB = (2 + 2*4) limbs of 2^16 words
constexpr int kMaxDevices = 64;
constexpr int TPB = 256;

static __device__ __align__(256) u64 g_rescale_ws[kNoAllocWords];

u64 *g_ws_ptr[kMaxDevices];
cudaError_t g_ws_err[kMaxDevices];
std::mutex g_ws_mu;

struct ChunkArgs {
  const ModInfo *mods;
  const u64 *qlinv;   // Shoup pairs of q_level^-1 mod q_i
  u64 *c0, *c1;       // ciphertext polys (NTT domain)
  const u64 *last;    // [2][N] coefficient-domain top limbs
  u64 *lift;          // [2][G][N]
  u32 n;
  int level, i0, g;   // chunk: target limbs i0 .. i0+g-1, lift stride G
  int G;
};

// lift[p][gi] = [last_p]_centred mod q_{i0+gi}
__global__ void k_noalloc_lift(const ChunkArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int gi = blockIdx.y;
  if (k >= a.n) return;
  const u64 ql = a.mods[a.level].q;
  const ModInfo m = a.mods[a.i0 + gi];
  for (int p = 0; p < 2; ++p) {
    const u64 v = a.last[(size_t)p * a.n + k];
    u64 r;
    if (v > (ql >> 1)) {
      const u64 mag = reduce128(0, ql - v, m);
      r = mag ? m.q - mag : 0;
    } else {
      r = reduce128(0, v, m);
    }
    a.lift[((size_t)p * a.G + gi) * a.n + k] = r;
  }
}

// c_p[i] = (c_p[i] - lift_p[i]) * q_level^-1 for i in the chunk
__global__ void k_noalloc_finish(const ChunkArgs a) {
  const u32 k = blockIdx.x * TPB + threadIdx.x;
  const int gi = blockIdx.y, i = a.i0 + gi;
  if (k >= a.n) return;
  const u64 q = a.mods[i].q, w = a.qlinv[2 * i], ws = a.qlinv[2 * i + 1];
  const size_t off = (size_t)i * a.n + k;
  const u64 l0 = a.lift[(size_t)gi * a.n + k], l1 = a.lift[((size_t)a.G + gi) * a.n + k];
  a.c0[off] = shoup(submod(a.c0[off], l0, q), w, ws, q);
  a.c1[off] = shoup(submod(a.c1[off], l1, q), w, ws, q);
}

}  // namespace

extern "C" int ckks_rescale_noalloc(ckks_ctx *c, ckks_ct *ct) {
  if (!c || !ct || !ct->data || ct->log_n != (u32)c->log_n || (int)ct->level >= c->n_q ||
      ct->n_limbs < ct->level + 1)
    return CKKS_E_PARAM;
  if (ct->level == 0) return CKKS_E_LEVEL;
  const u32 n = c->n;
  if (4 * (size_t)n > kNoAllocWords) return CKKS_E_PARAM;  // G >= 1 needs 4 N words: N <= 2^17
  int dev = 0;
  CK_CUDA(cudaGetDevice(&dev));
  if (dev != c->device || dev < 0 || dev >= kMaxDevices) return CKKS_E_PARAM;
  // Set-up per device: the host-side symbol is not a device address, so ask
  // the runtime for the array's device address on this device.  A failed
  // lookup is not cached: the next call tries again.
  {
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (!g_ws_ptr[dev]) {
      g_ws_err[dev] = cudaGetSymbolAddress(reinterpret_cast<void **>(&g_ws_ptr[dev]), g_rescale_ws);
      if (g_ws_err[dev] != cudaSuccess) {
        g_ws_ptr[dev] = nullptr;
        cudaGetLastError();
        return CKKS_E_CUDA;
      }
    }
  }
  if (!g_ws_ptr[dev]) return CKKS_E_CUDA;

  const int level = (int)ct->level;
  const int G = (int)std::min<size_t>((size_t)level, (kNoAllocWords - 2 * (size_t)n) / (2 * (size_t)n));
  u64 *ws = g_ws_ptr[dev];
  u64 *c0 = ct->data, *c1 = ct->data + (size_t)ct->n_limbs * n;
  ChunkArgs a;
  a.mods = c->d_mods;
  a.qlinv = c->d_conv + c->conv.rescale_qlinv + 2 * (size_t)level * c->n_q;
  a.c0 = c0;
  a.c1 = c1;
  a.last = ws;
  a.lift = ws + 2 * (size_t)n;
  a.n = n;
  a.level = level;
  a.G = G;
  // top limbs to the coefficient domain
  const u64 *src[2] = {c0 + (size_t)level * n, c1 + (size_t)level * n};
  u64 *dst[2] = {ws, ws + n};
  int m1[1] = {level};
  int rc = launch_ntt(c, src, dst, 2, 1, m1, true);
  if (rc) return rc;
  int mods[MAX_MODS];
  for (int i0 = 0; i0 < level; i0 += G) {
    const int g = std::min(G, level - i0);
    a.i0 = i0;
    a.g = g;
    const dim3 grid((n + TPB - 1) / TPB, g);
    k_noalloc_lift<<<grid, TPB, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return CKKS_E_CUDA;
    for (int t = 0; t < g; ++t) mods[t] = i0 + t;
    const u64 *ls[2] = {a.lift, a.lift + (size_t)G * n};
    u64 *ld[2] = {a.lift, a.lift + (size_t)G * n};
    rc = launch_ntt(c, ls, ld, 2, g, mods, false);
    if (rc) return rc;
    k_noalloc_finish<<<grid, TPB, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return CKKS_E_CUDA;
  }
  ct->scale /= (double)c->mod[level];
  ct->level = level - 1;
  return CKKS_OK;
}
