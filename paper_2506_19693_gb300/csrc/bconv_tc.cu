// Fast basis conversion (reading C8) on the 5th-generation tensor cores,
// exact, as a byte-split GEMM.
//
//   y_t = sum_i y_i * c_(i,t)  mod t,   y_i = [x_i Bhat_i^-1]_(b_i) < 2^62,
//   c_(i,t) = Bhat_i mod t.
// Split y_i into bytes y_(i,a) (y_i = sum_a y_(i,a) 2^(8a)) and fold 2^(8a) into
// the constant: c'_(i,a,t) = 2^(8a) c_(i,t) mod t; split c' into bytes
// c'_(i,a,t,b).  Then
//   y_t = sum_b 2^(8b) sum_(i,a) y_(i,a) c'_(i,a,t,b)   mod t,
// where the inner sum is a GEMM  D[n][(t,b)] = sum_(i,a) A[n][(i,a)] B[(t,b)][(i,a)]
// with 8-bit operands (exact in fp16) and K = 8 * sources <= 128 terms, so every
// accumulator is an integer below 128 * 255 * 255 < 2^23, exact in fp32.  The
// epilogue recombines the 8 byte planes of each target in 128-bit integers and
// reduces mod t: bit-identical to the uint64 kernel.
//
// GB300 mapping: one CTA owns a 128 x N accumulator in tensor memory (TMEM,
// N = 8 * targets rounded up to 16 <= 256 columns).  Per tile of 128
// coefficients, all 128 threads compute y_i for their coefficient and write its
// bytes into the shared-memory A tile (canonical K-major, no swizzle); one
// thread issues K/16 tcgen05.mma (kind::f16, fp32 accumulate) and commits them
// to an mbarrier; each warp then reads its 32 TMEM lanes with tcgen05.ld and
// finishes its 32 coefficients.  B (the constants) is loaded into shared memory
// once per CTA.  Every wait is bounded: on expiry the kernel records an error
// flag, frees its TMEM and returns.
#include <cuda_fp16.h>

#include <algorithm>

#include "ops.cuh"

namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_TMEM_COLS = 256;
constexpr u64 TC_WAIT_NS = 1000000000ULL;  // bounded waits give up after about 1 s

__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u64 global_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin on an mbarrier phase for at most TC_WAIT_NS; 1 when the phase completed.
__device__ __forceinline__ u32 wait_parity(u32 mbar_addr, u32 phase) {
  const u64 t0 = global_ns();
  u32 done = 0;
  while (!done) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(mbar_addr), "r"(phase));
    if (!done && global_ns() - t0 > TC_WAIT_NS) break;
  }
  return done;
}

// Canonical K-major, no-swizzle layout of an R x K fp16 operand: core matrices of
// 8 rows x 8 elements (16 bytes per row, 128 bytes each); adjacent along K at
// LBO = 128 bytes, adjacent along R at SBO = K/8 * 128 bytes.
__device__ __forceinline__ u32 canon_offset(int row, int k, int kpad) {
  return (u32)((row >> 3) * (kpad / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ u64 make_desc(u32 saddr, u32 lbo, u32 sbo) {
  return (u64)((saddr >> 4) & 0x3FFF) | ((u64)((lbo >> 4) & 0x3FFF) << 16) | ((u64)((sbo >> 4) & 0x3FFF) << 32) |
         (1ULL << 46);  // descriptor version 1; base offset 0; no swizzle
}

struct TcArgs {
  const ModInfo *mods;
  u32 n;
  int ns, nt, kpad, npad;
  const u64 *inv;                   // [ns] pairs: [Bhat_i^-1]_{b_i}, Shoup
  const __half *bmat;               // [npad][kpad] row-major constants (bytes)
  unsigned char src_mod[16];
  unsigned char dst_mod[MAX_MODS];
  unsigned char dst_pos[MAX_MODS];
  const u64 *src[MAX_CTS];
  u64 *dst[MAX_CTS];
  int np;
  int *err;                         // set to 1 when a bounded wait expires
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_bconv_tc(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __half *sA = reinterpret_cast<__half *>(smem);                               // 128 x kpad
  __half *sB = reinterpret_cast<__half *>(smem + TC_M * a.kpad * 2);           // npad x kpad
  u64 *mbar = reinterpret_cast<u64 *>(smem + TC_M * a.kpad * 2 + a.npad * a.kpad * 2);
  u32 *tmem_slot = reinterpret_cast<u32 *>(mbar + 1);

  // constants into the canonical layout
  for (int idx = tid; idx < a.npad * a.kpad; idx += TC_THREADS) {
    const int r = idx / a.kpad, k = idx % a.kpad;
    *reinterpret_cast<__half *>(reinterpret_cast<unsigned char *>(sB) + canon_offset(r, k, a.kpad)) = a.bmat[idx];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const u32 tmem = *tmem_slot;

  // instruction descriptor: D fp32, A and B fp16, both K-major, M = 128, N = npad
  const u32 idesc = (1u << 4) | ((u32)(a.npad >> 3) << 17) | ((u32)(TC_M >> 4) << 24);
  const u32 sA_addr = smem_u32(sA), sB_addr = smem_u32(sB);
  const u32 sbo = (u32)(a.kpad / 8) * 128;
  u32 phase = 0;
  bool failed = false;

  const int tiles_per_poly = a.n / TC_M;
  const int total = tiles_per_poly * a.np;
  for (int tile = blockIdx.x; tile < total && !failed; tile += gridDim.x) {
    const int p = tile / tiles_per_poly;
    const u32 k0 = (u32)(tile % tiles_per_poly) * TC_M;
    const u32 kc = k0 + tid;
    // A row tid: the bytes of y_i for coefficient kc
    const u64 *src = a.src[p];
    unsigned char *rowbase = reinterpret_cast<unsigned char *>(sA);
    for (int i = 0; i < a.kpad / 8; ++i) {  // core-matrix column i holds the 8 bytes of y_i
      u64 y = 0;
      if (i < a.ns) {
        const u64 q = a.mods[a.src_mod[i]].q;
        y = shoup(src[(size_t)i * a.n + kc], a.inv[2 * i], a.inv[2 * i + 1], q);
      }
      __align__(16) __half h[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) h[b] = __uint2half_rn((unsigned)((y >> (8 * b)) & 0xFF));
      *reinterpret_cast<uint4 *>(rowbase + canon_offset(tid, i * 8, a.kpad)) = *reinterpret_cast<uint4 *>(h);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      for (int kk = 0; kk < a.kpad / 16; ++kk) {
        const u64 ad = make_desc(sA_addr + kk * 256, 128, sbo);
        const u64 bd = make_desc(sB_addr + kk * 256, 128, sbo);
        const u32 acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar)));
    }
    // bounded wait for the MMAs; the outcome is agreed by the whole CTA
    const u32 done = wait_parity(smem_u32(mbar), phase);
    if (__syncthreads_or(done == 0)) {
      failed = true;
      break;
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = coefficients k0 + 32w + lane
    u64 *dst = a.dst[p];
    for (int t = 0; t < a.nt; ++t) {
      u32 v[8];
      const u32 taddr = tmem + ((u32)(warp * 32) << 16) + (u32)(t * 8);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      u64 lo = 0, hi = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const u64 x = (u64)__float2uint_rn(__uint_as_float(v[b]));  // exact integer < 2^23
        const u64 sl = b ? x << (8 * b) : x, sh = b > 0 && 8 * b > 40 ? x >> (64 - 8 * b) : 0;
        lo += sl;
        hi += sh + (lo < sl ? 1 : 0);
      }
      dst[(size_t)a.dst_pos[t] * a.n + k0 + warp * 32 + lane] = reduce128(hi, lo, a.mods[a.dst_mod[t]]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // A tile and accumulator are reused by the next tile
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (failed) {
    // record the error, give the MMAs in flight one more bounded wait, then free TMEM
    if (tid == 0) atomicExch(a.err, 1);
    wait_parity(smem_u32(mbar), phase);
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

}  // namespace

// Host: the byte-plane constant matrix of one conversion, cached on the device
// (built on first use, outside any graph capture), then the launch.
// key identifies the conversion (table offset); tab_host rows are [nt][ns].
int launch_bconv_tc(ckks_ctx *c, size_t key, const u64 *inv_dev, const u64 *tab_host, int ns, int nt,
                    const int *src_mod, const int *dst_mod, const int *dst_pos, const u64 *const *src,
                    u64 *const *dst, int np) {
  if (ns < 1 || ns > 16 || nt < 1 || 8 * nt > TC_TMEM_COLS || np < 1 || np > MAX_CTS) return CKKS_E_PARAM;
  if (c->n % TC_M) return CKKS_E_PARAM;
  const int kpad = ((8 * ns + 15) / 16) * 16, npad = ((8 * nt + 15) / 16) * 16;
  if (!c->tc_err) {
    if (c->capturing) return CKKS_E_STATE;
    if (cudaMalloc(&c->tc_err, sizeof(int)) != cudaSuccess) return CKKS_E_OOM;
    CK_CUDA(cudaMemset(c->tc_err, 0, sizeof(int)));
  }
  auto it = c->tc_bmats.find(key);
  if (it == c->tc_bmats.end()) {
    if (c->capturing) return CKKS_E_STATE;
    // B[(t,b)][(i,a)] = byte b of (2^(8a) * c_(i,t) mod t)
    std::vector<__half> bm((size_t)npad * kpad, __float2half(0.f));
    for (int t = 0; t < nt; ++t) {
      const u64 m = c->mod[dst_mod[t]];
      for (int i = 0; i < ns; ++i) {
        const u64 cc = tab_host[(size_t)t * ns + i] % m;
        for (int aa = 0; aa < 8; ++aa) {
          const u64 cf = host_mulmod(cc, host_powmod(2, 8 * aa, m), m);
          for (int b = 0; b < 8; ++b)
            bm[(size_t)(t * 8 + b) * kpad + i * 8 + aa] = __float2half((float)((cf >> (8 * b)) & 0xFF));
        }
      }
    }
    void *d = nullptr;
    if (cudaMalloc(&d, bm.size() * sizeof(__half)) != cudaSuccess) return CKKS_E_OOM;
    CK_CUDA(cudaMemcpy(d, bm.data(), bm.size() * sizeof(__half), cudaMemcpyHostToDevice));
    it = c->tc_bmats.emplace(key, d).first;
  }
  TcArgs a;
  a.mods = c->d_mods;
  a.n = c->n;
  a.ns = ns;
  a.nt = nt;
  a.kpad = kpad;
  a.npad = npad;
  a.inv = inv_dev;
  a.bmat = reinterpret_cast<const __half *>(it->second);
  for (int i = 0; i < ns; ++i) a.src_mod[i] = (unsigned char)src_mod[i];
  for (int t = 0; t < nt; ++t) {
    a.dst_mod[t] = (unsigned char)dst_mod[t];
    a.dst_pos[t] = (unsigned char)dst_pos[t];
  }
  for (int i = 0; i < np; ++i) {
    a.src[i] = src[i];
    a.dst[i] = dst[i];
  }
  a.np = np;
  a.err = c->tc_err;
  // at least 100 KB of shared memory per CTA: at most two CTAs share an SM, so
  // their two 256-column TMEM allocations always fit the SM's 512 columns
  const size_t need = (size_t)TC_M * kpad * 2 + (size_t)npad * kpad * 2 + 16;
  const size_t smem = std::max<size_t>(need, 100 * 1024);
  CK_CUDA(cudaFuncSetAttribute(k_bconv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int total = (int)(c->n / TC_M) * np;
  const int grid = std::min(total, 2 * sms);
  PROF_LAUNCH(c, PK_BCONV_TC, (u64)np * nt * ns, (k_bconv_tc<<<grid, TC_THREADS, smem, c->stream>>>(a)));
  return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}
