// Per-kernel-class launch accounting: a launch counter that is always on and,
// when enabled, a CUDA event pair around every launch on the context stream so
// that device time per kernel class can be read back (ckks_ctx_profile_read).
#pragma once

#include <vector>

#include "common.cuh"

enum ProfKind {
  PK_NTT_FWD_A = 0,
  PK_NTT_FWD_B,
  PK_NTT_INV_A,
  PK_NTT_INV_B,
  PK_BCONV,
  PK_INNER,
  PK_COMBINE,
  PK_TENSOR,
  PK_AUTOMORPH,
  PK_RESCALE,
  PK_ELEMENTWISE,
  PK_ENCODE,
  PK_BCONV_TC,
  PK_BOOT_MAC,        // units: limbs of N words moved (algorithmic)
  PK_BOOT_LINCOMB,    // units: limbs of N words moved (algorithmic)
  PK_CONV_FUSED,      // units: source-target limb pairs of one polynomial (as the conversions)
  PK_NTT_FWD_CLUSTER, // units: limbs (the one-pass forward transform on a cluster)
  PK_INNER_TC,        // units: ciphertext limbs of the tensor-core inner product prototype
  PK_INNER_FLAT,      // units: ciphertext limbs of its CUDA-core comparison kernel
  PK_NTT_FWD_FINISH,  // units: limbs (the forward row pass with the key-switch finish)
  // counting-only classes (no launches, no time): limbs of the forward NTT
  // passes whose prime takes the strict butterfly (65 q >= 2^64), and limbs of
  // inverse passes launched with the exact quotient (a prime >= 2^61)
  PK_NTT_FWD_STRICT,
  PK_NTT_INV_EXACT,
  // counting-only: limbs through the fused conversion's inverse column stages
  // (sources), its forward column stages (targets), and the strict-butterfly
  // targets among them
  PK_FUSED_SRC_LIMBS,
  PK_FUSED_DST_LIMBS,
  PK_FUSED_DST_STRICT,
  PK_BOOT_MAC_MACS,   // counting-only: k_mac_ext's 128-bit multiply-accumulates
  PK_FINISH_BASE_LIMBS,  // counting-only: limbs of the fused finish that read a base
  PK_COUNT
};
constexpr int PROF_MAX_LEVEL = 64;

struct Profiler {
  bool on = false;
  unsigned long long launches = 0;
  unsigned long long kind_launches[PK_COUNT] = {0};
  // work units per class: limbs processed, except basis conversion, which
  // counts multiply-accumulates per coefficient (polys x targets x sources)
  unsigned long long kind_units[PK_COUNT] = {0};
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int kind;
    int ev;  // index of start event; stop is ev + 1
  };
  std::vector<Rec> recs;
  double kind_ms[PK_COUNT] = {0};
  // key switches by level: outputs of key inner products (each reads one
  // switching key), indexed by the level they run at
  unsigned long long ks_level[PROF_MAX_LEVEL] = {0};

  void count(int kind, unsigned long long units) { kind_units[kind] += units; }
  void count_ks(int level, unsigned long long n) {
    if (level >= 0 && level < PROF_MAX_LEVEL) ks_level[level] += n;
  }

  int begin(int kind, unsigned long long units, cudaStream_t st) {
    ++launches;
    ++kind_launches[kind];
    kind_units[kind] += units;
    if (!on) return -1;
    const size_t need = 2 * (recs.size() + 1);
    while (pool.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
    const int ev = (int)(2 * recs.size());
    cudaEventRecord(pool[ev], st);
    recs.push_back({kind, ev});
    return ev;
  }
  void end(int ev, cudaStream_t st) {
    if (ev >= 0) cudaEventRecord(pool[ev + 1], st);
  }
  // fold recorded pairs into kind_ms (synchronises the events)
  void collect() {
    for (const Rec &r : recs) {
      float ms = 0.f;
      cudaEventSynchronize(pool[r.ev + 1]);
      if (cudaEventElapsedTime(&ms, pool[r.ev], pool[r.ev + 1]) == cudaSuccess) kind_ms[r.kind] += ms;
    }
    recs.clear();
  }
  void reset() {
    collect();
    for (int k = 0; k < PK_COUNT; ++k) {
      kind_ms[k] = 0;
      kind_launches[k] = 0;
      kind_units[k] = 0;
    }
    for (int l = 0; l < PROF_MAX_LEVEL; ++l) ks_level[l] = 0;
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

#define PROF_LAUNCH(ctx, kind, units, launch_stmt)                  \
  do {                                                               \
    const int _ev = (ctx)->prof.begin((kind), (units), (ctx)->stream); \
    launch_stmt;                                                     \
    (ctx)->prof.end(_ev, (ctx)->stream);                             \
  } while (0)
