// Batched executor for uneven workloads: many independent operations on
// ciphertexts of different ring degrees and levels, grouped so that each
// (context, operation, level) group runs as one batched launch set, and
// optionally captured once into a CUDA graph that later replays the whole
// batch with a single cudaGraphLaunch (no per-call host work).  A small
// autotuner picks, per context, the key inner product's outputs-per-thread
// group by timing the candidates on the device.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include <cmath>

#include "ops.cuh"

struct ckks_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

struct GroupKey {
  ckks_ctx *c;
  int op, level, flag;
  bool operator<(const GroupKey &o) const {
    return std::tie(c, op, level, flag) < std::tie(o.c, o.op, o.level, o.flag);
  }
};

int validate(const ckks_op_desc *ops, int n) {
  if (!ops || n < 0) return CKKS_E_PARAM;
  for (int i = 0; i < n; ++i) {
    const ckks_op_desc &d = ops[i];
    if (!d.ctx || !d.a || !d.out) return CKKS_E_PARAM;
    if (d.op == CKKS_OP_MUL_RELIN && !d.b) return CKKS_E_PARAM;
    if (d.op != CKKS_OP_MUL_RELIN && d.op != CKKS_OP_ROTATE && d.op != CKKS_OP_RESCALE) return CKKS_E_PARAM;
    if (d.out->data == d.a->data || (d.b && d.out->data == d.b->data)) return CKKS_E_PARAM;  // out of place
  }
  return CKKS_OK;
}

int run_grouped(const ckks_op_desc *ops, int n) {
  std::map<GroupKey, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) {
    const ckks_op_desc &d = ops[i];
    groups[{d.ctx, d.op, (int)d.a->level, d.op == CKKS_OP_MUL_RELIN ? d.rescale : 0}].push_back(i);
  }
  for (auto &kv : groups) {
    ckks_ctx *c = kv.first.c;
    const std::vector<int> &ix = kv.second;
    const int m = (int)ix.size();
    std::vector<ckks_ct> a(m), b(m), out(m);
    std::vector<int32_t> ks(m);
    for (int j = 0; j < m; ++j) {
      a[j] = *ops[ix[j]].a;
      if (ops[ix[j]].b) b[j] = *ops[ix[j]].b;
      out[j] = *ops[ix[j]].out;
      ks[j] = ops[ix[j]].k;
    }
    int rc = CKKS_OK;
    switch (kv.first.op) {
      case CKKS_OP_MUL_RELIN:
        rc = ckks_mul_relin_batch(c, a.data(), b.data(), out.data(), m, kv.first.flag);
        break;
      case CKKS_OP_ROTATE:
        rc = ckks_rotate_batch(c, a.data(), ks.data(), out.data(), m);
        break;
      case CKKS_OP_RESCALE: {
        for (int j = 0; j < m; ++j) {  // out of place: copy the active limbs, then rescale the copy
          if (out[j].n_limbs < a[j].level + 1) return CKKS_E_LEVEL;
          const size_t w = (size_t)(a[j].level + 1) * c->n;
          CK_CUDA(cudaMemcpyAsync(out[j].data, a[j].data, w * 8, cudaMemcpyDeviceToDevice, c->stream));
          CK_CUDA(cudaMemcpyAsync(out[j].data + (size_t)out[j].n_limbs * c->n,
                                  a[j].data + (size_t)a[j].n_limbs * c->n, w * 8, cudaMemcpyDeviceToDevice,
                                  c->stream));
          out[j].level = a[j].level;
          out[j].scale = a[j].scale;
          out[j].is_ntt = 1;
          out[j].log_n = c->log_n;
        }
        rc = ckks_rescale_batch(c, out.data(), m);
        break;
      }
      default:
        return CKKS_E_PARAM;
    }
    if (rc) return rc;
    for (int j = 0; j < m; ++j) *ops[ix[j]].out = out[j];
  }
  return CKKS_OK;
}

std::vector<ckks_ctx *> contexts_of(const ckks_op_desc *ops, int n) {
  std::vector<ckks_ctx *> cs;
  for (int i = 0; i < n; ++i)
    if (std::find(cs.begin(), cs.end(), ops[i].ctx) == cs.end()) cs.push_back(ops[i].ctx);
  return cs;
}

}  // namespace

extern "C" {

int ckks_exec(const ckks_op_desc *ops, int n) {
  int rc = validate(ops, n);
  if (rc) return rc;
  return run_grouped(ops, n);
}

int ckks_exec_capture(const ckks_op_desc *ops, int n, void *stream, ckks_graph **out) {
  if (!out) return CKKS_E_PARAM;
  *out = nullptr;
  int rc = validate(ops, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return CKKS_E_PARAM;
  std::vector<ckks_ctx *> cs = contexts_of(ops, n);
  std::vector<cudaStream_t> saved;
  for (ckks_ctx *c : cs) {
    saved.push_back(c->stream);
    c->stream = st;
  }
  auto restore = [&]() {
    for (size_t i = 0; i < cs.size(); ++i) {
      cs[i]->stream = saved[i];
      cs[i]->capturing = false;
    }
  };
  // one eager pass sizes every scratch buffer, so the capture allocates nothing
  rc = run_grouped(ops, n);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = CKKS_E_CUDA;
  if (rc) { restore(); return rc; }
  for (ckks_ctx *c : cs) c->capturing = true;
  ckks_graph *g = new ckks_graph();
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    restore();
    delete g;
    return CKKS_E_CUDA;
  }
  rc = run_grouped(ops, n);
  cudaError_t e = cudaStreamEndCapture(st, &g->graph);
  restore();
  if (rc || e != cudaSuccess || !g->graph) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    cudaGetLastError();
    return rc ? rc : CKKS_E_CUDA;
  }
  if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
    cudaGraphDestroy(g->graph);
    delete g;
    cudaGetLastError();
    return CKKS_E_CUDA;
  }
  *out = g;
  return CKKS_OK;
}

int ckks_graph_launch(ckks_graph *g, void *stream) {
  if (!g || !g->exec) return CKKS_E_PARAM;
  return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? CKKS_OK : CKKS_E_CUDA;
}

int ckks_graph_destroy(ckks_graph *g) {
  if (!g) return CKKS_E_PARAM;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return CKKS_OK;
}

int ckks_tune(ckks_ctx *c, int level, int batch, int *chosen) {
  if (!c || level < 0 || level >= c->n_q || batch < 1 || batch > MAX_CTS) return CKKS_E_PARAM;
  if (!c->relin.data) return CKKS_E_NOKEY;
  const u32 n = c->n;
  // inputs: the relinearisation key's own limbs are valid residues at every level
  std::vector<const u64 *> d(batch), keys(batch);
  std::vector<u64 *> o0(batch), o1(batch);
  u64 *outs = nullptr;
  if (cudaMalloc(&outs, sizeof(u64) * 2 * (size_t)(level + 1) * n * batch) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  for (int i = 0; i < batch; ++i) {
    d[i] = c->relin.data;
    keys[i] = c->relin.data;
    o0[i] = outs + (size_t)2 * (level + 1) * n * i;
    o1[i] = o0[i] + (size_t)(level + 1) * n;
  }
  int rc = ensure_scratch(c, ks_ws_words(c, level, batch));
  const int cands[] = {2, 4, 8, 16, 32};
  float best = 1e30f;
  int best_g = c->ip_group;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int cand : cands) {
    if (rc) break;
    c->ip_group = cand;
    float tot = 0.f;
    for (int rep = 0; rep < 3 && !rc; ++rep) {
      cudaEventRecord(e0, c->stream);
      rc = ks_batch(c, level, batch, d.data(), keys.data(), nullptr, nullptr, o0.data(), o1.data(), c->scratch);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep) tot += ms;  // first run warms up
    }
    if (!rc && tot < best) {
      best = tot;
      best_g = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(outs);
  c->ip_group = best_g;
  if (chosen) *chosen = best_g;
  return rc;
}

int ckks_tune_dnum(const ckks_params *p, void *cuda_stream, const uint32_t *cands, int n_cands, int batch,
                   uint64_t seed, uint32_t *best, double *ms_per_op) {
  if (!p || !cands || n_cands < 1 || batch < 1 || batch > MAX_CTS || p->n_q < 2 || p->n_p < 1) return CKKS_E_PARAM;
  double best_ms = 1e300;
  uint32_t best_d = 0;
  for (int i = 0; i < n_cands; ++i) {
    if (ms_per_op) ms_per_op[i] = HUGE_VAL;
    const uint32_t d = cands[i];
    if (d < 1 || d > p->n_q) continue;
    const uint32_t alpha = (p->n_q + d - 1) / d;
    if (alpha + 1 > 16 || alpha > CKKS_MAX_P) continue;  // basis conversions of up to 16 sources
    ckks_params q = *p;
    q.dnum = d;
    q.n_p = alpha;  // P spans one digit
    for (uint32_t k = 0; k < alpha; ++k) q.p_bits[k] = p->p_bits[0];
    ckks_ctx *c = nullptr;
    int rc = ckks_ctx_create(&q, cuda_stream, &c);
    if (!rc) rc = ckks_keygen_from_seed(c, seed, nullptr, 0, 0, 0);
    double ms = HUGE_VAL;
    if (!rc) {
      // inputs: the relinearisation key's limbs are valid residues at every level
      const int level = (int)q.n_q - 1;
      const size_t w = (size_t)(level + 1) * c->n;
      std::vector<ckks_ct> a(batch), o(batch);
      u64 *outs = nullptr;
      if (cudaMalloc(&outs, sizeof(u64) * 2 * w * batch) != cudaSuccess) {
        cudaGetLastError();
        rc = CKKS_E_OOM;
      }
      for (int j = 0; j < batch && !rc; ++j) {
        a[j] = ckks_ct{c->relin.data, (uint32_t)c->log_n, (uint32_t)level, (uint32_t)(level + 1), 1, 1.0};
        o[j] = ckks_ct{outs + 2 * w * j, (uint32_t)c->log_n, (uint32_t)level, (uint32_t)(level + 1), 1, 1.0};
      }
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float tot = 0.f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(e0, c->stream);
        rc = ckks_mul_relin_batch(c, a.data(), a.data(), o.data(), batch, CKKS_RESCALE_MERGED);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep) tot += t;  // first run warms up
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaFree(outs);
      if (!rc) ms = tot / 2 / batch;
    }
    if (c) ckks_ctx_destroy(c);
    if (rc == CKKS_E_OOM) return rc;
    if (rc) continue;
    if (ms_per_op) ms_per_op[i] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best_d = d;
    }
  }
  if (!best_d) return CKKS_E_PARAM;
  if (best) *best = best_d;
  return CKKS_OK;
}

int ckks_ctx_set_ntt_rows(ckks_ctx *c, int rows) {
  if (!c || (rows != 8 && rows != 16)) return CKKS_E_PARAM;
  c->ntt_rows = rows;
  return CKKS_OK;
}

int ckks_ctx_ntt_config(const ckks_ctx *c, int *rows, int *cluster) {
  if (!c) return CKKS_E_PARAM;
  if (rows) *rows = c->ntt_rows;
  if (cluster) *cluster = c->ntt_cluster ? 1 : 0;
  return CKKS_OK;
}

int ckks_ctx_set_ntt_cluster(ckks_ctx *c, int on, int *max_clusters) {
  if (!c) return CKKS_E_PARAM;
  if (!on) {
    c->ntt_cluster = false;
    return CKKS_OK;
  }
  const int rc = ntt_cluster_prepare(c, max_clusters);
  if (rc) return rc;
  c->ntt_cluster = true;
  return CKKS_OK;
}

int ckks_ctx_set_fused_finish(ckks_ctx *c, int on) {
  if (!c || (on != 0 && on != 1)) return CKKS_E_PARAM;
  c->fuse_finish = on != 0;
  return CKKS_OK;
}

int ckks_ctx_set_finish_rows(ckks_ctx *c, int rows) {
  if (!c || (rows != 0 && rows != 8 && rows != 16)) return CKKS_E_PARAM;
  c->fin_rows = rows;
  return CKKS_OK;
}

int ckks_ctx_finish_rows(const ckks_ctx *c, int *rows) {
  if (!c || !rows) return CKKS_E_PARAM;
  *rows = c->fin_rows ? c->fin_rows : c->ntt_rows;
  return CKKS_OK;
}

int ckks_tune_ntt(ckks_ctx *c, int n_polys, int *rows) {
  if (!c || n_polys < 1 || n_polys > 64) return CKKS_E_PARAM;
  if (c->capturing) return CKKS_E_STATE;
  if (!c->relin.data) return CKKS_E_NOKEY;
  const u32 n = c->n;
  const int nl = c->n_q;
  // inputs: the relinearisation key's limbs are valid residues of q_0..q_{n_q-1}
  u64 *outs = nullptr;
  if (cudaMalloc(&outs, sizeof(u64) * (size_t)nl * n * n_polys) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  std::vector<const u64 *> src(n_polys);
  std::vector<u64 *> dst(n_polys);
  std::vector<const u64 *> dstc(n_polys);
  int mods[MAX_MODS];
  for (int t = 0; t < nl; ++t) mods[t] = t;
  for (int i = 0; i < n_polys; ++i) {
    src[i] = c->relin.data;
    dst[i] = outs + (size_t)nl * n * i;
    dstc[i] = dst[i];
  }
  const int cands[] = {16, 8};
  float best = 1e30f;
  int best_r = c->ntt_rows, rc = CKKS_OK;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int cand : cands) {
    c->ntt_rows = cand;
    float tot = 0.f;
    for (int rep = 0; rep < 3 && !rc; ++rep) {
      cudaEventRecord(e0, c->stream);
      rc = launch_ntt(c, src.data(), dst.data(), n_polys, nl, mods, false);
      if (!rc) rc = launch_ntt(c, dstc.data(), dst.data(), n_polys, nl, mods, true);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep) tot += ms;  // first run warms up
    }
    if (!rc && tot < best) {
      best = tot;
      best_r = cand;
    }
  }
  c->ntt_rows = best_r;
  // at N = 2^16, the one-pass forward transform on clusters against the two passes
  const bool was_cluster = c->ntt_cluster;
  bool best_cluster = false;
  if (!rc && c->log_n == 16 && ntt_cluster_prepare(c, nullptr) == CKKS_OK) {
    for (int on = 0; on < 2 && !rc; ++on) {
      c->ntt_cluster = on != 0;
      float tot = 0.f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(e0, c->stream);
        rc = launch_ntt(c, src.data(), dst.data(), n_polys, nl, mods, false);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) tot += ms;
      }
      if (!on) best = tot;
      else if (tot < best) best_cluster = true;
    }
  }
  c->ntt_cluster = rc ? was_cluster : best_cluster;
  // the row tile of the forward row pass with the key-switch finish, timed on
  // the key's limbs as accumulators and bases (with the ModDown constants)
  if (!rc) {
    RowFinish f;
    f.w = c->d_conv + c->conv.moddown_pinv;
    for (int i = 0; i < n_polys; ++i) {
      f.acc[i] = c->relin.data;
      f.base[i] = c->relin.data;
      f.gal[i] = 1u;
      f.out[i] = dst[i];
    }
    float fbest = 1e30f;
    int fbest_r = 0;
    for (int cand : cands) {
      c->fin_rows = cand;
      float tot = 0.f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(e0, c->stream);
        rc = launch_ntt_fwd_finish(c, src.data(), dst.data(), n_polys, nl, mods, NTT_BOTH, f);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) tot += ms;
      }
      if (!rc && tot < fbest) {
        fbest = tot;
        fbest_r = cand;
      }
    }
    c->fin_rows = rc ? 0 : fbest_r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(outs);
  if (rows) *rows = best_r;
  return rc;
}

}  // extern "C"
