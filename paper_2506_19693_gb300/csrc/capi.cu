// C ABI entry points (include/ckks.h): context, keys, encryption and the
// homomorphic operations of ReBoot Sec. 3, orchestrated over the kernels in
// ntt.cu, ops.cu, keyswitch.cu and encode.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ops.cuh"

// ---------------------------------------------------------------- scratch
int ensure_scratch(ckks_ctx *c, size_t words) {
  if (words <= c->scratch_words) return CKKS_OK;
  if (c->capturing) return CKKS_E_STATE;  // no allocation inside a graph capture
  CK_CUDA(cudaStreamSynchronize(c->stream));
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_words = 0;
  if (cudaMalloc(&c->scratch, words * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  c->scratch_words = words;
  return CKKS_OK;
}
int ensure_fscratch(ckks_ctx *c, size_t words) {
  if (words <= c->fscratch_words) return CKKS_OK;
  if (c->capturing) return CKKS_E_STATE;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  if (c->fscratch) cudaFree(c->fscratch);
  c->fscratch = nullptr;
  c->fscratch_words = 0;
  if (cudaMalloc(&c->fscratch, words * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  c->fscratch_words = words;
  return CKKS_OK;
}

namespace {

int last_err() { return cudaGetLastError() == cudaSuccess ? CKKS_OK : CKKS_E_CUDA; }
u64 *poly1(const ckks_ct *ct, u32 n) { return ct->data + (size_t)ct->n_limbs * n; }

bool ct_ok(const ckks_ctx *c, const ckks_ct *ct) {
  return ct && ct->data && ct->log_n == (u32)c->log_n && (int)ct->level < c->n_q && ct->n_limbs >= ct->level + 1;
}

void free_keys(ckks_ctx *c) {
  if (c->relin.data) cudaFree(c->relin.data);
  c->relin.data = nullptr;
  for (auto &kv : c->galois) cudaFree(kv.second.data);
  c->galois.clear();
  if (c->d_pk) cudaFree(c->d_pk);
  c->d_pk = nullptr;
}

size_t full_key_words(const ckks_ctx *c) { return (size_t)c->n_digits * 2 * (c->n_q + c->n_p) * c->n; }
size_t key_words(const ckks_ctx *c) {
  return c->key_compressed ? KEY_HDR + (size_t)c->n_digits * (c->n_q + c->n_p) * c->n : full_key_words(c);
}

static_assert(KEY_HDR >= 8, "a compressed key's header holds one generator state per digit (at most 8)");

// Build a switching key from s' (NTT domain over all n_q + n_p moduli) to s
// (reading C7); key_id 0 = relinearisation, else the Galois element.
int make_key(ckks_ctx *c, u64 key_id, const u64 *sp_ntt, DevKey *out) {
  const int ext = c->n_q + c->n_p;
  const u32 n = c->n;
  u64 *data = nullptr;
  if (cudaMalloc(&data, key_words(c) * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  int rc = ensure_scratch(c, (size_t)(c->key_compressed ? 2 : 1) * ext * n + n);
  if (rc) { cudaFree(data); return rc; }
  u64 *e_res = c->scratch;
  i64 *e_dev = reinterpret_cast<i64 *>(c->scratch + (size_t)ext * n);
  u64 *a_drop = c->scratch + (size_t)ext * n + n;  // compressed keys: the a row is not kept
  u64 seeds[KEY_HDR] = {0};
  std::vector<i64> e(n);
  int mods[MAX_MODS];
  for (int i = 0; i < ext; ++i) mods[i] = i;
  KeyArgs ka;
  ka.sp_ntt = sp_ntt;
  ka.err = e_res;
  for (int t = 0; t < c->n_q; ++t) {
    u64 p = 1;
    for (int k = 0; k < c->n_p; ++k) p = host_mulmod(p, c->mod[c->n_q + k] % c->mod[t], c->mod[t]);
    ka.p_mod[t] = p;
  }
  for (int j = 0; j < c->n_digits; ++j) {
    sample_gaussian(sm_stream(c->key_seed, TAG_KEY_E, key_id * 256 + j), n, c->sigma, c->e_bound, e.data());
    CK_CUDA(cudaMemcpyAsync(e_dev, e.data(), sizeof(i64) * n, cudaMemcpyHostToDevice, c->stream));
    rc = ew_signed_to_res(c, e_dev, e_res, 0, ext);
    if (rc) break;
    const u64 *s1[1] = {e_res};
    u64 *d1[1] = {e_res};
    rc = launch_ntt(c, s1, d1, 1, ext, mods, false);
    if (rc) break;
    ka.key_a = sm_stream(c->key_seed, TAG_KEY_A, key_id * 256 + j);
    seeds[j] = ka.key_a;
    ka.lo = j * c->alpha;
    ka.hi = std::min((j + 1) * c->alpha, c->n_q);
    if (c->key_compressed) {
      ka.b = data + KEY_HDR + (size_t)j * ext * n;
      ka.a = a_drop;
    } else {
      ka.b = data + (size_t)(2 * j) * ext * n;
      ka.a = data + (size_t)(2 * j + 1) * ext * n;
    }
    rc = ew_keyrow(c, ka, ext);
    if (rc) break;
    // the host error buffer is reused next digit: finish the copy first
    CK_CUDA(cudaStreamSynchronize(c->stream));
  }
  if (!rc && c->key_compressed &&
      (cudaMemcpyAsync(data, seeds, sizeof(seeds), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
       cudaStreamSynchronize(c->stream) != cudaSuccess))
    rc = CKKS_E_CUDA;
  if (rc) { cudaFree(data); return rc; }
  out->data = data;
  return CKKS_OK;
}

int galois_key(ckks_ctx *c, u64 g) {
  if (!c->have_secret) return CKKS_E_STATE;
  if ((g & 1) == 0 || g >= 2ULL * c->n) return CKKS_E_PARAM;
  if (c->galois.count(g)) return CKKS_OK;
  const int ext = c->n_q + c->n_p;
  u64 *sp = nullptr;
  if (cudaMalloc(&sp, (size_t)ext * c->n * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  EwArgs a;
  a.x0[0] = c->d_s_ntt;
  a.o0[0] = sp;
  const u32 g32 = (u32)g;
  int rc = ew_automorph(c, a, &g32, ext, 1, false);
  DevKey k;
  if (!rc) rc = make_key(c, g, sp, &k);
  cudaStreamSynchronize(c->stream);
  cudaFree(sp);
  if (rc) return rc;
  c->galois[g] = k;
  return CKKS_OK;
}

}  // namespace
int galois_key_for(ckks_ctx *c, u64 g) { return galois_key(c, g); }
namespace {

const DevKey *find_galois(const ckks_ctx *c, u64 g) {
  auto it = c->galois.find(g);
  return it == c->galois.end() ? nullptr : &it->second;
}

}  // namespace

// in-place rescale of n <= MAX_CTS ciphertexts at one level (reading C10)
int rescale_chunk(ckks_ctx *c, ckks_ct *cts, int n) {
  const int level = cts[0].level;
  const u32 nn = c->n;
  const size_t per = (size_t)2 * nn + (size_t)2 * level * nn;
  int rc = ensure_scratch(c, per * n);
  if (rc) return rc;
  std::vector<const u64 *> src(2 * n);
  std::vector<u64 *> dst(2 * n);
  RescaleArgs r;
  r.level = level;
  r.qlinv = c->d_conv + c->conv.rescale_qlinv + 2 * (size_t)level * c->n_q;
  for (int i = 0; i < n; ++i) {
    u64 *last = c->scratch + per * i;
    src[2 * i] = cts[i].data + (size_t)level * nn;
    src[2 * i + 1] = poly1(&cts[i], nn) + (size_t)level * nn;
    dst[2 * i] = last;
    dst[2 * i + 1] = last + nn;
    r.c0[i] = cts[i].data;
    r.c1[i] = poly1(&cts[i], nn);
    r.last[i] = last;
    r.lift[i] = last + 2 * nn;
  }
  int m1[1] = {level};
  rc = launch_ntt(c, src.data(), dst.data(), 2 * n, 1, m1, true);
  if (rc) return rc;
  rc = ew_rescale_lift(c, r, n);
  if (rc) return rc;
  std::vector<const u64 *> ls(2 * n);
  std::vector<u64 *> ld(2 * n);
  for (int i = 0; i < n; ++i)
    for (int p = 0; p < 2; ++p) {
      ld[2 * i + p] = r.lift[i] + (size_t)p * level * nn;
      ls[2 * i + p] = ld[2 * i + p];
    }
  int mods[MAX_MODS];
  for (int l = 0; l < level; ++l) mods[l] = l;
  // c_i = (c_i - lift_i) q_l^-1 in the output stage of the lift's forward
  // transform (in place: each output word is read before it is written), or by
  // k_rescale_finish after it
  bool fused = c->fuse_finish;
  RowFinish f;
  if (fused) {
    f.w = r.qlinv;
    for (int i = 0; i < n && fused; ++i)
      for (int p = 0; p < 2; ++p) {
        u64 *cp = p ? r.c1[i] : r.c0[i];
        f.acc[2 * i + p] = cp;
        f.base[2 * i + p] = nullptr;
        f.gal[2 * i + p] = 1u;
        f.out[2 * i + p] = cp;
        if ((uintptr_t)cp & 15) fused = false;
      }
  }
  if (fused) {
    rc = launch_ntt_fwd_finish(c, ls.data(), ld.data(), 2 * n, level, mods, NTT_BOTH, f);
    if (rc) return rc;
  } else {
    rc = launch_ntt(c, ls.data(), ld.data(), 2 * n, level, mods, false);
    if (rc) return rc;
    rc = ew_rescale_finish(c, r, n);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    cts[i].scale /= (double)c->mod[level];
    cts[i].level = level - 1;
  }
  return CKKS_OK;
}

int mul_relin_chunk(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n, bool merged) {
  const int level = a[0].level, nl = level + 1;
  if (merged && level < 1) return CKKS_E_LEVEL;
  const u32 nn = c->n;
  if (!c->relin.data) return CKKS_E_NOKEY;
  const size_t d2w = (size_t)nl * nn * n;
  int rc = ensure_scratch(c, d2w + ks_ws_words(c, level, n));
  if (rc) return rc;
  std::vector<u64 *> d2(n);
  EwArgs e;
  for (int i = 0; i < n; ++i) {
    d2[i] = c->scratch + (size_t)nl * nn * i;
    e.x0[i] = a[i].data;
    e.x1[i] = poly1(&a[i], nn);
    e.y0[i] = b[i].data;
    e.y1[i] = poly1(&b[i], nn);
    e.o0[i] = out[i].data;
    e.o1[i] = poly1(&out[i], nn);
  }
  rc = ew_tensor(c, e, d2.data(), nl, n);
  if (rc) return rc;
  std::vector<const u64 *> dd(n), keys(n), b0(n), b1(n);
  std::vector<u64 *> o0(n), o1(n);
  for (int i = 0; i < n; ++i) {
    dd[i] = d2[i];
    keys[i] = c->relin.data;
    b0[i] = e.o0[i];
    b1[i] = e.o1[i];
    o0[i] = e.o0[i];
    o1[i] = e.o1[i];
  }
  std::vector<double> scales(n);
  for (int i = 0; i < n; ++i) scales[i] = a[i].scale * b[i].scale;
  rc = ks_batch(c, level, n, dd.data(), keys.data(), b0.data(), b1.data(), o0.data(), o1.data(),
                c->scratch + d2w, merged);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    out[i].level = merged ? level - 1 : level;
    out[i].scale = merged ? scales[i] / (double)c->mod[level] : scales[i];
    out[i].is_ntt = 1;
    out[i].log_n = c->log_n;
  }
  return CKKS_OK;
}

// out[i] = sigma_{g[i]}(in[i]) followed by key switching (reading C11)
int automorph_chunk(ckks_ctx *c, const ckks_ct *in, const u64 *g, ckks_ct *out, int n) {
  const int level = in[0].level, nl = level + 1;
  const u32 nn = c->n;
  std::vector<const u64 *> keys(n);
  for (int i = 0; i < n; ++i) {
    const DevKey *k = find_galois(c, g[i]);
    if (!k) return CKKS_E_NOKEY;
    keys[i] = k->data;
  }
  const size_t tw = (size_t)2 * nl * nn * n;
  int rc = ensure_scratch(c, tw + ks_ws_words(c, level, n));
  if (rc) return rc;
  std::vector<const u64 *> t1(n), t0(n);
  std::vector<u64 *> o0(n), o1(n);
  std::vector<u32> g32(n);
  EwArgs e;
  for (int i = 0; i < n; ++i) {
    u64 *tmp = c->scratch + (size_t)2 * nl * nn * i;
    e.x0[i] = in[i].data;
    e.x1[i] = poly1(&in[i], nn);
    e.o0[i] = tmp;
    e.o1[i] = tmp + (size_t)nl * nn;
    g32[i] = (u32)g[i];
    t0[i] = tmp;
    t1[i] = tmp + (size_t)nl * nn;
    o0[i] = out[i].data;
    o1[i] = poly1(&out[i], nn);
  }
  rc = ew_automorph(c, e, g32.data(), nl, n, true);
  if (rc) return rc;
  std::vector<double> scales(n);
  for (int i = 0; i < n; ++i) scales[i] = in[i].scale;
  rc = ks_batch(c, level, n, t1.data(), keys.data(), t0.data(), nullptr, o0.data(), o1.data(),
                c->scratch + tw);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    out[i].level = level;
    out[i].scale = scales[i];
    out[i].is_ntt = 1;
    out[i].log_n = c->log_n;
  }
  return CKKS_OK;
}

const u64 *galois_key_data(ckks_ctx *c, u64 g) {
  const DevKey *k = find_galois(c, g);
  return k ? k->data : nullptr;
}

// Giant step of a merged linear level (reading B10): t = sigma_g(in[i]) (both
// polynomials, NTT domain), then acc[i] (= or, accumulate, +=) the key-switch
// accumulator of t.c1 over q_0..q_l, P, and base0[i] += t.c0 over q_0..q_l.
// n <= MAX_CTS, all at one level.
int rotate_accumulate_chunk(ckks_ctx *c, const ckks_ct *in, u64 g, int n, u64 *const *acc, u64 *const *base0,
                            bool accumulate) {
  const int level = in[0].level, nl = level + 1;
  const u32 nn = c->n;
  const DevKey *k = find_galois(c, g);
  if (!k) return CKKS_E_NOKEY;
  const size_t tw = (size_t)2 * nl * nn * n;
  int rc = ensure_scratch(c, tw + ks_modup_words(c, level, n));
  if (rc) return rc;
  std::vector<const u64 *> t0(n), t1(n), keys(n, k->data);
  std::vector<u32> g32(n, (u32)g);
  EwArgs e;
  for (int i = 0; i < n; ++i) {
    u64 *tmp = c->scratch + (size_t)2 * nl * nn * i;
    e.x0[i] = in[i].data;
    e.x1[i] = poly1(&in[i], nn);
    e.o0[i] = tmp;
    e.o1[i] = tmp + (size_t)nl * nn;
    t0[i] = tmp;
    t1[i] = tmp + (size_t)nl * nn;
  }
  rc = ew_automorph(c, e, g32.data(), nl, n, true);
  if (rc) return rc;
  std::vector<u64 *> eb(n);
  rc = ks_modup(c, level, n, t1.data(), c->scratch + tw, eb.data());
  if (rc) return rc;
  std::vector<const u64 *> ebc(eb.begin(), eb.end());
  rc = ks_accumulate(c, level, n, t1.data(), ebc.data(), keys.data(), nullptr, acc, accumulate);
  if (rc) return rc;
  // base0[i] += t0[i]: two single polynomials per element-wise slot (an odd
  // last one paired with itself: both lanes write the same sum)
  EwArgs s;
  const int slots = (n + 1) / 2;
  for (int j = 0; j < slots; ++j) {
    const int i0 = 2 * j, i1 = std::min(2 * j + 1, n - 1);
    s.x0[j] = base0[i0];
    s.y0[j] = t0[i0];
    s.o0[j] = base0[i0];
    s.x1[j] = base0[i1];
    s.y1[j] = t0[i1];
    s.o1[j] = base0[i1];
  }
  return ew_addsub(c, s, nl, slots, false);
}

// Hoisted rotations: one ModUp of c1 per input serves every Galois element;
// out[j * n + i] = sigma_{g[j]}(in[i]) key-switched back to s.  Outputs must
// not alias inputs.  All inputs at one level.
int rotate_hoisted_internal(ckks_ctx *c, const ckks_ct *in, int n, const u64 *g, int m, ckks_ct *out) {
  if (n <= 0 || m <= 0) return CKKS_OK;
  const int level = in[0].level;
  const u32 nn = c->n;
  std::vector<const u64 *> keys(m);
  for (int j = 0; j < m; ++j) {
    const DevKey *k = find_galois(c, g[j]);
    if (!k) return CKKS_E_NOKEY;
    keys[j] = k->data;
  }
  // inputs per chunk: keep np * m outputs within one tail launch set of <= MAX_CTS each
  const int np_max = std::max(1, std::min(MAX_CTS, MAX_CTS / m > 0 ? MAX_CTS / m : 1));
  for (int i0 = 0; i0 < n; i0 += np_max) {
    const int np = std::min(np_max, n - i0);
    const size_t mw = ks_modup_words(c, level, np);
    const int nv_max = std::min(MAX_CTS, np * m);
    int rc = ensure_scratch(c, mw + ks_tail_words(c, level, nv_max));
    if (rc) return rc;
    std::vector<const u64 *> c1(np);
    std::vector<u64 *> eb(np);
    for (int i = 0; i < np; ++i) c1[i] = poly1(&in[i0 + i], nn);
    rc = ks_modup(c, level, np, c1.data(), c->scratch, eb.data());
    if (rc) return rc;
    const int nv_total = np * m;
    for (int v0 = 0; v0 < nv_total; v0 += MAX_CTS) {
      const int nv = std::min(MAX_CTS, nv_total - v0);
      std::vector<const u64 *> d(nv), e(nv), k(nv), b0(nv);
      std::vector<u32> gal(nv);
      std::vector<u64 *> o0(nv), o1(nv);
      for (int v = 0; v < nv; ++v) {
        const int idx = v0 + v, j = idx / np, i = idx % np;
        d[v] = c1[i];
        e[v] = eb[i];
        k[v] = keys[j];
        gal[v] = (u32)g[j];
        b0[v] = in[i0 + i].data;
        ckks_ct &o = out[(size_t)j * n + i0 + i];
        o0[v] = o.data;
        o1[v] = poly1(&o, nn);
      }
      rc = ks_tail(c, level, nv, d.data(), e.data(), k.data(), gal.data(), b0.data(), gal.data(), nullptr,
                   o0.data(), o1.data(), c->scratch + mw);
      if (rc) return rc;
    }
  }
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < n; ++i) {
      ckks_ct &o = out[(size_t)j * n + i];
      o.level = level;
      o.scale = in[i].scale;
      o.is_ntt = 1;
      o.log_n = c->log_n;
    }
  return CKKS_OK;
}

extern "C" {

int ckks_rotate_hoisted(ckks_ctx *c, const ckks_ct *in, int n, const int32_t *k, int n_k, ckks_ct *out) {
  if (!c || !in || !k || !out || n < 0 || n_k < 0) return CKKS_E_PARAM;
  if (n == 0 || n_k == 0) return CKKS_OK;
  const u32 level = in[0].level;
  for (int i = 0; i < n; ++i) {
    if (!ct_ok(c, &in[i])) return CKKS_E_PARAM;
    if (in[i].level != level) return CKKS_E_LEVEL;
  }
  for (int i = 0; i < n * n_k; ++i) {
    if (!out[i].data) return CKKS_E_PARAM;
    if (out[i].n_limbs < level + 1) return CKKS_E_LEVEL;
    for (int j = 0; j < n; ++j)
      if (out[i].data == in[j].data) return CKKS_E_PARAM;  // no aliasing
  }
  std::vector<u64> g(n_k);
  for (int j = 0; j < n_k; ++j) g[j] = ckks_galois_elt(c, k[j]);
  return rotate_hoisted_internal(c, in, n, g.data(), n_k, out);
}

const char *ckks_status_str(int s) {
  switch (s) {
    case CKKS_OK: return "ok";
    case CKKS_E_PARAM: return "invalid argument or parameter set";
    case CKKS_E_LEVEL: return "level mismatch or out of range";
    case CKKS_E_SCALE: return "scale out of range";
    case CKKS_E_NOKEY: return "required key missing";
    case CKKS_E_OOM: return "out of memory";
    case CKKS_E_CUDA: return "CUDA runtime error";
    case CKKS_E_TIMEOUT: return "bounded device wait expired";
    case CKKS_E_STATE: return "call made in the wrong state";
    default: return "unknown status";
  }
}

int ckks_ctx_create(const ckks_params *p, void *stream, ckks_ctx **out) {
  if (!p || !out) return CKKS_E_PARAM;
  *out = nullptr;
  if (p->log_n < 12 || p->log_n > 17 || p->n_q < 1 || p->n_q > CKKS_MAX_Q || p->n_p < 1 ||
      p->n_p > CKKS_MAX_P || p->dnum < 1 || p->n_q + p->n_p > MAX_MODS || p->h < 1 ||
      p->h > (1u << p->log_n) || !(p->sigma > 0))
    return CKKS_E_PARAM;
  ckks_ctx *c = new (std::nothrow) ckks_ctx();
  if (!c) return CKKS_E_OOM;
  cudaGetDevice(&c->device);
  c->stream = (cudaStream_t)stream;
  c->log_n = p->log_n;
  c->n = 1u << p->log_n;
  c->n_q = p->n_q;
  c->n_p = p->n_p;
  c->dnum = p->dnum;
  c->alpha = (c->n_q + c->dnum - 1) / c->dnum;
  c->n_digits = (c->n_q + c->alpha - 1) / c->alpha;
  c->h = p->h;
  c->sigma = p->sigma;
  c->e_bound = (i64)std::floor(6.0 * p->sigma);
  c->default_scale = std::ldexp(1.0, 0) * std::pow(2.0, p->log2_scale);
  if (c->alpha > 16 || c->n_p > 16 || c->n_digits > 8) { delete c; return CKKS_E_PARAM; }
  unsigned bits[MAX_MODS];
  for (int i = 0; i < c->n_q; ++i) bits[i] = p->q_bits[i];
  for (int i = 0; i < c->n_p; ++i) bits[c->n_q + i] = p->p_bits[i];
  if (host_gen_primes(c->n_q + c->n_p, bits, std::max(17, c->log_n + 1), c->mod) != CKKS_OK) {
    delete c;
    return CKKS_E_PARAM;
  }
  for (int i = 0; i < c->n_q + c->n_p; ++i) c->psi[i] = host_find_psi(c->mod[i], c->n);
  int rc = build_tables(c);
  if (rc) { ckks_ctx_destroy(c); return rc; }
  *out = c;
  return CKKS_OK;
}

int ckks_ctx_destroy(ckks_ctx *c) {
  if (!c) return CKKS_E_PARAM;
  cudaStreamSynchronize(c->stream);
  free_keys(c);
  cudaFree(c->d_mods);
  cudaFree(c->d_tw_fwd);
  cudaFree(c->d_tw_inv);
  cudaFree(c->d_tw_row_fwd);
  cudaFree(c->d_tw_row_inv);
  cudaFree(c->d_conv);
  cudaFree(c->d_s_ntt);
  cudaFree(c->scratch);
  cudaFree(c->fscratch);
  for (auto &kv : c->tc_bmats) cudaFree(kv.second);
  cudaFree(c->tc_err);
  if (c->h2d) cudaStreamSynchronize(c->h2d), cudaStreamDestroy(c->h2d);
  if (c->d2h) cudaStreamSynchronize(c->d2h), cudaStreamDestroy(c->d2h);
  for (int i = 0; i < 3; ++i) {
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_comp[i]) cudaEventDestroy(c->ev_comp[i]);
    if (c->ev_out[i]) cudaEventDestroy(c->ev_out[i]);
  }
  cudaFree(c->stage);
  boot_free(c);
  if (c->pinned) cudaFreeHost(c->pinned);
  delete c;
  return CKKS_OK;
}

int ckks_ctx_set_stream(ckks_ctx *c, void *stream) {
  if (!c) return CKKS_E_PARAM;
  c->stream = (cudaStream_t)stream;
  return CKKS_OK;
}

int ckks_ctx_moduli(const ckks_ctx *c, uint64_t *out, int cap) {
  if (!c || !out) return CKKS_E_PARAM;
  const int m = std::min(cap, c->n_q + c->n_p);
  for (int i = 0; i < m; ++i) out[i] = c->mod[i];
  return m;
}

int ckks_ctx_roots(const ckks_ctx *c, uint64_t *out, int cap) {
  if (!c || !out) return CKKS_E_PARAM;
  const int m = std::min(cap, c->n_q + c->n_p);
  for (int i = 0; i < m; ++i) out[i] = c->psi[i];
  return m;
}

int ckks_ctx_digits(const ckks_ctx *c, int *n_digits, int *alpha) {
  if (!c) return CKKS_E_PARAM;
  if (n_digits) *n_digits = c->n_digits;
  if (alpha) *alpha = c->alpha;
  return CKKS_OK;
}

int ckks_ctx_device_bytes(const ckks_ctx *c, uint64_t *bytes) {
  if (!c || !bytes) return CKKS_E_PARAM;
  size_t b = c->table_bytes + c->scratch_words * 8 + c->fscratch_words * 8;
  if (c->d_s_ntt) b += (size_t)(c->n_q + c->n_p) * c->n * 8;
  if (c->relin.data) b += key_words(c) * 8;
  b += c->galois.size() * key_words(c) * 8;
  *bytes = b;
  return CKKS_OK;
}

int ckks_ctx_profile(ckks_ctx *c, int enable) {
  if (!c) return CKKS_E_PARAM;
  c->prof.reset();
  c->prof.on = enable != 0;
  return CKKS_OK;
}

int ckks_ctx_ks_histogram(ckks_ctx *c, uint64_t *counts, int cap) {
  if (!c || cap < 0 || (cap > 0 && !counts)) return CKKS_E_PARAM;
  for (int l = 0; l < cap && l < PROF_MAX_LEVEL; ++l) counts[l] = c->prof.ks_level[l];
  return PROF_MAX_LEVEL;
}

int ckks_ctx_profile_read(ckks_ctx *c, double *ms, uint64_t *launches, uint64_t *limbs, int cap) {
  if (!c || cap < 0) return CKKS_E_PARAM;
  c->prof.collect();
  const int m = std::min(cap, (int)PK_COUNT);
  for (int k = 0; k < m; ++k) {
    if (ms) ms[k] = c->prof.kind_ms[k];
    if (launches) launches[k] = c->prof.kind_launches[k];
    if (limbs) limbs[k] = c->prof.kind_units[k];
  }
  c->prof.reset();
  return (int)PK_COUNT;
}

int ckks_profile_kinds(void) { return (int)PK_COUNT; }

int ckks_ctx_set_form(ckks_ctx *c, int form) {
  if (!c || (form != CKKS_FORM_UINT64 && form != CKKS_FORM_TENSOR && form != CKKS_FORM_FUSED)) return CKKS_E_PARAM;
  c->use_tc = form == CKKS_FORM_TENSOR;
  c->use_fused = form == CKKS_FORM_FUSED;
  return CKKS_OK;
}

int ckks_ctx_device_error(ckks_ctx *c) {
  if (!c) return CKKS_E_PARAM;
  if (!c->tc_err) return CKKS_OK;
  int h = 0;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  CK_CUDA(cudaMemcpy(&h, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    CK_CUDA(cudaMemset(c->tc_err, 0, sizeof(int)));
    return h == 1 ? CKKS_E_TIMEOUT : CKKS_E_CUDA;
  }
  return CKKS_OK;
}

const char *ckks_profile_kind_name(int k) {
  static const char *names[PK_COUNT] = {"ntt_fwd_pass_a", "ntt_fwd_pass_b", "ntt_inv_pass_a", "ntt_inv_pass_b",
                                        "bconv", "ks_inner_product", "ks_moddown_combine", "tensor",
                                        "automorph", "rescale", "elementwise", "encode_decode", "bconv_tc",
                                        "boot_mac_ext", "boot_lincomb", "conv_fused", "ntt_fwd_cluster", "ks_inner_tc",
                                        "ks_inner_flat", "ntt_fwd_pass_b_finish",
                                        "ntt_fwd_strict_limbs",
                                        "ntt_inv_exact_limbs", "fused_src_limbs", "fused_dst_limbs",
                                        "fused_dst_strict_limbs", "boot_mac_ext_macs", "finish_base_limbs"};
  return (k >= 0 && k < PK_COUNT) ? names[k] : "unknown";
}

int ckks_ctx_launch_count(const ckks_ctx *c, uint64_t *count) {
  if (!c || !count) return CKKS_E_PARAM;
  *count = c->prof.launches;
  return CKKS_OK;
}

uint64_t ckks_galois_elt(const ckks_ctx *c, int32_t k) {
  const i64 half = c->n / 2;
  const i64 r = ((k % half) + half) % half;
  return host_powmod(5, (u64)r, 2ULL * c->n);
}

int ckks_keygen_from_seed(ckks_ctx *c, uint64_t seed, const int32_t *rot, int n_rot, int want_conj,
                          int want_boot) {
  if (!c || n_rot < 0 || (n_rot > 0 && !rot)) return CKKS_E_PARAM;
  std::vector<int> boot_steps;
  if (want_boot) {
    int rc0 = boot_rotation_steps(c, boot_steps);
    if (rc0) return rc0;
  }
  CK_CUDA(cudaStreamSynchronize(c->stream));
  free_keys(c);
  const int ext = c->n_q + c->n_p;
  const u32 n = c->n;
  c->key_seed = seed;
  c->s_host.assign(n, 0);
  sample_secret(seed, n, c->h, c->s_host.data());
  if (!c->d_s_ntt && cudaMalloc(&c->d_s_ntt, (size_t)ext * n * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  int rc = ensure_scratch(c, n);
  if (rc) return rc;
  std::vector<i64> s64(n);
  for (u32 i = 0; i < n; ++i) s64[i] = c->s_host[i];
  i64 *s_dev = reinterpret_cast<i64 *>(c->scratch);
  CK_CUDA(cudaMemcpyAsync(s_dev, s64.data(), sizeof(i64) * n, cudaMemcpyHostToDevice, c->stream));
  rc = ew_signed_to_res(c, s_dev, c->d_s_ntt, 0, ext);
  if (rc) return rc;
  int mods[MAX_MODS];
  for (int i = 0; i < ext; ++i) mods[i] = i;
  const u64 *s1[1] = {c->d_s_ntt};
  u64 *d1[1] = {c->d_s_ntt};
  rc = launch_ntt(c, s1, d1, 1, ext, mods, false);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  c->have_secret = true;
  // relinearisation key: s' = s^2
  u64 *s2 = nullptr;
  if (cudaMalloc(&s2, (size_t)ext * n * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  rc = ew_square(c, s2, c->d_s_ntt, ext);
  if (!rc) rc = make_key(c, 0, s2, &c->relin);
  cudaStreamSynchronize(c->stream);
  cudaFree(s2);
  if (rc) return rc;
  for (int i = 0; i < n_rot; ++i) {
    rc = galois_key(c, ckks_galois_elt(c, rot[i]));
    if (rc) return rc;
  }
  if (want_conj || want_boot) {
    rc = galois_key(c, 2ULL * n - 1);
    if (rc) return rc;
  }
  for (int k : boot_steps) {
    rc = galois_key(c, ckks_galois_elt(c, k));
    if (rc) return rc;
  }
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_set_key_compression(ckks_ctx *c, int on) {
  if (!c) return CKKS_E_PARAM;
  if (c->relin.data || !c->galois.empty()) return CKKS_E_STATE;
  c->key_compressed = on != 0;
  return CKKS_OK;
}

int ckks_keygen_galois(ckks_ctx *c, uint64_t g) {
  if (!c) return CKKS_E_PARAM;
  int rc = galois_key(c, g);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_debug_secret(const ckks_ctx *c, int8_t *out) {
  if (!c || !out) return CKKS_E_PARAM;
  if (!c->have_secret) return CKKS_E_STATE;
  std::memcpy(out, c->s_host.data(), c->n);
  return CKKS_OK;
}

int ckks_debug_key(const ckks_ctx *c, uint64_t g, uint64_t *out) {
  if (!c || !out) return CKKS_E_PARAM;
  const DevKey *k = g == 0 ? (c->relin.data ? &c->relin : nullptr) : find_galois(c, g);
  if (!k) return CKKS_E_NOKEY;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  const int ext = c->n_q + c->n_p;
  const size_t row = (size_t)ext * c->n;
  if (c->key_compressed) {
    // b rows from the device; a rows regenerated from the header (C22), in Montgomery form like b
    u64 seeds[KEY_HDR];
    CK_CUDA(cudaMemcpy(seeds, k->data, sizeof(seeds), cudaMemcpyDeviceToHost));
    for (int j = 0; j < c->n_digits; ++j) {
      CK_CUDA(cudaMemcpy(out + 2 * j * row, k->data + KEY_HDR + j * row, row * sizeof(u64), cudaMemcpyDeviceToHost));
      for (int t = 0; t < ext; ++t) {
        const u64 q = c->mod[t];
        const u64 r64 = (u64)(((unsigned __int128)1 << 64) % q);
        for (u32 k2 = 0; k2 < c->n; ++k2)
          out[(2 * j + 1) * row + (size_t)t * c->n + k2] =
              host_mulmod(sample_uniform(seeds[j], (u64)t * c->n + k2, q), r64, q);
      }
    }
  } else {
    CK_CUDA(cudaMemcpy(out, k->data, key_words(c) * sizeof(u64), cudaMemcpyDeviceToHost));
  }
  // stored in Montgomery form (x 2^64 mod q): multiply by 2^-64 mod q
  for (int t = 0; t < ext; ++t) {
    const u64 q = c->mod[t];
    const u64 rinv = host_invmod((u64)(((unsigned __int128)1 << 64) % q), q);
    for (size_t r = 0; r < (size_t)c->n_digits * 2; ++r) {
      u64 *row = out + (r * ext + t) * c->n;
      for (u32 k2 = 0; k2 < c->n; ++k2) row[k2] = host_mulmod(row[k2], rinv, q);
    }
  }
  return CKKS_OK;
}

int ckks_pt_from_int(ckks_ctx *c, const int64_t *m, uint32_t level, uint64_t *pt) {
  if (!c || !m || !pt) return CKKS_E_PARAM;
  if ((int)level >= c->n_q) return CKKS_E_LEVEL;
  const u32 n = c->n;
  int rc = ensure_scratch(c, n);
  if (rc) return rc;
  i64 *dv = reinterpret_cast<i64 *>(c->scratch);
  CK_CUDA(cudaMemcpyAsync(dv, m, sizeof(i64) * n, cudaMemcpyHostToDevice, c->stream));
  rc = ew_signed_to_res(c, dv, pt, 0, level + 1);
  if (rc) return rc;
  int mods[MAX_MODS];
  for (u32 l = 0; l <= level; ++l) mods[l] = l;
  const u64 *s1[1] = {pt};
  u64 *d1[1] = {pt};
  rc = launch_ntt(c, s1, d1, 1, level + 1, mods, false);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int pt_from_int_ext(ckks_ctx *c, const int64_t *m, uint32_t level, uint64_t *pt) {
  if (!c || !m || !pt) return CKKS_E_PARAM;
  if ((int)level >= c->n_q) return CKKS_E_LEVEL;
  const u32 n = c->n;
  int rc = ensure_scratch(c, n);
  if (rc) return rc;
  i64 *dv = reinterpret_cast<i64 *>(c->scratch);
  CK_CUDA(cudaMemcpyAsync(dv, m, sizeof(i64) * n, cudaMemcpyHostToDevice, c->stream));
  rc = ew_signed_to_res(c, dv, pt, 0, level + 1);
  if (!rc) rc = ew_signed_to_res(c, dv, pt + (size_t)(level + 1) * n, c->n_q, c->n_p);
  if (rc) return rc;
  int mods[MAX_MODS];
  for (u32 l = 0; l <= level; ++l) mods[l] = l;
  for (int k = 0; k < c->n_p; ++k) mods[level + 1 + k] = c->n_q + k;
  const u64 *s1[1] = {pt};
  u64 *d1[1] = {pt};
  rc = launch_ntt(c, s1, d1, 1, level + 1 + c->n_p, mods, false);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_ntt(ckks_ctx *c, uint64_t *data, uint32_t n_limbs, uint32_t first_mod, int inverse) {
  if (!c || !data || n_limbs == 0 || first_mod + n_limbs > (u32)(c->n_q + c->n_p)) return CKKS_E_PARAM;
  int mods[MAX_MODS];
  for (u32 l = 0; l < n_limbs; ++l) mods[l] = first_mod + l;
  const u64 *s1[1] = {data};
  u64 *d1[1] = {data};
  return launch_ntt(c, s1, d1, 1, n_limbs, mods, inverse != 0);
}

int ckks_encrypt(ckks_ctx *c, const uint64_t *pt, uint32_t level, double scale, uint64_t enc_seed,
                 ckks_ct *out) {
  if (!c || !pt || !out || !out->data) return CKKS_E_PARAM;
  if (!c->have_secret) return CKKS_E_NOKEY;
  if ((int)level >= c->n_q || out->n_limbs < level + 1) return CKKS_E_LEVEL;
  const u32 n = c->n;
  const int nl = level + 1;
  int rc = ensure_scratch(c, (size_t)nl * n + n);
  if (rc) return rc;
  u64 *e_res = c->scratch;
  i64 *e_dev = reinterpret_cast<i64 *>(c->scratch + (size_t)nl * n);
  std::vector<i64> e(n);
  sample_gaussian(sm_stream(enc_seed, TAG_ENC_E, 0), n, c->sigma, c->e_bound, e.data());
  CK_CUDA(cudaMemcpyAsync(e_dev, e.data(), sizeof(i64) * n, cudaMemcpyHostToDevice, c->stream));
  rc = ew_signed_to_res(c, e_dev, e_res, 0, nl);
  if (rc) return rc;
  int mods[MAX_MODS];
  for (int l = 0; l < nl; ++l) mods[l] = l;
  const u64 *s1[1] = {e_res};
  u64 *d1[1] = {e_res};
  rc = launch_ntt(c, s1, d1, 1, nl, mods, false);
  if (rc) return rc;
  EncArgs ea;
  ea.key_a[0] = sm_stream(enc_seed, TAG_ENC_A, 0);
  ea.pt[0] = pt;
  ea.err[0] = e_res;
  ea.c0[0] = out->data;
  ea.c1[0] = poly1(out, n);
  rc = ew_encrypt(c, ea, nl, 1);
  if (rc) return rc;
  out->level = level;
  out->scale = scale;
  out->is_ntt = 1;
  out->log_n = c->log_n;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

// Signed host coefficients (n each, `count` polynomials) -> NTT-domain
// residues over q_0..q_{nl-1} at out + i * nl * N; uses the scratch after `out`.
static int upload_small_polys(ckks_ctx *c, const std::vector<i64> &host, int count, int nl, u64 *out) {
  const u32 n = c->n;
  i64 *dev = reinterpret_cast<i64 *>(out + (size_t)count * nl * n);
  CK_CUDA(cudaMemcpyAsync(dev, host.data(), sizeof(i64) * (size_t)count * n, cudaMemcpyHostToDevice, c->stream));
  std::vector<const u64 *> src(count);
  std::vector<u64 *> dst(count);
  for (int i = 0; i < count; ++i) {
    int rc = ew_signed_to_res(c, dev + (size_t)i * n, out + (size_t)i * nl * n, 0, nl);
    if (rc) return rc;
    src[i] = dst[i] = out + (size_t)i * nl * n;
  }
  int mods[MAX_MODS];
  for (int l = 0; l < nl; ++l) mods[l] = l;
  return launch_ntt(c, src.data(), dst.data(), count, nl, mods, false);
}

int ckks_keygen_public(ckks_ctx *c) {
  if (!c) return CKKS_E_PARAM;
  if (!c->have_secret) return CKKS_E_NOKEY;
  if (c->capturing) return CKKS_E_STATE;
  const u32 n = c->n;
  const int nl = c->n_q;
  if (!c->d_pk && cudaMalloc(&c->d_pk, sizeof(u64) * 2 * (size_t)nl * n) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  int rc = ensure_scratch(c, (size_t)nl * n + n);
  if (rc) return rc;
  std::vector<i64> e(n);
  sample_gaussian(sm_stream(c->key_seed, TAG_PK_E, 0), n, c->sigma, c->e_bound, e.data());
  rc = upload_small_polys(c, e, 1, nl, c->scratch);
  if (rc) return rc;
  // the secret-key encryption of 0: b = e - a s, a uniform from the key seed
  CK_CUDA(cudaMemsetAsync(c->d_pk, 0, sizeof(u64) * (size_t)nl * n, c->stream));
  EncArgs ea;
  ea.key_a[0] = sm_stream(c->key_seed, TAG_PK_A, 0);
  ea.pt[0] = c->d_pk;
  ea.err[0] = c->scratch;
  ea.c0[0] = c->d_pk;
  ea.c1[0] = c->d_pk + (size_t)nl * n;
  rc = ew_encrypt(c, ea, nl, 1);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_public_key_export(ckks_ctx *c, uint64_t *out) {
  if (!c || !out) return CKKS_E_PARAM;
  if (!c->d_pk) return CKKS_E_NOKEY;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  CK_CUDA(cudaMemcpy(out, c->d_pk, sizeof(u64) * 2 * (size_t)c->n_q * c->n, cudaMemcpyDeviceToHost));
  return CKKS_OK;
}

int ckks_encrypt_pk(ckks_ctx *c, const uint64_t *pt, uint32_t level, double scale, uint64_t enc_seed,
                    ckks_ct *out) {
  if (!c || !pt || !out || !out->data) return CKKS_E_PARAM;
  if (!c->d_pk) return CKKS_E_NOKEY;
  if ((int)level >= c->n_q || out->n_limbs < level + 1) return CKKS_E_LEVEL;
  const u32 n = c->n;
  const int nl = level + 1;
  int rc = ensure_scratch(c, 3 * (size_t)nl * n + 3 * (size_t)n);
  if (rc) return rc;
  std::vector<i64> h(3 * (size_t)n);
  sample_pk_mask(sm_stream(enc_seed, TAG_PKENC_V, 0), n, h.data());
  sample_gaussian(sm_stream(enc_seed, TAG_PKENC_E0, 0), n, c->sigma, c->e_bound, h.data() + n);
  sample_gaussian(sm_stream(enc_seed, TAG_PKENC_E1, 0), n, c->sigma, c->e_bound, h.data() + 2 * (size_t)n);
  rc = upload_small_polys(c, h, 3, nl, c->scratch);
  if (rc) return rc;
  EncPkArgs ea;
  ea.b = c->d_pk;
  ea.a = c->d_pk + (size_t)c->n_q * n;
  ea.v = c->scratch;
  ea.e0 = c->scratch + (size_t)nl * n;
  ea.e1 = c->scratch + 2 * (size_t)nl * n;
  ea.pt = pt;
  ea.c0 = out->data;
  ea.c1 = poly1(out, n);
  rc = ew_encrypt_pk(c, ea, nl);
  if (rc) return rc;
  out->level = level;
  out->scale = scale;
  out->is_ntt = 1;
  out->log_n = c->log_n;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_decrypt(ckks_ctx *c, const ckks_ct *ct, uint64_t *pt) {
  if (!c || !pt || !ct_ok(c, ct)) return CKKS_E_PARAM;
  if (!c->have_secret) return CKKS_E_NOKEY;
  EwArgs a;
  a.x0[0] = ct->data;
  a.x1[0] = poly1(ct, c->n);
  a.o0[0] = pt;
  return ew_decrypt(c, a, ct->level + 1, 1);
}

int ckks_add(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out) {
  if (!c || !ct_ok(c, a) || !ct_ok(c, b) || !out || !out->data) return CKKS_E_PARAM;
  if (a->level != b->level || out->n_limbs < a->level + 1) return CKKS_E_LEVEL;
  EwArgs e;
  e.x0[0] = a->data; e.x1[0] = poly1(a, c->n);
  e.y0[0] = b->data; e.y1[0] = poly1(b, c->n);
  e.o0[0] = out->data; e.o1[0] = poly1(out, c->n);
  const double s = a->scale;
  const u32 lv = a->level;
  int rc = ew_addsub(c, e, lv + 1, 1, false);
  if (rc) return rc;
  out->level = lv; out->scale = s; out->is_ntt = 1; out->log_n = c->log_n;
  return CKKS_OK;
}

int ckks_sub(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out) {
  if (!c || !ct_ok(c, a) || !ct_ok(c, b) || !out || !out->data) return CKKS_E_PARAM;
  if (a->level != b->level || out->n_limbs < a->level + 1) return CKKS_E_LEVEL;
  EwArgs e;
  e.x0[0] = a->data; e.x1[0] = poly1(a, c->n);
  e.y0[0] = b->data; e.y1[0] = poly1(b, c->n);
  e.o0[0] = out->data; e.o1[0] = poly1(out, c->n);
  const double s = a->scale;
  const u32 lv = a->level;
  int rc = ew_addsub(c, e, lv + 1, 1, true);
  if (rc) return rc;
  out->level = lv; out->scale = s; out->is_ntt = 1; out->log_n = c->log_n;
  return CKKS_OK;
}

int ckks_mul_plain(ckks_ctx *c, const ckks_ct *a, const uint64_t *pt, double pt_scale, ckks_ct *out) {
  if (!c || !ct_ok(c, a) || !pt || !out || !out->data) return CKKS_E_PARAM;
  if (out->n_limbs < a->level + 1) return CKKS_E_LEVEL;
  EwArgs e;
  e.x0[0] = a->data; e.x1[0] = poly1(a, c->n);
  e.y0[0] = pt;
  e.o0[0] = out->data; e.o1[0] = poly1(out, c->n);
  const double s = a->scale * pt_scale;
  const u32 lv = a->level;
  int rc = ew_plain(c, e, lv + 1, 1, 0);
  if (rc) return rc;
  out->level = lv; out->scale = s; out->is_ntt = 1; out->log_n = c->log_n;
  return CKKS_OK;
}

int ckks_add_plain(ckks_ctx *c, const ckks_ct *a, const uint64_t *pt, ckks_ct *out) {
  if (!c || !ct_ok(c, a) || !pt || !out || !out->data) return CKKS_E_PARAM;
  if (out->n_limbs < a->level + 1) return CKKS_E_LEVEL;
  EwArgs e;
  e.x0[0] = a->data; e.x1[0] = poly1(a, c->n);
  e.y0[0] = pt;
  e.o0[0] = out->data; e.o1[0] = poly1(out, c->n);
  const double s = a->scale;
  const u32 lv = a->level;
  int rc = ew_plain(c, e, lv + 1, 1, 1);
  if (rc) return rc;
  out->level = lv; out->scale = s; out->is_ntt = 1; out->log_n = c->log_n;
  return CKKS_OK;
}

int ckks_mul_int(ckks_ctx *c, const ckks_ct *a, int64_t k, ckks_ct *out) {
  if (!c || !ct_ok(c, a) || !out || !out->data) return CKKS_E_PARAM;
  if (out->n_limbs < a->level + 1) return CKKS_E_LEVEL;
  EwArgs e;
  e.x0[0] = a->data; e.x1[0] = poly1(a, c->n);
  e.o0[0] = out->data; e.o1[0] = poly1(out, c->n);
  const double s = a->scale;
  const u32 lv = a->level;
  int rc = ew_mul_int(c, e, lv + 1, 1, k);
  if (rc) return rc;
  out->level = lv; out->scale = s; out->is_ntt = 1; out->log_n = c->log_n;
  return CKKS_OK;
}

int ckks_mul_relin_batch(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n,
                         int do_rescale) {
  if (!c || !a || !b || !out || n < 0) return CKKS_E_PARAM;
  if (n == 0) return CKKS_OK;
  const u32 level = a[0].level;
  for (int i = 0; i < n; ++i) {
    if (!ct_ok(c, &a[i]) || !ct_ok(c, &b[i]) || !out[i].data) return CKKS_E_PARAM;
    if (a[i].level != level || b[i].level != level || out[i].n_limbs < level + 1) return CKKS_E_LEVEL;
  }
  if (do_rescale < CKKS_RESCALE_NONE || do_rescale > CKKS_RESCALE_MERGED) return CKKS_E_PARAM;
  if (do_rescale && level == 0) return CKKS_E_LEVEL;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    int rc = mul_relin_chunk(c, a + i0, b + i0, out + i0, cnt, do_rescale == CKKS_RESCALE_MERGED);
    if (rc) return rc;
    if (do_rescale == CKKS_RESCALE_SEPARATE) {
      rc = rescale_chunk(c, out + i0, cnt);
      if (rc) return rc;
    }
  }
  return last_err();
}

int ckks_mul_relin(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out) {
  return ckks_mul_relin_batch(c, a, b, out, 1, 0);
}

int ckks_rescale_batch(ckks_ctx *c, ckks_ct *cts, int n) {
  if (!c || !cts || n < 0) return CKKS_E_PARAM;
  if (n == 0) return CKKS_OK;
  const u32 level = cts[0].level;
  for (int i = 0; i < n; ++i) {
    if (!ct_ok(c, &cts[i])) return CKKS_E_PARAM;
    if (cts[i].level != level) return CKKS_E_LEVEL;
  }
  if (level == 0) return CKKS_E_LEVEL;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    int rc = rescale_chunk(c, cts + i0, std::min(MAX_CTS, n - i0));
    if (rc) return rc;
  }
  return CKKS_OK;
}

int ckks_rescale(ckks_ctx *c, ckks_ct *ct) { return ckks_rescale_batch(c, ct, 1); }

// ---- batched element-wise calls (one launch per <= 128 ciphertexts) ----
namespace {
int ew_batch_check(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n) {
  if (!c || !a || !out || n < 0) return CKKS_E_PARAM;
  for (int i = 0; i < n; ++i) {
    if (!ct_ok(c, &a[i]) || (b && !ct_ok(c, &b[i])) || !out[i].data) return CKKS_E_PARAM;
    if (a[i].level != a[0].level || (b && b[i].level != a[0].level) || out[i].n_limbs < a[0].level + 1)
      return CKKS_E_LEVEL;
  }
  return CKKS_OK;
}
void ew_fill(ckks_ctx *c, EwArgs &e, const ckks_ct *a, const ckks_ct *b, const u64 *pt, ckks_ct *out, int i0,
             int cnt) {
  for (int i = 0; i < cnt; ++i) {
    e.x0[i] = a[i0 + i].data;
    e.x1[i] = poly1(&a[i0 + i], c->n);
    e.y0[i] = b ? b[i0 + i].data : pt;
    e.y1[i] = b ? poly1(&b[i0 + i], c->n) : nullptr;
    e.o0[i] = out[i0 + i].data;
    e.o1[i] = poly1(&out[i0 + i], c->n);
  }
}
void ew_finish(ckks_ctx *c, const ckks_ct *a, ckks_ct *out, int n, const double *scales) {
  for (int i = 0; i < n; ++i) {
    out[i].level = a[0].level;
    out[i].scale = scales[i];
    out[i].is_ntt = 1;
    out[i].log_n = c->log_n;
  }
}
}  // namespace

int ckks_add_batch(ckks_ctx *c, const ckks_ct *a, const ckks_ct *b, ckks_ct *out, int n, int subtract) {
  int rc = ew_batch_check(c, a, b, out, n);
  if (rc || n == 0) return rc;
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = a[i].scale;
  const int nl = a[0].level + 1;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    EwArgs e;
    ew_fill(c, e, a, b, nullptr, out, i0, cnt);
    rc = ew_addsub(c, e, nl, cnt, subtract != 0);
    if (rc) return rc;
  }
  ew_finish(c, a, out, n, s.data());
  return CKKS_OK;
}

int ckks_mul_int_batch(ckks_ctx *c, const ckks_ct *a, int64_t k, ckks_ct *out, int n) {
  int rc = ew_batch_check(c, a, nullptr, out, n);
  if (rc || n == 0) return rc;
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = a[i].scale;
  const int nl = a[0].level + 1;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    EwArgs e;
    ew_fill(c, e, a, nullptr, nullptr, out, i0, cnt);
    rc = ew_mul_int(c, e, nl, cnt, k);
    if (rc) return rc;
  }
  ew_finish(c, a, out, n, s.data());
  return CKKS_OK;
}

int ckks_mul_plain_batch(ckks_ctx *c, const ckks_ct *a, const uint64_t *pt, double pt_scale, ckks_ct *out, int n) {
  if (!pt) return CKKS_E_PARAM;
  int rc = ew_batch_check(c, a, nullptr, out, n);
  if (rc || n == 0) return rc;
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = a[i].scale * pt_scale;
  const int nl = a[0].level + 1;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    EwArgs e;
    ew_fill(c, e, a, nullptr, pt, out, i0, cnt);
    rc = ew_plain(c, e, nl, cnt, 0);
    if (rc) return rc;
  }
  ew_finish(c, a, out, n, s.data());
  return CKKS_OK;
}

int ckks_add_plain_batch(ckks_ctx *c, const ckks_ct *a, const uint64_t *pt, ckks_ct *out, int n) {
  if (!pt) return CKKS_E_PARAM;
  int rc = ew_batch_check(c, a, nullptr, out, n);
  if (rc || n == 0) return rc;
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = a[i].scale;
  const int nl = a[0].level + 1;
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    EwArgs e;
    ew_fill(c, e, a, nullptr, pt, out, i0, cnt);
    rc = ew_plain(c, e, nl, cnt, 1);
    if (rc) return rc;
  }
  ew_finish(c, a, out, n, s.data());
  return CKKS_OK;
}

int ckks_automorph(ckks_ctx *c, const ckks_ct *a, uint64_t g, ckks_ct *out) {
  if (!c || !ct_ok(c, a) || !out || !out->data) return CKKS_E_PARAM;
  if (out->n_limbs < a->level + 1) return CKKS_E_LEVEL;
  u64 gg = g;
  return automorph_chunk(c, a, &gg, out, 1);
}

int ckks_rotate(ckks_ctx *c, const ckks_ct *a, int32_t k, ckks_ct *out) {
  if (!c) return CKKS_E_PARAM;
  return ckks_automorph(c, a, ckks_galois_elt(c, k), out);
}

int ckks_conjugate(ckks_ctx *c, const ckks_ct *a, ckks_ct *out) {
  if (!c) return CKKS_E_PARAM;
  return ckks_automorph(c, a, 2ULL * c->n - 1, out);
}

int ckks_rotate_batch(ckks_ctx *c, const ckks_ct *in, const int32_t *k, ckks_ct *out, int n) {
  if (!c || !in || !k || !out || n < 0) return CKKS_E_PARAM;
  if (n == 0) return CKKS_OK;
  const u32 level = in[0].level;
  for (int i = 0; i < n; ++i) {
    if (!ct_ok(c, &in[i]) || !out[i].data) return CKKS_E_PARAM;
    if (in[i].level != level || out[i].n_limbs < level + 1) return CKKS_E_LEVEL;
  }
  for (int i0 = 0; i0 < n; i0 += MAX_CTS) {
    const int cnt = std::min(MAX_CTS, n - i0);
    std::vector<u64> g(cnt);
    for (int i = 0; i < cnt; ++i) g[i] = ckks_galois_elt(c, k[i0 + i]);
    int rc = automorph_chunk(c, in + i0, g.data(), out + i0, cnt);
    if (rc) return rc;
  }
  return CKKS_OK;
}

// The host-streamed multiply in either wire format: raw (uint64 limbs) or
// packed (limbs at their primes' bit widths, unpacked and packed on the GPU).
static int mul_relin_host_impl(ckks_ctx *c, const void *a_host, const void *b_host, double scale_a,
                               double scale_b, uint32_t level, int n, int do_rescale, int chunk, void *out_host,
                               double *out_scale, bool packed) {
  if (!c || !a_host || !b_host || !out_host || n < 0 || chunk < 1 || chunk > MAX_CTS) return CKKS_E_PARAM;
  if (level >= (uint32_t)c->n_q) return CKKS_E_LEVEL;
  if (do_rescale < CKKS_RESCALE_NONE || do_rescale > CKKS_RESCALE_MERGED) return CKKS_E_PARAM;
  if (do_rescale && level == 0) return CKKS_E_LEVEL;
  if (c->capturing) return CKKS_E_STATE;
  if (n == 0) return CKKS_OK;
  const u32 nn = c->n;
  const uint32_t out_level = do_rescale ? level - 1 : level;
  const size_t in_w = (size_t)2 * (level + 1) * nn, out_w = (size_t)2 * (out_level + 1) * nn;
  const WireLayout Lin = wire_layout(c, (int)level), Lout = wire_layout(c, (int)out_level);
  const size_t win = packed ? (size_t)2 * Lin.off[Lin.nl] / 8 : 0;    // words per packed input
  const size_t wout = packed ? (size_t)2 * Lout.off[Lout.nl] / 8 : 0;  // words per packed output
  // per slot: a, b and the product (full capacity), then the packed a, b and product
  const size_t slot_w = (size_t)chunk * (3 * in_w + 2 * win + wout);
  if (!c->h2d) CK_CUDA(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking));
  if (!c->d2h) CK_CUDA(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking));
  for (int i = 0; i < 3; ++i) {
    if (!c->ev_in[i]) CK_CUDA(cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming));
    if (!c->ev_comp[i]) CK_CUDA(cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming));
    if (!c->ev_out[i]) CK_CUDA(cudaEventCreateWithFlags(&c->ev_out[i], cudaEventDisableTiming));
  }
  if (c->stage_words < 3 * slot_w) {
    CK_CUDA(cudaStreamSynchronize(c->d2h));
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_words = 0;
    if (cudaMalloc(&c->stage, sizeof(u64) * 3 * slot_w) != cudaSuccess) {
      cudaGetLastError();
      return CKKS_E_OOM;
    }
    c->stage_words = 3 * slot_w;
  }
  double sc = 0.0;
  // chunk sizes: ramped up at the start and down at the end (chunk/4, chunk/2,
  // chunk, ..., chunk/2, chunk/4), so that the first copy-in and the last
  // product and copy-out, which overlap nothing, are short
  std::vector<int> sizes;
  {
    std::vector<int> head, tail;
    int left = n;
    for (int d = 4; d >= 2 && left > 0; d /= 2) {
      const int a = std::max(1, chunk / d);
      if (left >= 2 * a + chunk) {
        head.push_back(a);
        tail.push_back(a);
        left -= 2 * a;
      }
    }
    sizes = head;
    while (left > 0) {
      const int a = std::min(chunk, left);
      sizes.push_back(a);
      left -= a;
    }
    sizes.insert(sizes.end(), tail.rbegin(), tail.rend());
  }
  const int nchunks = (int)sizes.size();
  const u64 *a64 = static_cast<const u64 *>(a_host), *b64 = static_cast<const u64 *>(b_host);
  u64 *o64 = static_cast<u64 *>(out_host);
  for (int ci = 0, i0 = 0; ci < nchunks; i0 += sizes[ci], ++ci) {
    const int s = ci % 3, cnt = sizes[ci];
    u64 *sa = c->stage + (size_t)s * slot_w, *sb = sa + (size_t)chunk * in_w, *so = sb + (size_t)chunk * in_w;
    u64 *pa = so + (size_t)chunk * in_w, *pb = pa + (size_t)chunk * win, *po = pb + (size_t)chunk * win;
    // inputs of this chunk, once the slot's previous products have left
    CK_CUDA(cudaStreamWaitEvent(c->h2d, c->ev_out[s], 0));
    const size_t iw = packed ? win : in_w;
    CK_CUDA(cudaMemcpyAsync(packed ? pa : sa, a64 + (size_t)i0 * iw, sizeof(u64) * cnt * iw, cudaMemcpyHostToDevice,
                            c->h2d));
    CK_CUDA(cudaMemcpyAsync(packed ? pb : sb, b64 + (size_t)i0 * iw, sizeof(u64) * cnt * iw, cudaMemcpyHostToDevice,
                            c->h2d));
    CK_CUDA(cudaEventRecord(c->ev_in[s], c->h2d));
    // the products on the context stream
    CK_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in[s], 0));
    std::vector<ckks_ct> ha(cnt), hb(cnt), ho(cnt);
    std::vector<unsigned char *> wa(cnt), wb(cnt), wo(cnt);
    std::vector<u64 *> ca(cnt), cb(cnt), co(cnt);
    std::vector<u32> nlim(cnt, level + 1);
    for (int i = 0; i < cnt; ++i) {
      const uint32_t ln = (uint32_t)c->log_n;
      ha[i] = ckks_ct{sa + (size_t)i * in_w, ln, level, level + 1, 1, scale_a};
      hb[i] = ckks_ct{sb + (size_t)i * in_w, ln, level, level + 1, 1, scale_b};
      ho[i] = ckks_ct{so + (size_t)i * in_w, ln, level, level + 1, 1, 1.0};
      wa[i] = reinterpret_cast<unsigned char *>(pa + (size_t)i * win);
      wb[i] = reinterpret_cast<unsigned char *>(pb + (size_t)i * win);
      wo[i] = reinterpret_cast<unsigned char *>(po + (size_t)i * wout);
      ca[i] = ha[i].data;
      cb[i] = hb[i].data;
      co[i] = ho[i].data;
    }
    int rc = CKKS_OK;
    if (packed) {
      rc = ew_wire(c, Lin, wa.data(), ca.data(), nlim.data(), cnt, false);
      if (!rc) rc = ew_wire(c, Lin, wb.data(), cb.data(), nlim.data(), cnt, false);
      if (rc) return rc;
    }
    rc = ckks_mul_relin_batch(c, ha.data(), hb.data(), ho.data(), cnt, do_rescale);
    if (rc) return rc;
    if (packed) {
      rc = ew_wire(c, Lout, wo.data(), co.data(), nlim.data(), cnt, true);
      if (rc) return rc;
    }
    sc = ho[0].scale;
    CK_CUDA(cudaEventRecord(c->ev_comp[s], c->stream));
    // the products back
    CK_CUDA(cudaStreamWaitEvent(c->d2h, c->ev_comp[s], 0));
    if (packed) {  // contiguous per chunk
      CK_CUDA(cudaMemcpyAsync(o64 + (size_t)i0 * wout, po, sizeof(u64) * cnt * wout, cudaMemcpyDeviceToHost,
                              c->d2h));
    } else {  // the active limbs of both polynomials, contiguous per pair
      const size_t half = out_w / 2;
      for (int i = 0; i < cnt; ++i) {
        u64 *dst = o64 + (size_t)(i0 + i) * out_w;
        CK_CUDA(cudaMemcpyAsync(dst, ho[i].data, sizeof(u64) * half, cudaMemcpyDeviceToHost, c->d2h));
        CK_CUDA(cudaMemcpyAsync(dst + half, ho[i].data + (size_t)(level + 1) * nn, sizeof(u64) * half,
                                cudaMemcpyDeviceToHost, c->d2h));
      }
    }
    CK_CUDA(cudaEventRecord(c->ev_out[s], c->d2h));
  }
  CK_CUDA(cudaStreamSynchronize(c->d2h));
  if (out_scale) *out_scale = sc;
  return last_err();
}

int ckks_mul_relin_host(ckks_ctx *c, const uint64_t *a_host, const uint64_t *b_host, double scale_a,
                        double scale_b, uint32_t level, int n, int do_rescale, int chunk, uint64_t *out_host,
                        double *out_scale) {
  return mul_relin_host_impl(c, a_host, b_host, scale_a, scale_b, level, n, do_rescale, chunk, out_host, out_scale,
                             false);
}

int ckks_mul_relin_host_packed(ckks_ctx *c, const uint8_t *a_host, const uint8_t *b_host, double scale_a,
                               double scale_b, uint32_t level, int n, int do_rescale, int chunk, uint8_t *out_host,
                               double *out_scale) {
  if (((uintptr_t)a_host | (uintptr_t)b_host | (uintptr_t)out_host) & 7) return CKKS_E_PARAM;
  return mul_relin_host_impl(c, a_host, b_host, scale_a, scale_b, level, n, do_rescale, chunk, out_host, out_scale,
                             true);
}

int ckks_wire_bytes(const ckks_ctx *c, uint32_t level, uint64_t *bytes) {
  if (!c || !bytes) return CKKS_E_PARAM;
  if (level >= (uint32_t)c->n_q) return CKKS_E_LEVEL;
  const WireLayout L = wire_layout(c, (int)level);
  *bytes = (uint64_t)2 * L.off[L.nl];
  return CKKS_OK;
}

int ckks_ct_export_packed(ckks_ctx *c, const ckks_ct *ct, uint8_t *out) {
  if (!c || !ct_ok(c, ct) || !out || ((uintptr_t)out & 7)) return CKKS_E_PARAM;
  const WireLayout L = wire_layout(c, (int)ct->level);
  const size_t bytes = (size_t)2 * L.off[L.nl];
  int rc = ensure_scratch(c, bytes / 8);
  if (rc) return rc;
  unsigned char *w = reinterpret_cast<unsigned char *>(c->scratch);
  u64 *d = ct->data;
  const u32 nl = ct->n_limbs;
  rc = ew_wire(c, L, &w, &d, &nl, 1, true);
  if (rc) return rc;
  CK_CUDA(cudaMemcpyAsync(out, w, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_ct_import_packed(ckks_ctx *c, const uint8_t *in, ckks_ct *ct) {
  if (!c || !ct_ok(c, ct) || !in || ((uintptr_t)in & 7)) return CKKS_E_PARAM;
  const WireLayout L = wire_layout(c, (int)ct->level);
  const size_t bytes = (size_t)2 * L.off[L.nl];
  int rc = ensure_scratch(c, bytes / 8);
  if (rc) return rc;
  unsigned char *w = reinterpret_cast<unsigned char *>(c->scratch);
  CK_CUDA(cudaMemcpyAsync(w, in, bytes, cudaMemcpyHostToDevice, c->stream));
  u64 *d = ct->data;
  const u32 nl = ct->n_limbs;
  rc = ew_wire(c, L, &w, &d, &nl, 1, false);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_ct_export_ntt(ckks_ctx *c, const ckks_ct *ct, uint64_t *out) {
  if (!c || !ct_ok(c, ct) || !out) return CKKS_E_PARAM;
  const size_t w = (size_t)(ct->level + 1) * c->n;
  CK_CUDA(cudaMemcpyAsync(out, ct->data, w * 8, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaMemcpyAsync(out + w, poly1(ct, c->n), w * 8, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_ct_import_ntt(ckks_ctx *c, const uint64_t *in, ckks_ct *ct) {
  if (!c || !ct_ok(c, ct) || !in) return CKKS_E_PARAM;
  const size_t w = (size_t)(ct->level + 1) * c->n;
  CK_CUDA(cudaMemcpyAsync(ct->data, in, w * 8, cudaMemcpyHostToDevice, c->stream));
  CK_CUDA(cudaMemcpyAsync(poly1(ct, c->n), in + w, w * 8, cudaMemcpyHostToDevice, c->stream));
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

// Coefficient domain: the active limbs of both polynomials go through the
// inverse NTT into the context scratch, then to the host.
int ckks_ct_export(ckks_ctx *c, const ckks_ct *ct, uint64_t *out) {
  if (!c || !ct_ok(c, ct) || !out) return CKKS_E_PARAM;
  if (c->capturing) return CKKS_E_STATE;
  const int nl = (int)ct->level + 1;
  const size_t w = (size_t)nl * c->n;
  int rc = ensure_scratch(c, 2 * w);
  if (rc) return rc;
  int mods[MAX_MODS];
  for (int t = 0; t < nl; ++t) mods[t] = t;
  const u64 *src[2] = {ct->data, poly1(ct, c->n)};
  u64 *dst[2] = {c->scratch, c->scratch + w};
  rc = launch_ntt(c, src, dst, 2, nl, mods, true);
  if (rc) return rc;
  CK_CUDA(cudaMemcpyAsync(out, c->scratch, 2 * w * 8, cudaMemcpyDeviceToHost, c->stream));
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

// Coefficient-domain limbs in [0, q_t) (checked on the host: CKKS_E_PARAM),
// copied in, then transformed to the NTT domain in place.
int ckks_ct_import(ckks_ctx *c, const uint64_t *in, ckks_ct *ct) {
  if (!c || !ct_ok(c, ct) || !in) return CKKS_E_PARAM;
  const int nl = (int)ct->level + 1;
  const size_t w = (size_t)nl * c->n;
  for (int p = 0; p < 2; ++p)
    for (int t = 0; t < nl; ++t) {
      const u64 q = c->mod[t], *row = in + (size_t)p * w + (size_t)t * c->n;
      for (u32 k = 0; k < c->n; ++k)
        if (row[k] >= q) return CKKS_E_PARAM;
    }
  CK_CUDA(cudaMemcpyAsync(ct->data, in, w * 8, cudaMemcpyHostToDevice, c->stream));
  CK_CUDA(cudaMemcpyAsync(poly1(ct, c->n), in + w, w * 8, cudaMemcpyHostToDevice, c->stream));
  int mods[MAX_MODS];
  for (int t = 0; t < nl; ++t) mods[t] = t;
  const u64 *src[2] = {ct->data, poly1(ct, c->n)};
  u64 *dst[2] = {ct->data, poly1(ct, c->n)};
  int rc = launch_ntt(c, src, dst, 2, nl, mods, false);
  if (rc) return rc;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  return CKKS_OK;
}

int ckks_ct_alloc(ckks_ctx *c, uint32_t n_limbs, ckks_ct *out) {
  if (!c || !out || n_limbs < 1 || n_limbs > (uint32_t)c->n_q) return CKKS_E_PARAM;
  if (c->capturing) return CKKS_E_STATE;
  void *p = nullptr;
  const size_t bytes = (size_t)2 * n_limbs * c->n * sizeof(u64);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CKKS_E_OOM;
  }
  if (cudaMemsetAsync(p, 0, bytes, c->stream) != cudaSuccess) {
    cudaFree(p);
    return CKKS_E_CUDA;
  }
  *out = ckks_ct{static_cast<uint64_t *>(p), (uint32_t)c->log_n, n_limbs - 1, n_limbs, 1, c->default_scale};
  return CKKS_OK;
}

int ckks_ct_free(ckks_ctx *c, ckks_ct *ct) {
  if (!c || !ct) return CKKS_E_PARAM;
  if (c->capturing) return CKKS_E_STATE;
  if (!ct->data) return CKKS_OK;
  CK_CUDA(cudaStreamSynchronize(c->stream));
  CK_CUDA(cudaFree(ct->data));
  ct->data = nullptr;
  return CKKS_OK;
}

}  // extern "C"
