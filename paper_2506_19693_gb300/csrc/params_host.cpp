// Host-side parameter derivation: prime chain (reading C1), roots (C2), NTT
// twiddle tables and the basis-conversion constants of ModUp / ModDown /
// rescale (C8-C10), uploaded once per context.
#include <cstring>
#include <vector>

#include "ctx.h"

typedef unsigned __int128 u128;

u64 host_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 host_powmod(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  for (; e; e >>= 1) {
    if (e & 1) r = host_mulmod(r, b, q);
    b = host_mulmod(b, b, q);
  }
  return r;
}
u64 host_invmod(u64 a, u64 q) {
  // extended Euclid over signed 128-bit
  __int128 t = 0, nt = 1, r = q, nr = a % q;
  while (nr != 0) {
    __int128 quo = r / nr, tmp;
    tmp = t - quo * nt; t = nt; nt = tmp;
    tmp = r - quo * nr; r = nr; nr = tmp;
  }
  if (t < 0) t += q;
  return (u64)t;
}
u64 host_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
u64 host_bitrev(u64 x, int bits) {
  u64 r = 0;
  for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// Strong-probable-prime test to the bases 2..37 (deterministic for 64 bits).
static bool sprp(u64 n, u64 a) {
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) { d >>= 1; ++s; }
  u64 x = host_powmod(a, d, n);
  if (x == 1 || x == n - 1) return true;
  for (int i = 1; i < s; ++i) {
    x = host_mulmod(x, x, n);
    if (x == n - 1) return true;
  }
  return false;
}
static bool is_prime(u64 n) {
  const u64 base[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : base)
    if (n % p == 0) return n == p;
  for (u64 a : base)
    if (!sprp(n, a)) return false;
  return true;
}

// C1: per bit size b, candidates 2^b + 1 - m 2^e (m = 1, 2, ...) with
// e = log_step = max(17, log2(2N)), primes kept in order of discovery; each
// chain entry takes the next one of its size.
int host_gen_primes(int count, const unsigned *bits, int log_step, u64 *out) {
  u64 cursor[64];
  if (log_step < 17 || log_step > 40) return CKKS_E_PARAM;
  for (int i = 0; i < 64; ++i) cursor[i] = 1;
  for (int i = 0; i < count; ++i) {
    unsigned b = bits[i];
    if (b < 20 || b > 62) return CKKS_E_PARAM;
    while (true) {
      u64 m = cursor[b]++;
      if ((m << log_step) >= (1ULL << b)) return CKKS_E_PARAM;
      u64 cand = (1ULL << b) + 1 - (m << log_step);
      if (is_prime(cand)) { out[i] = cand; break; }
    }
  }
  return CKKS_OK;
}

// C2: psi = g^((q-1)/2N) for the least quadratic non-residue g >= 2.
u64 host_find_psi(u64 q, u64 n) {
  u64 g = 2;
  while (host_powmod(g, (q - 1) >> 1, q) != q - 1) ++g;
  return host_powmod(g, (q - 1) / (2 * n), q);
}

static void push_pair(std::vector<u64> &v, u64 w, u64 q) {
  v.push_back(w);
  v.push_back(host_shoup(w, q));
}

int build_tables(ckks_ctx *c) {
  const int nm = c->n_q + c->n_p;
  const u32 n = c->n;
  // ---- per-modulus scalars ----
  std::vector<ModInfo> mi(nm);
  for (int i = 0; i < nm; ++i) {
    u64 q = c->mod[i];
    ModInfo m{};
    m.q = q;
    m.twoq = 2 * q;
    m.r64 = (u64)(((u128)1 << 64) % q);
    m.r64_s = host_shoup(m.r64, q);
    m.one_s = (u64)(((u128)1 << 64) / q);
    m.ninv = host_invmod(n % q, q);
    m.ninv_s = host_shoup(m.ninv, q);
    u64 inv = q;  // q^-1 mod 2^64 by Newton's iteration (q odd: 5 doublings of 3 correct bits)
    for (int it = 0; it < 5; ++it) inv *= 2 - q * inv;
    m.qinv_neg = (u64)0 - inv;
    mi[i] = m;
  }
  // ---- twiddles: tw[k] = psi^brv(k) (k in [0, N)), inverse with psi^-1 ----
  std::vector<ulonglong2> fwd((size_t)nm * n), inv((size_t)nm * n);
  for (int i = 0; i < nm; ++i) {
    u64 q = c->mod[i], psi = c->psi[i], ipsi = host_invmod(psi, q);
    std::vector<u64> pw(n), ipw(n);
    pw[0] = ipw[0] = 1;
    for (u32 k = 1; k < n; ++k) {
      pw[k] = host_mulmod(pw[k - 1], psi, q);
      ipw[k] = host_mulmod(ipw[k - 1], ipsi, q);
    }
    for (u32 k = 0; k < n; ++k) {
      u64 e = host_bitrev(k, c->log_n);
      fwd[(size_t)i * n + k] = make_ulonglong2(pw[e], host_shoup(pw[e], q));
      inv[(size_t)i * n + k] = make_ulonglong2(ipw[e], host_shoup(ipw[e], q));
    }
    // index 0 is never a stage twiddle (stage m uses indices m..2m-1): the
    // inverse table keeps there psi^-brv(1) N^-1, the last stage's twiddle
    // with the final N^-1 folded in
    const u64 w0 = host_mulmod(inv[(size_t)i * n + 1].x, mi[i].ninv, q);
    inv[(size_t)i * n] = make_ulonglong2(w0, host_shoup(w0, q));
  }
  // ---- the row pass's twiddles, regrouped (see ctx.h) ----
  const size_t n16 = n / 16, row_per = 15 * n16;
  std::vector<ulonglong2> rfwd((size_t)nm * row_per), rinv((size_t)nm * row_per);
  for (int i = 0; i < nm; ++i)
    for (int s2 = 0; s2 < 4; ++s2)
      for (int ii = 0; ii < (1 << s2); ++ii)
        for (size_t m2 = 0; m2 < n16; ++m2) {
          const size_t dst = (size_t)i * row_per + (size_t)((1 << s2) - 1 + ii) * n16 + m2;
          const size_t src = (size_t)i * n + (((n16 + m2) << s2) + ii);
          rfwd[dst] = fwd[src];
          rinv[dst] = inv[src];
        }
  // ---- basis conversion constants ----
  ConvTables &t = c->conv;
  std::vector<u64> &v = c->h_conv;
  v.clear();
  const int K = c->n_p;
  t.modup_off.assign((size_t)c->n_q * c->n_digits, 0);
  for (int l = 0; l < c->n_q; ++l) {
    for (int j = 0; j < c->n_digits; ++j) {
      int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, l + 1);
      t.modup_off[(size_t)l * c->n_digits + j] = v.size();
      if (lo >= hi) continue;
      int ns = hi - lo;
      for (int i = 0; i < ns; ++i) {
        u64 qi = c->mod[lo + i], prod = 1;
        for (int k = 0; k < ns; ++k)
          if (k != i) prod = host_mulmod(prod, c->mod[lo + k] % qi, qi);
        push_pair(v, host_invmod(prod, qi), qi);
      }
      // targets: q_0..q_l except [lo,hi), then p_0..p_{K-1}
      for (int tt = 0; tt < l + 1 + K; ++tt) {
        if (tt >= lo && tt < hi) continue;
        u64 mt = c->mod[c->ext_mod(l, tt)];
        for (int i = 0; i < ns; ++i) {
          u64 prod = 1;
          for (int k = 0; k < ns; ++k)
            if (k != i) prod = host_mulmod(prod, c->mod[lo + k] % mt, mt);
          v.push_back(prod);
        }
      }
    }
  }
  t.moddown_phat_inv = v.size();
  for (int k = 0; k < K; ++k) {
    u64 pk = c->mod[c->n_q + k], prod = 1;
    for (int r = 0; r < K; ++r)
      if (r != k) prod = host_mulmod(prod, c->mod[c->n_q + r] % pk, pk);
    push_pair(v, host_invmod(prod, pk), pk);
  }
  t.moddown_phat_mod = v.size();
  for (int i = 0; i < c->n_q; ++i) {
    u64 qi = c->mod[i];
    for (int k = 0; k < K; ++k) {
      u64 prod = 1;
      for (int r = 0; r < K; ++r)
        if (r != k) prod = host_mulmod(prod, c->mod[c->n_q + r] % qi, qi);
      v.push_back(prod);
    }
  }
  t.moddown_pinv = v.size();
  for (int i = 0; i < c->n_q; ++i) {
    u64 qi = c->mod[i], prod = 1;
    for (int k = 0; k < K; ++k) prod = host_mulmod(prod, c->mod[c->n_q + k] % qi, qi);
    push_pair(v, host_invmod(prod, qi), qi);
  }
  t.mdr_off.assign(c->n_q, 0);
  for (int l = 1; l < c->n_q; ++l) {
    t.mdr_off[l] = v.size();
    std::vector<u64> smod(K + 1);  // the sources s_0 = q_l, s_{1+k} = p_k
    smod[0] = c->mod[l];
    for (int k = 0; k < K; ++k) smod[1 + k] = c->mod[c->n_q + k];
    auto shat_mod = [&](int i, u64 m) {  // (S / s_i) mod m; i = -1 gives S mod m
      u64 prod = 1;
      for (int r = 0; r <= K; ++r)
        if (r != i) prod = host_mulmod(prod, smod[r] % m, m);
      return prod;
    };
    std::vector<u64> inv(K + 1);
    for (int i = 0; i <= K; ++i) {
      inv[i] = host_invmod(shat_mod(i, smod[i]), smod[i]);
      push_pair(v, inv[i], smod[i]);
    }
    for (int tt = 0; tt < l; ++tt)
      for (int i = 0; i <= K; ++i) v.push_back(shat_mod(i, c->mod[tt]));
    for (int i = 0; i <= K; ++i) v.push_back(host_mulmod((smod[i] - 1) / 2, inv[i], smod[i]));
    for (int tt = 0; tt < l; ++tt) {  // (S - 1)/2 mod q_t
      const u64 qt = c->mod[tt], sm = shat_mod(-1, qt);
      v.push_back(host_mulmod((sm + qt - 1) % qt, (qt + 1) / 2, qt));
    }
    for (int tt = 0; tt < l; ++tt) push_pair(v, host_invmod(shat_mod(-1, c->mod[tt]), c->mod[tt]), c->mod[tt]);
    for (int tt = 0; tt < l; ++tt) push_pair(v, host_invmod(c->mod[l] % c->mod[tt], c->mod[tt]), c->mod[tt]);
    u64 pm = 1;
    for (int k = 0; k < K; ++k) pm = host_mulmod(pm, c->mod[c->n_q + k] % c->mod[l], c->mod[l]);
    push_pair(v, pm, c->mod[l]);
    for (int i = 0; i <= K; ++i) v.push_back((u64)(((unsigned __int128)1 << 96) / smod[i]));  // R_i low words
    for (int i = 0; i <= K; ++i)  // R_i high words: nonzero only for s_i < 2^32
      v.push_back((u64)((((unsigned __int128)1 << 96) / smod[i]) >> 64));
    for (int tt = 0; tt < l; ++tt) {                                                          // -S mod q_t
      const u64 qt = c->mod[tt], sm = shat_mod(-1, qt);
      v.push_back(sm ? qt - sm : 0);
    }
  }
  t.rescale_qlinv = v.size();
  for (int l = 0; l < c->n_q; ++l)
    for (int i = 0; i < c->n_q; ++i) {
      u64 qi = c->mod[i];
      if (i < l) push_pair(v, host_invmod(c->mod[l] % qi, qi), qi);
      else { v.push_back(0); v.push_back(0); }
    }
  t.garner_inv = v.size();
  for (int i = 0; i < c->n_q; ++i)
    for (int j = 0; j < c->n_q; ++j) {
      u64 qi = c->mod[i];
      if (j < i) push_pair(v, host_invmod(c->mod[j] % qi, qi), qi);
      else { v.push_back(0); v.push_back(0); }
    }
  // mixed-radix digits of (Q_l - 1)/2 for each level l: Q_l odd.
  t.halfq_digits = v.size();
  for (int l = 0; l < c->n_q; ++l) {
    // compute (Q_l - 1)/2 as a little-endian multiword integer, then its
    // mixed-radix digits by repeated division by q_0, q_1, ...
    std::vector<u64> w(1, 1);
    for (int i = 0; i <= l; ++i) {  // w *= q_i
      u128 carry = 0;
      for (auto &x : w) {
        u128 p = (u128)x * c->mod[i] + carry;
        x = (u64)p;
        carry = p >> 64;
      }
      if (carry) w.push_back((u64)carry);
    }
    // w -= 1 (Q odd, so w >= 1 and no borrow past word 0 issue handled)
    for (auto &x : w) {
      if (x-- != 0) break;
    }
    // w >>= 1
    for (size_t k = 0; k < w.size(); ++k) {
      w[k] >>= 1;
      if (k + 1 < w.size()) w[k] |= (w[k + 1] & 1) << 63;
    }
    std::vector<u64> dig(c->n_q, 0);
    for (int i = 0; i <= l; ++i) {
      u128 rem = 0;
      for (int k = (int)w.size() - 1; k >= 0; --k) {
        u128 cur = (rem << 64) | w[k];
        w[k] = (u64)(cur / c->mod[i]);
        rem = cur % c->mod[i];
      }
      dig[i] = (u64)rem;
    }
    for (int i = 0; i < c->n_q; ++i) v.push_back(dig[i]);
  }
  t.total = v.size();

  // ---- upload ----
  size_t bytes_mods = sizeof(ModInfo) * nm, bytes_tw = sizeof(ulonglong2) * (size_t)nm * n;
  if (cudaMalloc(&c->d_mods, bytes_mods) != cudaSuccess) return CKKS_E_OOM;
  if (cudaMalloc(&c->d_tw_fwd, bytes_tw) != cudaSuccess) return CKKS_E_OOM;
  if (cudaMalloc(&c->d_tw_inv, bytes_tw) != cudaSuccess) return CKKS_E_OOM;
  if (cudaMalloc(&c->d_conv, sizeof(u64) * std::max<size_t>(1, t.total)) != cudaSuccess) return CKKS_E_OOM;
  CK_CUDA(cudaMemcpy(c->d_mods, mi.data(), bytes_mods, cudaMemcpyHostToDevice));
  CK_CUDA(cudaMemcpy(c->d_tw_fwd, fwd.data(), bytes_tw, cudaMemcpyHostToDevice));
  CK_CUDA(cudaMemcpy(c->d_tw_inv, inv.data(), bytes_tw, cudaMemcpyHostToDevice));
  const size_t bytes_row = sizeof(ulonglong2) * rfwd.size();
  if (cudaMalloc(&c->d_tw_row_fwd, bytes_row) != cudaSuccess) return CKKS_E_OOM;
  if (cudaMalloc(&c->d_tw_row_inv, bytes_row) != cudaSuccess) return CKKS_E_OOM;
  CK_CUDA(cudaMemcpy(c->d_tw_row_fwd, rfwd.data(), bytes_row, cudaMemcpyHostToDevice));
  CK_CUDA(cudaMemcpy(c->d_tw_row_inv, rinv.data(), bytes_row, cudaMemcpyHostToDevice));
  if (t.total) CK_CUDA(cudaMemcpy(c->d_conv, v.data(), sizeof(u64) * t.total, cudaMemcpyHostToDevice));
  c->table_bytes = bytes_mods + 2 * bytes_tw + 2 * bytes_row + sizeof(u64) * t.total;
  return CKKS_OK;
}
