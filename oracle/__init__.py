"""Plain CPU oracle for RNS-CKKS.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code, table or constant
with the CUDA library in ``paper_2506_19693_gb300``: the C core
(``ckks_oracle.c``) re-derives primes, roots, transforms, basis conversion,
key switching, rescale and automorphisms from their definitions, and this
module adds the FP64 canonical-embedding encode/decode and an exact big-integer
CRT written with Python integers.

Paper passages followed (ReBoot, arXiv 2506.19693):
  * Sec. 3 -- parameter set {N, q, Delta}; a multiplication costs one level,
    the top prime of the modulus chain being dropped (rescale);
  * Sec. 3 -- batching: N/2 complex slots through the complex canonical
    embedding phi : C^{N/2} -> Z[X]/(X^N + 1); secret-key encryption;
  * Sec. 3, Eq. add/sub/mult -- slot-wise +, -, x of ciphertexts and the
    plaintext variants; Rot(a, k) is a cyclic left shift by k slots with one
    key per k.
The scheme internals are textbook RNS-CKKS; every reading the paper leaves open
is named C1..C11 in the C file's header and in the design notes.

Parity: every function here is pinned by ``tests/test_oracle_*.py`` against
brute force on tiny rings, exact big-integer arithmetic, closed forms and
group laws.  Parity unpinned: nothing in this module.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_uint)


def build(force: bool = False) -> str:
    """Compile the C core with gcc into ``oracle/_build`` and return the path."""
    os.makedirs(_BUILD, exist_ok=True)
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    so = os.path.join(_BUILD, f"libckks_oracle_{tag}.so")
    if force or not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    V, P = ctypes.c_void_p, ctypes.c_int
    sig = {
        "oc_create": (V, [P, P, P, P, _up, _up, P, ctypes.c_double]),
        "oc_destroy": (None, [V]),
        "oc_n_digits": (P, [V]),
        "oc_alpha": (P, [V]),
        "oc_moduli": (None, [V, _u64p]),
        "oc_psis": (None, [V, _u64p]),
        "oc_gen_primes": (P, [P, _up, P, _u64p]),
        "oc_find_psi": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
        "oc_splitmix_draw": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
        "oc_ntt": (None, [V, _u64p, P, _ip]),
        "oc_intt": (None, [V, _u64p, P, _ip]),
        "oc_ntt_direct": (None, [V, P, _u64p, _u64p]),
        "oc_negacyclic_schoolbook": (None, [V, P, _u64p, _u64p, _u64p]),
        "oc_keygen": (P, [V, ctypes.c_uint64]),
        "oc_gen_galois_key": (P, [V, ctypes.c_uint64]),
        "oc_secret": (None, [V, _i64p]),
        "oc_key_data": (P, [V, ctypes.c_uint64, _u64p]),
        "oc_galois_elt": (ctypes.c_uint64, [V, ctypes.c_int64]),
        "oc_pt_from_signed": (None, [V, _i64p, P, _u64p]),
        "oc_encrypt": (P, [V, _u64p, P, ctypes.c_uint64, _u64p]),
        "oc_gen_public_key": (P, [V]),
        "oc_public_key": (P, [V, _u64p]),
        "oc_pk_mask": (None, [ctypes.c_uint64, ctypes.c_uint64, _i64p]),
        "oc_encrypt_pk": (P, [V, _u64p, P, ctypes.c_uint64, _u64p]),
        "oc_enc_error": (None, [V, ctypes.c_uint64, _i64p]),
        "oc_decrypt": (P, [V, _u64p, P, _u64p]),
        "oc_add": (None, [V, _u64p, _u64p, P, _u64p]),
        "oc_sub": (None, [V, _u64p, _u64p, P, _u64p]),
        "oc_mul_plain": (None, [V, _u64p, _u64p, P, _u64p]),
        "oc_add_plain": (None, [V, _u64p, _u64p, P, _u64p]),
        "oc_mul_int": (None, [V, _u64p, ctypes.c_int64, P, _u64p]),
        "oc_tensor": (None, [V, _u64p, _u64p, P, _u64p, _u64p, _u64p]),
        "oc_bconv": (None, [V, _u64p, P, _ip, _u64p, P, _ip]),
        "oc_keyswitch": (P, [V, _u64p, P, ctypes.c_uint64, _u64p, _u64p]),
        "oc_mul_relin": (P, [V, _u64p, _u64p, P, _u64p]),
        "oc_rescale": (P, [V, _u64p, P, _u64p]),
        "oc_moddown_rescale": (P, [V, _u64p, P, _u64p]),
        "oc_keyswitch_ext": (P, [V, _u64p, P, ctypes.c_uint64, _u64p]),
        "oc_rotate_hoisted_ext": (P, [V, _u64p, P, P, _u64p, _u64p]),
        "oc_moddown": (P, [V, _u64p, P, _u64p]),
        "oc_mul_elem": (None, [V, _u64p, _u64p, P, _ip, _u64p]),
        "oc_mul_scalars": (None, [V, _u64p, P, _ip, _u64p, _u64p]),
        "oc_mul_relin_rescale": (P, [V, _u64p, _u64p, P, _u64p]),
        "oc_automorph": (P, [V, _u64p, P, ctypes.c_uint64, _u64p]),
        "oc_automorph_coeff": (None, [V, _u64p, P, _ip, ctypes.c_uint64, _u64p]),
        "oc_rotate_hoisted": (P, [V, _u64p, P, P, _u64p, _u64p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def _pi64(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_i64p)


def _pint(seq) -> ctypes.Array:
    arr = (ctypes.c_int * max(1, len(seq)))(*seq)
    return arr


def gen_primes(bits, log_n: int = 16) -> list[int]:
    """C1 prime chain for a list of bit sizes (q's then p's): primes
    = 1 mod 2^max(17, log2(2N))."""
    lib = _load()
    b = (ctypes.c_uint * len(bits))(*bits)
    out = np.zeros(len(bits), dtype=np.uint64)
    if lib.oc_gen_primes(len(bits), b, max(17, log_n + 1), _p64(out)) != 0:
        raise ValueError("no prime chain for these bit sizes")
    return [int(x) for x in out]


def splitmix_draw(key: int, c: int) -> int:
    """Output number c+1 of SplitMix64 started at `key` (C4)."""
    return int(_load().oc_splitmix_draw(key, c))


@dataclass
class OCt:
    """An oracle ciphertext: data [2, level+1, N] uint64 residues (NTT domain)."""
    data: np.ndarray
    level: int
    scale: float


class Oracle:
    """One RNS-CKKS parameter set evaluated on the CPU (ReBoot Sec. 3)."""

    def __init__(self, log_n: int, q_bits, p_bits, dnum: int, h: int = 64, sigma: float = 3.2):
        self._lib = _load()
        qb = (ctypes.c_uint * len(q_bits))(*q_bits)
        pb = (ctypes.c_uint * len(p_bits))(*p_bits)
        ptr = self._lib.oc_create(log_n, len(q_bits), len(p_bits), dnum, qb, pb, h, sigma)
        if not ptr:
            raise ValueError("invalid oracle parameters")
        self._c = ctypes.c_void_p(ptr)
        self.log_n = log_n
        self.n = 1 << log_n
        self.n_q = len(q_bits)
        self.n_p = len(p_bits)
        self.dnum = dnum
        self.alpha = self._lib.oc_alpha(self._c)
        self.n_digits = self._lib.oc_n_digits(self._c)
        m = np.zeros(self.n_q + self.n_p, dtype=np.uint64)
        self._lib.oc_moduli(self._c, _p64(m))
        self.moduli = [int(x) for x in m]
        self.q = self.moduli[: self.n_q]
        self.p = self.moduli[self.n_q:]
        ps = np.zeros(self.n_q + self.n_p, dtype=np.uint64)
        self._lib.oc_psis(self._c, _p64(ps))
        self.psi = [int(x) for x in ps]
        self.h = h
        self.sigma = sigma

    def __del__(self):
        try:
            self._lib.oc_destroy(self._c)
        except Exception:
            pass

    # ---- transforms (C2) ----
    def ntt(self, a: np.ndarray, mods) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        self._lib.oc_ntt(self._c, _p64(a), len(mods), _pint(mods))
        return a

    def intt(self, a: np.ndarray, mods) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        self._lib.oc_intt(self._c, _p64(a), len(mods), _pint(mods))
        return a

    def ntt_direct(self, a: np.ndarray, mod_index: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.zeros(self.n, dtype=np.uint64)
        self._lib.oc_ntt_direct(self._c, mod_index, _p64(a), _p64(out))
        return out

    def negacyclic_schoolbook(self, a, b, mod_index: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros(self.n, dtype=np.uint64)
        self._lib.oc_negacyclic_schoolbook(self._c, mod_index, _p64(a), _p64(b), _p64(out))
        return out

    def bconv(self, x: np.ndarray, src, dst) -> np.ndarray:
        """Fast basis conversion (C8), uncentred, coefficient domain."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros((len(dst), self.n), dtype=np.uint64)
        self._lib.oc_bconv(self._c, _p64(x), len(src), _pint(src), _p64(out), len(dst), _pint(dst))
        return out

    # ---- keys (C4, C7) ----
    def keygen(self, seed: int) -> None:
        self._lib.oc_keygen(self._c, seed)

    def galois_elt(self, k: int) -> int:
        return int(self._lib.oc_galois_elt(self._c, k))

    def conj_elt(self) -> int:
        return 2 * self.n - 1

    def gen_galois_key(self, g: int) -> None:
        if self._lib.oc_gen_galois_key(self._c, g) != 0:
            raise ValueError("galois key generation failed")

    def gen_rotation_keys(self, steps) -> None:
        for k in steps:
            self.gen_galois_key(self.galois_elt(k))

    def secret(self) -> np.ndarray:
        s = np.zeros(self.n, dtype=np.int64)
        self._lib.oc_secret(self._c, _pi64(s))
        return s

    def key_data(self, galois: int) -> np.ndarray:
        ext = self.n_q + self.n_p
        out = np.zeros((self.n_digits, 2, ext, self.n), dtype=np.uint64)
        if self._lib.oc_key_data(self._c, galois, _p64(out)) != 0:
            raise KeyError(galois)
        return out

    # ---- encoding (Sec. 3 batching; reading C3) ----
    def slot_exponents(self) -> np.ndarray:
        """g_j = 5^j mod 2N for j < N/2: slot j is the value at zeta^{g_j}."""
        g = np.zeros(self.n // 2, dtype=np.int64)
        v = 1
        for j in range(self.n // 2):
            g[j] = v
            v = (v * 5) % (2 * self.n)
        return g

    def embed_inverse(self, z: np.ndarray) -> np.ndarray:
        """tau^{-1}: slots z (N/2 complex) -> real coefficients m with m(zeta^{g_j}) = z_j.

        m_k = (1/N) sum over odd e of w[e] zeta^{-e k}, where w[g_j] = z_j and
        w[2N - g_j] = conj(z_j): one length-2N FFT."""
        n = self.n
        z = np.asarray(z, dtype=np.complex128)
        zz = np.zeros(n // 2, dtype=np.complex128)
        zz[: len(z)] = z
        g = self.slot_exponents()
        w = np.zeros(2 * n, dtype=np.complex128)
        w[g] = zz
        w[2 * n - g] = np.conj(zz)
        return (np.fft.fft(w)[:n] / n).real

    def embed(self, m: np.ndarray) -> np.ndarray:
        """tau: real coefficients m -> slots z_j = m(zeta^{g_j})."""
        n = self.n
        x = np.zeros(2 * n, dtype=np.complex128)
        x[:n] = np.asarray(m, dtype=np.float64)
        vals = np.fft.ifft(x) * (2 * n)
        return vals[self.slot_exponents()]

    @staticmethod
    def round_half_away(x: np.ndarray) -> np.ndarray:
        t = np.trunc(x)
        frac = np.abs(x - t)
        return (t + np.sign(x) * (frac >= 0.5)).astype(np.int64)

    def encode(self, z, scale: float) -> np.ndarray:
        """Integer plaintext coefficients round(Delta * tau^{-1}(z)) (C3)."""
        v = self.embed_inverse(z) * scale
        if np.max(np.abs(v)) >= 2.0 ** 62:
            raise OverflowError("scaled plaintext exceeds 2^62")
        return self.round_half_away(v)

    def decode_coeffs(self, m, scale: float) -> np.ndarray:
        """Slots from real (or big-integer) coefficients, divided by the scale."""
        mf = np.array([float(v) for v in m], dtype=np.float64) if not isinstance(m, np.ndarray) else m.astype(np.float64)
        return self.embed(mf) / scale

    # ---- plaintexts ----
    def pt_from_int(self, m: np.ndarray, level: int) -> np.ndarray:
        m = np.ascontiguousarray(m, dtype=np.int64)
        pt = np.zeros((level + 1, self.n), dtype=np.uint64)
        self._lib.oc_pt_from_signed(self._c, _pi64(m), level, _p64(pt))
        return pt

    def crt_centred(self, residues: np.ndarray, level: int) -> list[int]:
        """Exact centred CRT of coefficient-domain residues over q_0..q_level."""
        qs = self.q[: level + 1]
        Q = 1
        for q in qs:
            Q *= q
        coef = []
        for q in qs:
            Mi = Q // q
            coef.append(Mi * pow(Mi % q, -1, q))
        rows = [residues[i].tolist() for i in range(level + 1)]
        out = []
        half = Q // 2
        for k in range(self.n):
            x = 0
            for i in range(level + 1):
                x += rows[i][k] * coef[i]
            x %= Q
            if x > half:
                x -= Q
            out.append(x)
        return out

    # ---- encryption (C5) ----
    def encrypt(self, pt: np.ndarray, level: int, scale: float, enc_seed: int) -> OCt:
        pt = np.ascontiguousarray(pt[: level + 1], dtype=np.uint64)
        ct = np.zeros((2, level + 1, self.n), dtype=np.uint64)
        if self._lib.oc_encrypt(self._c, _p64(pt), level, enc_seed, _p64(ct)) != 0:
            raise RuntimeError("encrypt failed (keygen first?)")
        return OCt(ct, level, scale)

    def gen_public_key(self) -> None:
        """pk = ([-a s + e]_Q, a) at the top level (C5, pk form); keygen first."""
        if self._lib.oc_gen_public_key(self._c) != 0:
            raise RuntimeError("public key generation failed (keygen first?)")

    def public_key(self) -> np.ndarray:
        out = np.zeros((2, self.n_q, self.n), dtype=np.uint64)
        if self._lib.oc_public_key(self._c, _p64(out)) != 0:
            raise RuntimeError("no public key")
        return out

    def pk_mask(self, enc_seed: int) -> np.ndarray:
        v = np.zeros(self.n, dtype=np.int64)
        self._lib.oc_pk_mask(enc_seed, self.n, _pi64(v))
        return v

    def encrypt_pk(self, pt: np.ndarray, level: int, scale: float, enc_seed: int) -> OCt:
        """ct = ([v b + m + e0]_Q, [v a + e1]_Q) with the public key (b, a)."""
        pt = np.ascontiguousarray(pt[: level + 1], dtype=np.uint64)
        ct = np.zeros((2, level + 1, self.n), dtype=np.uint64)
        if self._lib.oc_encrypt_pk(self._c, _p64(pt), level, enc_seed, _p64(ct)) != 0:
            raise RuntimeError("public-key encryption failed (gen_public_key first?)")
        return OCt(ct, level, scale)

    def enc_error(self, enc_seed: int) -> np.ndarray:
        e = np.zeros(self.n, dtype=np.int64)
        self._lib.oc_enc_error(self._c, enc_seed, _pi64(e))
        return e

    def decrypt(self, ct: OCt) -> np.ndarray:
        pt = np.zeros((ct.level + 1, self.n), dtype=np.uint64)
        self._lib.oc_decrypt(self._c, _p64(np.ascontiguousarray(ct.data)), ct.level, _p64(pt))
        return pt

    def decrypt_coeffs(self, ct: OCt) -> list[int]:
        """Centred integer coefficients of c0 + c1 s."""
        pt = self.decrypt(ct)
        return self.crt_centred(self.intt(pt, list(range(ct.level + 1))), ct.level)

    def decrypt_decode(self, ct: OCt) -> np.ndarray:
        return self.decode_coeffs(self.decrypt_coeffs(ct), ct.scale)

    # ---- homomorphic operations ----
    def _new(self, level: int) -> np.ndarray:
        return np.zeros((2, level + 1, self.n), dtype=np.uint64)

    def add(self, a: OCt, b: OCt) -> OCt:
        out = self._new(a.level)
        self._lib.oc_add(self._c, _p64(a.data), _p64(b.data), a.level, _p64(out))
        return OCt(out, a.level, a.scale)

    def sub(self, a: OCt, b: OCt) -> OCt:
        out = self._new(a.level)
        self._lib.oc_sub(self._c, _p64(a.data), _p64(b.data), a.level, _p64(out))
        return OCt(out, a.level, a.scale)

    def mul_plain(self, a: OCt, pt: np.ndarray, pt_scale: float) -> OCt:
        out = self._new(a.level)
        pt = np.ascontiguousarray(pt[: a.level + 1], dtype=np.uint64)
        self._lib.oc_mul_plain(self._c, _p64(a.data), _p64(pt), a.level, _p64(out))
        return OCt(out, a.level, a.scale * pt_scale)

    def add_plain(self, a: OCt, pt: np.ndarray) -> OCt:
        out = self._new(a.level)
        pt = np.ascontiguousarray(pt[: a.level + 1], dtype=np.uint64)
        self._lib.oc_add_plain(self._c, _p64(a.data), _p64(pt), a.level, _p64(out))
        return OCt(out, a.level, a.scale)

    def mul_int(self, a: OCt, k: int) -> OCt:
        out = self._new(a.level)
        self._lib.oc_mul_int(self._c, _p64(a.data), k, a.level, _p64(out))
        return OCt(out, a.level, a.scale)

    def tensor(self, a: OCt, b: OCt):
        nl = a.level + 1
        d = np.zeros((3, nl, self.n), dtype=np.uint64)
        self._lib.oc_tensor(self._c, _p64(a.data), _p64(b.data), a.level,
                            _p64(d[0]), _p64(d[1]), _p64(d[2]))
        return d

    def keyswitch(self, d: np.ndarray, level: int, galois: int):
        d = np.ascontiguousarray(d, dtype=np.uint64)
        o0 = np.zeros((level + 1, self.n), dtype=np.uint64)
        o1 = np.zeros((level + 1, self.n), dtype=np.uint64)
        if self._lib.oc_keyswitch(self._c, _p64(d), level, galois, _p64(o0), _p64(o1)) != 0:
            raise KeyError(galois)
        return o0, o1

    def mul_relin(self, a: OCt, b: OCt) -> OCt:
        if a.level != b.level:
            raise ValueError("level mismatch")
        out = self._new(a.level)
        if self._lib.oc_mul_relin(self._c, _p64(a.data), _p64(b.data), a.level, _p64(out)) != 0:
            raise KeyError("relinearisation key")
        return OCt(out, a.level, a.scale * b.scale)

    def rescale(self, a: OCt) -> OCt:
        out = self._new(a.level - 1)
        if self._lib.oc_rescale(self._c, _p64(a.data), a.level, _p64(out)) != 0:
            raise ValueError("cannot rescale level 0")
        return OCt(out, a.level - 1, a.scale / self.q[a.level])

    def keyswitch_ext(self, d: np.ndarray, level: int, galois: int) -> np.ndarray:
        """Key switch of d (NTT domain, level+1 limbs) stopped before ModDown:
        [2][level+1+K][N] over q_0..q_level, P."""
        d = np.ascontiguousarray(d, dtype=np.uint64)
        acc = np.zeros((2, level + 1 + self.n_p, self.n), dtype=np.uint64)
        if self._lib.oc_keyswitch_ext(self._c, _p64(d), level, galois, _p64(acc)) != 0:
            raise KeyError(galois)
        return acc

    def ext_mods(self, level: int) -> list:
        """Modulus indices of the extended basis q_0..q_level, p_0..p_{K-1}."""
        return list(range(level + 1)) + [self.n_q + k for k in range(self.n_p)]

    def rotate_hoisted_ext(self, a: OCt, steps) -> list:
        """Hoisted rotations stopped before ModDown: per step [2][level+1+K][N]
        = (P sigma(c0) + acc0, acc1) over q_0..q_level, P."""
        gs = np.array([self.galois_elt(k) for k in steps], dtype=np.uint64)
        ext = a.level + 1 + self.n_p
        outs = np.zeros((len(steps), 2, ext, self.n), dtype=np.uint64)
        if self._lib.oc_rotate_hoisted_ext(self._c, _p64(np.ascontiguousarray(a.data)), a.level, len(steps),
                                           _p64(gs), _p64(outs)) != 0:
            raise KeyError("galois key")
        return [np.ascontiguousarray(outs[i]) for i in range(len(steps))]

    def moddown(self, x: np.ndarray, level: int) -> np.ndarray:
        """C9 on one polynomial over q_0..q_level, P: returns [level+1][N]."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros((level + 1, self.n), dtype=np.uint64)
        self._lib.oc_moddown(self._c, _p64(x), level, _p64(out))
        return out

    def mul_elem(self, x: np.ndarray, y: np.ndarray, mods) -> np.ndarray:
        """x * y limb by limb mod the listed moduli."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        y = np.ascontiguousarray(y, dtype=np.uint64)
        out = np.zeros_like(x)
        self._lib.oc_mul_elem(self._c, _p64(x), _p64(y), len(mods), _pint(list(mods)), _p64(out))
        return out

    def pt_ext_from_int(self, m: np.ndarray, level: int) -> np.ndarray:
        """Integer coefficients as an NTT-domain plaintext over q_0..q_level, P."""
        q_part = self.pt_from_int(m, level)
        m = np.asarray(m, dtype=np.int64)
        p_res = np.stack([np.mod(m, np.int64(self.moduli[self.n_q + k])).astype(np.uint64)
                          for k in range(self.n_p)])
        p_part = self.ntt(p_res, [self.n_q + k for k in range(self.n_p)])
        return np.concatenate([q_part, p_part])

    def mul_scalars(self, x: np.ndarray, mods, w) -> np.ndarray:
        """x[t] * w[t] mod the t-th modulus (one scalar per limb)."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        ww = np.ascontiguousarray(np.array([int(v) for v in w], dtype=np.uint64))
        out = np.zeros_like(x)
        self._lib.oc_mul_scalars(self._c, _p64(x), len(mods), _pint(list(mods)), _p64(ww), _p64(out))
        return out

    def moddown_rescale(self, x: np.ndarray, level: int) -> np.ndarray:
        """Reading C21 on one polynomial: x [level+1+K][N] over q_0..q_l, P
        (NTT domain) divided by P q_l; returns [level][N] (NTT domain)."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros((level, self.n), dtype=np.uint64)
        if self._lib.oc_moddown_rescale(self._c, _p64(x), level, _p64(out)) != 0:
            raise ValueError("cannot rescale level 0")
        return out

    def mul_relin_rescale(self, a: OCt, b: OCt) -> OCt:
        """Relinearised product with ModDown and rescale merged (reading C21)."""
        if a.level != b.level:
            raise ValueError("level mismatch")
        out = self._new(a.level - 1)
        if self._lib.oc_mul_relin_rescale(self._c, _p64(a.data), _p64(b.data), a.level, _p64(out)) != 0:
            raise KeyError("relinearisation key or level 0")
        return OCt(out, a.level - 1, a.scale * b.scale / self.q[a.level])

    def automorph(self, a: OCt, g: int) -> OCt:
        out = self._new(a.level)
        if self._lib.oc_automorph(self._c, _p64(a.data), a.level, g, _p64(out)) != 0:
            raise KeyError(g)
        return OCt(out, a.level, a.scale)

    def rotate(self, a: OCt, k: int) -> OCt:
        return self.automorph(a, self.galois_elt(k))

    def rotate_hoisted(self, a: OCt, steps) -> list:
        """Rotations of one ciphertext by every k in steps sharing one ModUp."""
        gs = np.array([self.galois_elt(k) for k in steps], dtype=np.uint64)
        outs = np.zeros((len(steps), 2, a.level + 1, self.n), dtype=np.uint64)
        if self._lib.oc_rotate_hoisted(self._c, _p64(np.ascontiguousarray(a.data)), a.level, len(steps),
                                       _p64(gs), _p64(outs)) != 0:
            raise KeyError("galois key")
        return [OCt(np.ascontiguousarray(outs[i]), a.level, a.scale) for i in range(len(steps))]

    def conjugate(self, a: OCt) -> OCt:
        return self.automorph(a, self.conj_elt())

    def automorph_coeff(self, x: np.ndarray, mods, g: int) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros_like(x)
        self._lib.oc_automorph_coeff(self._c, _p64(x), len(mods), _pint(mods), g, _p64(out))
        return out
