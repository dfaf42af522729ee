"""Python binding of the GB300 RNS-CKKS library (``include/ckks.h``).

Argument marshalling only: every step of every operation runs in the CUDA
library ``_build/libckks.so``.  PyTorch provides device memory (ciphertexts
and plaintexts are torch tensors on the GPU) and the stream the library
enqueues on.  Importing this package without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

CKKS_OK = 0
STATUS = {0: "CKKS_OK", -1: "CKKS_E_PARAM", -2: "CKKS_E_LEVEL", -3: "CKKS_E_SCALE", -4: "CKKS_E_NOKEY",
          -5: "CKKS_E_OOM", -6: "CKKS_E_CUDA", -7: "CKKS_E_TIMEOUT", -8: "CKKS_E_STATE"}


class CkksError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class CkksParams(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_q", ctypes.c_uint32), ("n_p", ctypes.c_uint32),
                ("dnum", ctypes.c_uint32), ("h", ctypes.c_uint32),
                ("q_bits", ctypes.c_uint32 * 60), ("p_bits", ctypes.c_uint32 * 16),
                ("log2_scale", ctypes.c_double), ("sigma", ctypes.c_double), ("seed", ctypes.c_uint64)]


class CkksCt(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("log_n", ctypes.c_uint32), ("level", ctypes.c_uint32),
                ("n_limbs", ctypes.c_uint32), ("is_ntt", ctypes.c_uint32), ("scale", ctypes.c_double)]


OP_MUL_RELIN, OP_ROTATE, OP_RESCALE = 1, 2, 3
RESCALE_NONE, RESCALE_SEPARATE, RESCALE_MERGED = 0, 1, 2  # ckks_mul_relin_batch / Op.rescale


class CkksOpDesc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("ctx", ctypes.c_void_p), ("a", ctypes.POINTER(CkksCt)),
                ("b", ctypes.POINTER(CkksCt)), ("out", ctypes.POINTER(CkksCt)), ("k", ctypes.c_int32),
                ("rescale", ctypes.c_int)]


# C-ABI symbols and signatures, in header order.
_V, _I, _U64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
_CTP = ctypes.POINTER(CkksCt)
SIGNATURES = {
    "ckks_ctx_create": (_I, [ctypes.POINTER(CkksParams), _V, ctypes.POINTER(_V)]),
    "ckks_ctx_destroy": (_I, [_V]),
    "ckks_ctx_set_stream": (_I, [_V, _V]),
    "ckks_ctx_moduli": (_I, [_V, _V, _I]),
    "ckks_ctx_roots": (_I, [_V, _V, _I]),
    "ckks_ctx_digits": (_I, [_V, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ckks_ctx_device_bytes": (_I, [_V, ctypes.POINTER(_U64)]),
    "ckks_ctx_profile": (_I, [_V, _I]),
    "ckks_ctx_profile_read": (_I, [_V, _V, _V, _V, _I]),
    "ckks_profile_kinds": (_I, []),
    "ckks_profile_kind_name": (ctypes.c_char_p, [_I]),
    "ckks_ctx_launch_count": (_I, [_V, ctypes.POINTER(_U64)]),
    "ckks_alu_peaks": (_I, [_V, ctypes.POINTER(_D), _I]),
    "ckks_ctx_set_form": (_I, [_V, _I]),
    "ckks_ctx_device_error": (_I, [_V]),
    "ckks_ctx_ks_histogram": (_I, [_V, _V, _I]),
    "ckks_debug_tc_expire": (_I, [_V, _U64]),
    "ckks_keygen_from_seed": (_I, [_V, _U64, _V, _I, _I, _I]),
    "ckks_keygen_galois": (_I, [_V, _U64]),
    "ckks_galois_elt": (_U64, [_V, ctypes.c_int32]),
    "ckks_debug_secret": (_I, [_V, _V]),
    "ckks_debug_key": (_I, [_V, _U64, _V]),
    "ckks_encode": (_I, [_V, _V, _V, _I, ctypes.c_uint32, _D, _V]),
    "ckks_decode": (_I, [_V, _V, ctypes.c_uint32, _D, _V, _V, _I]),
    "ckks_pt_from_int": (_I, [_V, _V, ctypes.c_uint32, _V]),
    "ckks_ntt": (_I, [_V, _V, ctypes.c_uint32, ctypes.c_uint32, _I]),
    "ckks_encrypt": (_I, [_V, _V, ctypes.c_uint32, _D, _U64, _CTP]),
    "ckks_decrypt": (_I, [_V, _CTP, _V]),
    "ckks_keygen_public": (_I, [_V]),
    "ckks_ks_inner_tc": (_I, [_V, _V, _V, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _V]),
    "ckks_ks_inner_u64": (_I, [_V, _V, _V, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _V]),
    "ckks_public_key_export": (_I, [_V, _V]),
    "ckks_encrypt_pk": (_I, [_V, _V, ctypes.c_uint32, _D, _U64, _CTP]),
    "ckks_add": (_I, [_V, _CTP, _CTP, _CTP]),
    "ckks_sub": (_I, [_V, _CTP, _CTP, _CTP]),
    "ckks_mul_plain": (_I, [_V, _CTP, _V, _D, _CTP]),
    "ckks_add_plain": (_I, [_V, _CTP, _V, _CTP]),
    "ckks_mul_int": (_I, [_V, _CTP, ctypes.c_int64, _CTP]),
    "ckks_mul_relin": (_I, [_V, _CTP, _CTP, _CTP]),
    "ckks_rescale": (_I, [_V, _CTP]),
    "ckks_rescale_noalloc": (_I, [_V, _CTP]),
    "ckks_rotate": (_I, [_V, _CTP, ctypes.c_int32, _CTP]),
    "ckks_conjugate": (_I, [_V, _CTP, _CTP]),
    "ckks_automorph": (_I, [_V, _CTP, _U64, _CTP]),
    "ckks_mul_relin_batch": (_I, [_V, _CTP, _CTP, _CTP, _I, _I]),
    "ckks_rotate_batch": (_I, [_V, _CTP, _V, _CTP, _I]),
    "ckks_rescale_batch": (_I, [_V, _CTP, _I]),
    "ckks_mul_relin_host": (_I, [_V, _V, _V, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, _I, _I, _I, _V,
                                 ctypes.POINTER(ctypes.c_double)]),
    "ckks_rotate_hoisted": (_I, [_V, _CTP, _I, _V, _I, _CTP]),
    "ckks_add_batch": (_I, [_V, _CTP, _CTP, _CTP, _I, _I]),
    "ckks_mul_int_batch": (_I, [_V, _CTP, ctypes.c_int64, _CTP, _I]),
    "ckks_mul_plain_batch": (_I, [_V, _CTP, _V, _D, _CTP, _I]),
    "ckks_add_plain_batch": (_I, [_V, _CTP, _V, _CTP, _I]),
    "ckks_boot_setup": (_I, [_V]),
    "ckks_boot_rotation_steps": (_I, [_V, _V, _I]),
    "ckks_boot_constant_count": (_I, [_V]),
    "ckks_boot_import": (_I, [_V, _V, _I, _V, _I]),
    "ckks_boot_export": (_I, [_V, _V, _I, _V, _I]),
    "ckks_bootstrap": (_I, [_V, _CTP, _CTP]),
    "ckks_bootstrap_batch": (_I, [_V, _CTP, _CTP, _I]),
    "ckks_boot_linear": (_I, [_V, _I, _CTP, _CTP, _I]),
    "ckks_boot_set_slots": (_I, [_V, ctypes.c_uint32]),
    "ckks_set_key_compression": (_I, [_V, _I]),
    "ckks_bootstrap_iterative_batch": (_I, [_V, _CTP, _CTP, _I, _I]),
    "ckks_exec": (_I, [_V, _I]),
    "ckks_exec_capture": (_I, [_V, _I, _V, ctypes.POINTER(_V)]),
    "ckks_graph_launch": (_I, [_V, _V]),
    "ckks_graph_destroy": (_I, [_V]),
    "ckks_tune": (_I, [_V, _I, _I, ctypes.POINTER(_I)]),
    "ckks_tune_ntt": (_I, [_V, _I, ctypes.POINTER(ctypes.c_int)]),
    "ckks_ctx_set_ntt_rows": (_I, [_V, _I]),
    "ckks_ctx_set_ntt_cluster": (_I, [_V, _I, ctypes.POINTER(ctypes.c_int)]),
    "ckks_ctx_ntt_config": (_I, [_V, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "ckks_ctx_set_fused_finish": (_I, [_V, _I]),
    "ckks_ctx_set_finish_rows": (_I, [_V, _I]),
    "ckks_ctx_finish_rows": (_I, [_V, ctypes.POINTER(ctypes.c_int)]),
    "ckks_tune_dnum": (_I, [_V, _V, ctypes.POINTER(ctypes.c_uint32), _I, _I, ctypes.c_uint64,
                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double)]),
    "ckks_ntt_tc": (_I, [_V, _V, ctypes.c_uint32, ctypes.c_uint32]),
    "ckks_ct_alloc": (_I, [_V, ctypes.c_uint32, _CTP]),
    "ckks_ct_free": (_I, [_V, _CTP]),
    "ckks_ct_export": (_I, [_V, _CTP, _V]),
    "ckks_ct_import": (_I, [_V, _V, _CTP]),
    "ckks_ct_export_ntt": (_I, [_V, _CTP, _V]),
    "ckks_ct_import_ntt": (_I, [_V, _V, _CTP]),
    "ckks_wire_bytes": (_I, [_V, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]),
    "ckks_ct_export_packed": (_I, [_V, _CTP, _V]),
    "ckks_ct_import_packed": (_I, [_V, _V, _CTP]),
    "ckks_mul_relin_host_packed": (_I, [_V, _V, _V, ctypes.c_double, ctypes.c_double, ctypes.c_uint32, _I, _I, _I,
                                        _V, ctypes.POINTER(ctypes.c_double)]),
    "ckks_status_str": (ctypes.c_char_p, [_I]),
}

_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libckks.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.lib_path()
    if not os.path.exists(path):
        path = _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str) -> None:
    if rc != CKKS_OK:
        raise CkksError(rc, what)


def _torch():
    import torch
    return torch


@dataclass
class Ciphertext:
    """A ciphertext in HBM: ``data`` is an int64 torch tensor of shape
    [2, n_limbs, N] (bit pattern of uint64 residues, NTT domain)."""
    data: "object"
    level: int
    scale: float

    @property
    def n_limbs(self) -> int:
        return int(self.data.shape[1])

    def handle(self, log_n: int) -> CkksCt:
        return CkksCt(self.data.data_ptr(), log_n, self.level, self.n_limbs, 1, self.scale)


class Context:
    """One parameter set on the current CUDA device and stream."""

    def __init__(self, log_n: int, q_bits, p_bits, dnum: int, h: int = 64, sigma: float = 3.2,
                 log2_scale: float = 40.0, stream=None):
        torch = _torch()
        self.lib = load_library()
        p = CkksParams()
        p.log_n, p.n_q, p.n_p, p.dnum, p.h = log_n, len(q_bits), len(p_bits), dnum, h
        for i, b in enumerate(q_bits):
            p.q_bits[i] = b
        for i, b in enumerate(p_bits):
            p.p_bits[i] = b
        p.log2_scale, p.sigma = log2_scale, sigma
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.device("cuda", torch.cuda.current_device())
        h_ = ctypes.c_void_p()
        _check(self.lib.ckks_ctx_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h_)), "ckks_ctx_create")
        self._h = h_
        self.log_n, self.n = log_n, 1 << log_n
        self.n_q, self.n_p, self.dnum = len(q_bits), len(p_bits), dnum
        buf = (ctypes.c_uint64 * (self.n_q + self.n_p))()
        self.lib.ckks_ctx_moduli(self._h, buf, self.n_q + self.n_p)
        self.moduli = [int(x) for x in buf]
        self.q = self.moduli[: self.n_q]
        self.p = self.moduli[self.n_q:]
        self.lib.ckks_ctx_roots(self._h, buf, self.n_q + self.n_p)
        self.psi = [int(x) for x in buf]
        nd, al = ctypes.c_int(), ctypes.c_int()
        self.lib.ckks_ctx_digits(self._h, ctypes.byref(nd), ctypes.byref(al))
        self.n_digits, self.alpha = nd.value, al.value
        self.default_scale = 2.0 ** log2_scale

    @classmethod
    def from_workload(cls, w, stream=None) -> "Context":
        return cls(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma, w.log2_scale, stream)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self.lib.ckks_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- memory ----
    def new_ct(self, n_limbs: int, level: int | None = None, scale: float = 1.0) -> Ciphertext:
        torch = _torch()
        t = torch.empty((2, n_limbs, self.n), dtype=torch.int64, device=self.device)
        return Ciphertext(t, n_limbs - 1 if level is None else level, scale)

    def new_pt(self, level: int):
        torch = _torch()
        return torch.empty((level + 1, self.n), dtype=torch.int64, device=self.device)

    def device_bytes(self) -> int:
        b = ctypes.c_uint64()
        _check(self.lib.ckks_ctx_device_bytes(self._h, ctypes.byref(b)), "ckks_ctx_device_bytes")
        return b.value

    # ---- launch accounting ----
    def profile(self, enable: bool) -> None:
        _check(self.lib.ckks_ctx_profile(self._h, int(enable)), "ckks_ctx_profile")

    def profile_read(self) -> dict:
        """{kernel class: (device ms, launches, limbs)} since the last read."""
        k = self.lib.ckks_profile_kinds()
        ms = np.zeros(k)
        la = np.zeros(k, dtype=np.uint64)
        li = np.zeros(k, dtype=np.uint64)
        self.lib.ckks_ctx_profile_read(self._h, ms.ctypes.data, la.ctypes.data, li.ctypes.data, k)
        return {self.lib.ckks_profile_kind_name(i).decode(): (float(ms[i]), int(la[i]), int(li[i]))
                for i in range(k)}

    def ks_histogram(self) -> list:
        """Key switches per level since the last profile read (index = level)."""
        out = np.zeros(64, dtype=np.uint64)
        self.lib.ckks_ctx_ks_histogram(self._h, out.ctypes.data, 64)
        return [int(v) for v in out]

    def alu_peaks(self) -> dict:
        """Integer-pipe roofs of the production sequences measured on this GPU:
        {"mac_per_s", "bfly_fwd_loose_per_s", "bfly_fwd_strict_per_s", "bfly_inv_approx_per_s",
        "bfly_inv_exact_per_s"}."""
        out = (ctypes.c_double * 5)()
        rc = self.lib.ckks_alu_peaks(self._h, out, 5)
        if rc < 0:
            raise CkksError(rc, "ckks_alu_peaks")
        return dict(zip(("mac_per_s", "bfly_fwd_loose_per_s", "bfly_fwd_strict_per_s", "bfly_inv_approx_per_s",
                         "bfly_inv_exact_per_s"), (float(v) for v in out)))

    def set_form(self, form) -> None:
        """Basis-conversion form: "uint64" (or False), "tensor" (or True) or
        "fused" (the conversion fused with the transforms' column passes)."""
        code = {False: 0, True: 1, "uint64": 0, "tensor": 1, "fused": 2}[form]
        _check(self.lib.ckks_ctx_set_form(self._h, code), "ckks_ctx_set_form")

    def device_error(self) -> int:
        return self.lib.ckks_ctx_device_error(self._h)

    def debug_tc_expire(self, wait_ns: int = 1_000_000) -> None:
        """TEST ONLY: make the tensor-core kernel's bounded wait run out once."""
        _check(self.lib.ckks_debug_tc_expire(self._h, wait_ns), "ckks_debug_tc_expire")

    def set_ntt_rows(self, rows: int) -> None:
        _check(self.lib.ckks_ctx_set_ntt_rows(self._h, rows), "ckks_ctx_set_ntt_rows")

    def set_ntt_cluster(self, on: bool) -> int:
        """One-pass forward NTT on 8-CTA clusters (N = 2^16); returns the number
        of clusters the device holds at once (0 when switched off)."""
        m = ctypes.c_int(0)
        _check(self.lib.ckks_ctx_set_ntt_cluster(self._h, 1 if on else 0, ctypes.byref(m)),
               "ckks_ctx_set_ntt_cluster")
        return m.value

    def set_fused_finish(self, on: bool) -> None:
        """Key-switch finish in the forward NTT's row pass (on, the default) or
        in a separate element-wise kernel after it (off); same residues."""
        _check(self.lib.ckks_ctx_set_fused_finish(self._h, 1 if on else 0), "ckks_ctx_set_fused_finish")

    def set_finish_rows(self, rows: int) -> None:
        """Row tile of the row pass carrying the key-switch finish: 16, 8, or 0
        (follow the NTT row tile)."""
        _check(self.lib.ckks_ctx_set_finish_rows(self._h, rows), "ckks_ctx_set_finish_rows")

    def finish_rows(self) -> int:
        """The row tile in force for the row pass carrying the finish."""
        r = ctypes.c_int(0)
        _check(self.lib.ckks_ctx_finish_rows(self._h, ctypes.byref(r)), "ckks_ctx_finish_rows")
        return r.value

    def ntt_config(self) -> dict:
        """The NTT launch choices in force: {"rows": 16 or 8, "cluster": bool}."""
        r, cl = ctypes.c_int(0), ctypes.c_int(0)
        _check(self.lib.ckks_ctx_ntt_config(self._h, ctypes.byref(r), ctypes.byref(cl)), "ckks_ctx_ntt_config")
        return {"rows": r.value, "cluster": bool(cl.value)}

    def tune_ntt(self, n_polys: int = 16) -> int:
        """Autotune the NTT row pass (rows per CTA); returns the choice."""
        r = ctypes.c_int()
        _check(self.lib.ckks_tune_ntt(self._h, n_polys, ctypes.byref(r)), "ckks_tune_ntt")
        return r.value

    def tune(self, level: int, batch: int) -> int:
        """Autotune the key inner product for batches of this shape; returns the choice."""
        ch = ctypes.c_int()
        _check(self.lib.ckks_tune(self._h, level, batch, ctypes.byref(ch)), "ckks_tune")
        return ch.value

    def launch_count(self) -> int:
        c = ctypes.c_uint64()
        _check(self.lib.ckks_ctx_launch_count(self._h, ctypes.byref(c)), "ckks_ctx_launch_count")
        return c.value

    # ---- keys ----
    def keygen(self, seed: int, rot_steps=(), conj: bool = False) -> None:
        arr = (ctypes.c_int32 * max(1, len(rot_steps)))(*rot_steps)
        _check(self.lib.ckks_keygen_from_seed(self._h, seed, arr, len(rot_steps), int(conj), 0),
               "ckks_keygen_from_seed")

    def keygen_galois(self, g: int) -> None:
        _check(self.lib.ckks_keygen_galois(self._h, g), "ckks_keygen_galois")

    def galois_elt(self, k: int) -> int:
        return int(self.lib.ckks_galois_elt(self._h, k))

    def debug_secret(self) -> np.ndarray:
        s = np.zeros(self.n, dtype=np.int8)
        _check(self.lib.ckks_debug_secret(self._h, s.ctypes.data), "ckks_debug_secret")
        return s

    def debug_key(self, g: int) -> np.ndarray:
        out = np.zeros((self.n_digits, 2, self.n_q + self.n_p, self.n), dtype=np.uint64)
        _check(self.lib.ckks_debug_key(self._h, g, out.ctypes.data), "ckks_debug_key")
        return out

    # ---- plaintexts ----
    def encode(self, z, level: int, scale: float | None = None):
        z = np.asarray(z, dtype=np.complex128)
        re = np.ascontiguousarray(z.real)
        im = np.ascontiguousarray(z.imag)
        pt = self.new_pt(level)
        _check(self.lib.ckks_encode(self._h, re.ctypes.data, im.ctypes.data, len(z), level,
                                    scale or self.default_scale, pt.data_ptr()), "ckks_encode")
        return pt

    def decode(self, pt, level: int, scale: float, n_slots: int | None = None) -> np.ndarray:
        n_slots = n_slots or self.n // 2
        re = np.zeros(n_slots)
        im = np.zeros(n_slots)
        _check(self.lib.ckks_decode(self._h, pt.data_ptr(), level, scale, re.ctypes.data, im.ctypes.data,
                                    n_slots), "ckks_decode")
        return re + 1j * im

    def pt_from_int(self, m: np.ndarray, level: int):
        m = np.ascontiguousarray(m, dtype=np.int64)
        pt = self.new_pt(level)
        _check(self.lib.ckks_pt_from_int(self._h, m.ctypes.data, level, pt.data_ptr()), "ckks_pt_from_int")
        return pt

    def ntt(self, data, first_mod: int, inverse: bool = False) -> None:
        """In-place transform of a [limbs, N] int64 device tensor."""
        _check(self.lib.ckks_ntt(self._h, data.data_ptr(), int(data.shape[0]), first_mod, int(inverse)),
               "ckks_ntt")

    # ---- encryption ----
    def ntt_tc(self, data, n_polys: int, n_limbs: int) -> None:
        """Forward NTT with the first four stages on the tensor cores (ckks_ntt_tc):
        data is a device tensor of n_polys x n_limbs limbs, limb t under modulus t."""
        _check(self.lib.ckks_ntt_tc(self._h, data.data_ptr(), n_polys, n_limbs), "ckks_ntt_tc")

    def encrypt(self, pt, level: int, scale: float, enc_seed: int, n_limbs: int | None = None) -> Ciphertext:
        ct = self.new_ct(n_limbs or level + 1, level, scale)
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_encrypt(self._h, pt.data_ptr(), level, scale, enc_seed, ctypes.byref(h)),
               "ckks_encrypt")
        return ct

    def ks_inner(self, d, key, out, form: str = "tensor") -> None:
        """out[p][o][t] = sum_j d[p][j][t] key[j][o][t] mod q_t on device tensors
        d [P][D][L][N], key [D][2][L][N], out [P][2][L][N]; form "tensor"
        (tcgen05, P = 128) or "uint64"."""
        fn = {"tensor": self.lib.ckks_ks_inner_tc, "uint64": self.lib.ckks_ks_inner_u64}[form]
        P, D, L = int(d.shape[0]), int(d.shape[1]), int(d.shape[2])
        _check(fn(self._h, d.data_ptr(), key.data_ptr(), P, D, L, out.data_ptr()), "ckks_ks_inner")

    def keygen_public(self) -> None:
        """The public key pk = ([-a s + e]_Q, a) at the top level (after keygen)."""
        _check(self.lib.ckks_keygen_public(self._h), "ckks_keygen_public")

    def public_key(self) -> np.ndarray:
        """The public key as host uint64[2][n_q][N] (b, then a), NTT domain."""
        out = np.zeros((2, self.n_q, self.n), dtype=np.uint64)
        _check(self.lib.ckks_public_key_export(self._h, out.ctypes.data), "ckks_public_key_export")
        return out

    def encrypt_pk(self, pt, level: int, scale: float, enc_seed: int, n_limbs: int | None = None) -> Ciphertext:
        """Public-key encryption: ct = (v b + m + e0, v a + e1) over q_0..q_level."""
        ct = self.new_ct(n_limbs or level + 1, level, scale)
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_encrypt_pk(self._h, pt.data_ptr(), level, scale, enc_seed, ctypes.byref(h)),
               "ckks_encrypt_pk")
        return ct

    def decrypt(self, ct: Ciphertext):
        pt = self.new_pt(ct.level)
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_decrypt(self._h, ctypes.byref(h), pt.data_ptr()), "ckks_decrypt")
        return pt

    def decrypt_decode(self, ct: Ciphertext, n_slots: int | None = None) -> np.ndarray:
        return self.decode(self.decrypt(ct), ct.level, ct.scale, n_slots)

    # ---- evaluation ----
    def _out_like(self, a: Ciphertext, out: Ciphertext | None) -> Ciphertext:
        return out if out is not None else self.new_ct(a.level + 1, a.level, a.scale)

    def _binary(self, fn, a: Ciphertext, b: Ciphertext, out: Ciphertext | None, what: str) -> Ciphertext:
        out = self._out_like(a, out)
        ha, hb, ho = a.handle(self.log_n), b.handle(self.log_n), out.handle(self.log_n)
        _check(fn(self._h, ctypes.byref(ha), ctypes.byref(hb), ctypes.byref(ho)), what)
        out.level, out.scale = ho.level, ho.scale
        return out

    def add(self, a, b, out=None):
        return self._binary(self.lib.ckks_add, a, b, out, "ckks_add")

    def sub(self, a, b, out=None):
        return self._binary(self.lib.ckks_sub, a, b, out, "ckks_sub")

    def mul_relin(self, a, b, out=None):
        return self._binary(self.lib.ckks_mul_relin, a, b, out, "ckks_mul_relin")

    def mul_plain(self, a: Ciphertext, pt, pt_scale: float, out=None) -> Ciphertext:
        out = self._out_like(a, out)
        ha, ho = a.handle(self.log_n), out.handle(self.log_n)
        _check(self.lib.ckks_mul_plain(self._h, ctypes.byref(ha), pt.data_ptr(), pt_scale, ctypes.byref(ho)),
               "ckks_mul_plain")
        out.level, out.scale = ho.level, ho.scale
        return out

    def add_plain(self, a: Ciphertext, pt, out=None) -> Ciphertext:
        out = self._out_like(a, out)
        ha, ho = a.handle(self.log_n), out.handle(self.log_n)
        _check(self.lib.ckks_add_plain(self._h, ctypes.byref(ha), pt.data_ptr(), ctypes.byref(ho)),
               "ckks_add_plain")
        out.level, out.scale = ho.level, ho.scale
        return out

    def mul_int(self, a: Ciphertext, k: int, out=None) -> Ciphertext:
        out = self._out_like(a, out)
        ha, ho = a.handle(self.log_n), out.handle(self.log_n)
        _check(self.lib.ckks_mul_int(self._h, ctypes.byref(ha), k, ctypes.byref(ho)), "ckks_mul_int")
        out.level, out.scale = ho.level, ho.scale
        return out

    def rescale(self, a: Ciphertext) -> Ciphertext:
        """In place: drops the top prime."""
        h = a.handle(self.log_n)
        _check(self.lib.ckks_rescale(self._h, ctypes.byref(h)), "ckks_rescale")
        a.level, a.scale = h.level, h.scale
        return a

    def rescale_noalloc(self, a: Ciphertext) -> Ciphertext:
        """In place, like rescale(), without any device allocation (fixed
        workspace inside the library; concurrent calls race)."""
        h = a.handle(self.log_n)
        _check(self.lib.ckks_rescale_noalloc(self._h, ctypes.byref(h)), "ckks_rescale_noalloc")
        a.level, a.scale = h.level, h.scale
        return a

    def automorph(self, a: Ciphertext, g: int, out=None) -> Ciphertext:
        out = self._out_like(a, out)
        ha, ho = a.handle(self.log_n), out.handle(self.log_n)
        _check(self.lib.ckks_automorph(self._h, ctypes.byref(ha), g, ctypes.byref(ho)), "ckks_automorph")
        out.level, out.scale = ho.level, ho.scale
        return out

    def rotate(self, a: Ciphertext, k: int, out=None) -> Ciphertext:
        out = self._out_like(a, out)
        ha, ho = a.handle(self.log_n), out.handle(self.log_n)
        _check(self.lib.ckks_rotate(self._h, ctypes.byref(ha), k, ctypes.byref(ho)), "ckks_rotate")
        out.level, out.scale = ho.level, ho.scale
        return out

    def conjugate(self, a: Ciphertext, out=None) -> Ciphertext:
        out = self._out_like(a, out)
        ha, ho = a.handle(self.log_n), out.handle(self.log_n)
        _check(self.lib.ckks_conjugate(self._h, ctypes.byref(ha), ctypes.byref(ho)), "ckks_conjugate")
        out.level, out.scale = ho.level, ho.scale
        return out

    # ---- batched ----
    def _handles(self, cts):
        arr = (CkksCt * len(cts))()
        for i, c in enumerate(cts):
            arr[i] = c.handle(self.log_n)
        return arr

    def mul_relin_batch(self, a, b, out, rescale: int = RESCALE_NONE) -> None:
        """out[i] = a[i] * b[i] relinearised; rescale: RESCALE_NONE (False),
        RESCALE_SEPARATE (True: ModDown, then rescale) or RESCALE_MERGED."""
        ha, hb, ho = self._handles(a), self._handles(b), self._handles(out)
        _check(self.lib.ckks_mul_relin_batch(self._h, ha, hb, ho, len(a), int(rescale)), "ckks_mul_relin_batch")
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale

    def rotate_batch(self, cts, steps, out) -> None:
        hi, ho = self._handles(cts), self._handles(out)
        ks = (ctypes.c_int32 * len(steps))(*steps)
        _check(self.lib.ckks_rotate_batch(self._h, hi, ks, ho, len(cts)), "ckks_rotate_batch")
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale

    def rotate_hoisted(self, cts, steps, out) -> None:
        """out[j * len(cts) + i] = Rot(cts[i], steps[j]) sharing one ModUp per input."""
        hi, ho = self._handles(cts), self._handles(out)
        ks = (ctypes.c_int32 * len(steps))(*steps)
        _check(self.lib.ckks_rotate_hoisted(self._h, hi, len(cts), ks, len(steps), ho), "ckks_rotate_hoisted")
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale

    def _batch_out(self, a, out):
        return out if out is not None else [self.new_ct(c.level + 1, c.level, c.scale) for c in a]

    def _finish(self, out, ho):
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale
        return out

    def add_batch(self, a, b, out=None, subtract: bool = False):
        out = self._batch_out(a, out)
        ha, hb, ho = self._handles(a), self._handles(b), self._handles(out)
        _check(self.lib.ckks_add_batch(self._h, ha, hb, ho, len(a), int(subtract)), "ckks_add_batch")
        return self._finish(out, ho)

    def mul_int_batch(self, a, k: int, out=None):
        out = self._batch_out(a, out)
        ha, ho = self._handles(a), self._handles(out)
        _check(self.lib.ckks_mul_int_batch(self._h, ha, k, ho, len(a)), "ckks_mul_int_batch")
        return self._finish(out, ho)

    def mul_plain_batch(self, a, pt, pt_scale: float, out=None):
        out = self._batch_out(a, out)
        ha, ho = self._handles(a), self._handles(out)
        _check(self.lib.ckks_mul_plain_batch(self._h, ha, pt.data_ptr(), pt_scale, ho, len(a)),
               "ckks_mul_plain_batch")
        return self._finish(out, ho)

    def add_plain_batch(self, a, pt, out=None):
        out = self._batch_out(a, out)
        ha, ho = self._handles(a), self._handles(out)
        _check(self.lib.ckks_add_plain_batch(self._h, ha, pt.data_ptr(), ho, len(a)), "ckks_add_plain_batch")
        return self._finish(out, ho)

    def mul_relin_host(self, a_host, b_host, scale_a: float, scale_b: float, level: int, out_host,
                       rescale: int = RESCALE_NONE, chunk: int = 16) -> float:
        """Products of pairs held in host memory (page-locked torch tensors of
        shape [n, 2, level+1, N], int64 view of the residues), streamed through
        the GPU with copies overlapping compute; returns the products' scale."""
        n = int(a_host.shape[0])
        sc = ctypes.c_double()
        _check(self.lib.ckks_mul_relin_host(self._h, a_host.data_ptr(), b_host.data_ptr(), scale_a, scale_b, level,
                                            n, int(rescale), chunk, out_host.data_ptr(), ctypes.byref(sc)),
               "ckks_mul_relin_host")
        return sc.value

    def rescale_batch(self, cts) -> None:
        h = self._handles(cts)
        _check(self.lib.ckks_rescale_batch(self._h, h, len(cts)), "ckks_rescale_batch")
        for i, c in enumerate(cts):
            c.level, c.scale = h[i].level, h[i].scale

    def set_key_compression(self, on: bool) -> None:
        """Keys generated afterwards store b and the generator state of a only."""
        _check(self.lib.ckks_set_key_compression(self._h, int(on)), "ckks_set_key_compression")

    # ---- bootstrapping ----
    def keygen_boot(self, seed: int, rot_steps=(), conj: bool = True) -> None:
        arr = (ctypes.c_int32 * max(1, len(rot_steps)))(*rot_steps)
        _check(self.lib.ckks_keygen_from_seed(self._h, seed, arr, len(rot_steps), int(conj), 1),
               "ckks_keygen_from_seed")

    def boot_set_slots(self, n_slots: int) -> None:
        """Sparse-slot bootstrapping (before keygen_boot and boot_setup)."""
        _check(self.lib.ckks_boot_set_slots(self._h, n_slots), "ckks_boot_set_slots")

    def boot_setup(self) -> None:
        _check(self.lib.ckks_boot_setup(self._h), "ckks_boot_setup")

    def boot_rotation_steps(self) -> list:
        n = self.lib.ckks_boot_rotation_steps(self._h, None, 0)
        if n < 0:
            raise CkksError(n, "ckks_boot_rotation_steps")
        out = (ctypes.c_int32 * max(1, n))()
        self.lib.ckks_boot_rotation_steps(self._h, out, n)
        return [int(x) for x in out[:n]]

    def boot_constant_count(self) -> int:
        n = self.lib.ckks_boot_constant_count(self._h)
        if n < 0:
            raise CkksError(n, "ckks_boot_constant_count")
        return n

    def boot_import(self, coeffs, cheb) -> None:
        arr = np.ascontiguousarray(np.stack(coeffs), dtype=np.int64)
        ch = np.ascontiguousarray(cheb, dtype=np.float64)
        _check(self.lib.ckks_boot_import(self._h, arr.ctypes.data, arr.shape[0], ch.ctypes.data, len(ch)),
               "ckks_boot_import")

    def boot_export(self):
        cnt = self.boot_constant_count()
        arr = np.zeros((cnt, self.n), dtype=np.int64)
        ch = np.zeros(61)
        _check(self.lib.ckks_boot_export(self._h, arr.ctypes.data, cnt, ch.ctypes.data, 61), "ckks_boot_export")
        return arr, ch

    def bootstrap_batch(self, cts, out=None) -> list:
        out_level = self.n_q - 1 - 16
        out = out if out is not None else [self.new_ct(out_level + 1) for _ in cts]
        hi, ho = self._handles(cts), self._handles(out)
        _check(self.lib.ckks_bootstrap_batch(self._h, hi, ho, len(cts)), "ckks_bootstrap_batch")
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale
        return out

    def boot_linear(self, index: int, cts, out=None) -> list:
        """Plan level `index` of the bootstrap's special DFT alone (ckks_boot_linear)."""
        if out is None:
            out = [self.new_ct(c.level) for c in cts]
        hi, ho = self._handles(cts), self._handles(out)
        _check(self.lib.ckks_boot_linear(self._h, index, hi, ho, len(cts)), "ckks_boot_linear")
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale
        return out

    def bootstrap(self, ct) -> "Ciphertext":
        return self.bootstrap_batch([ct])[0]

    def bootstrap_iterative_batch(self, cts, log2_k: int, out=None) -> list:
        out_level = self.n_q - 1 - 16
        out = out if out is not None else [self.new_ct(out_level + 1) for _ in cts]
        hi, ho = self._handles(cts), self._handles(out)
        _check(self.lib.ckks_bootstrap_iterative_batch(self._h, hi, ho, len(cts), int(log2_k)),
               "ckks_bootstrap_iterative_batch")
        for i, c in enumerate(out):
            c.level, c.scale = ho[i].level, ho[i].scale
        return out

    # ---- host exchange ----
    def export_ct(self, ct: Ciphertext) -> np.ndarray:
        """The active limbs as they live in HBM: uint64 [2, level+1, N], NTT domain."""
        out = np.zeros((2, ct.level + 1, self.n), dtype=np.uint64)
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_ct_export_ntt(self._h, ctypes.byref(h), out.ctypes.data), "ckks_ct_export_ntt")
        return out

    def export_coeff(self, ct) -> np.ndarray:
        """The active limbs in the coefficient domain (ckks_ct_export); ct is a
        Ciphertext or a raw CkksCt handle."""
        h = ct if isinstance(ct, CkksCt) else ct.handle(self.log_n)
        out = np.zeros((2, h.level + 1, self.n), dtype=np.uint64)
        _check(self.lib.ckks_ct_export(self._h, ctypes.byref(h), out.ctypes.data), "ckks_ct_export")
        return out

    def import_coeff(self, arr: np.ndarray, ct) -> None:
        """Fill ct's active limbs from coefficient-domain limbs (ckks_ct_import)."""
        arr = np.ascontiguousarray(arr, dtype=np.uint64)
        h = ct if isinstance(ct, CkksCt) else ct.handle(self.log_n)
        _check(self.lib.ckks_ct_import(self._h, arr.ctypes.data, ctypes.byref(h)), "ckks_ct_import")

    def ct_alloc(self, n_limbs: int) -> CkksCt:
        """A library-owned ciphertext buffer (ckks_ct_alloc): a raw handle."""
        h = CkksCt()
        _check(self.lib.ckks_ct_alloc(self._h, n_limbs, ctypes.byref(h)), "ckks_ct_alloc")
        return h

    def ct_free(self, h: CkksCt) -> None:
        _check(self.lib.ckks_ct_free(self._h, ctypes.byref(h)), "ckks_ct_free")

    def export_host(self, ct: Ciphertext, host) -> None:
        """Copy the active NTT-domain limbs into a (pinned) host torch tensor [2, level+1, N]."""
        assert host.device.type == "cpu" and host.is_contiguous() and host.numel() >= 2 * (ct.level + 1) * self.n
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_ct_export_ntt(self._h, ctypes.byref(h), host.data_ptr()), "ckks_ct_export_ntt")

    def import_host(self, ct: Ciphertext, host) -> None:
        """Fill ct's active NTT-domain limbs from a (pinned) host torch tensor [2, level+1, N]."""
        assert host.device.type == "cpu" and host.is_contiguous() and host.numel() >= 2 * (ct.level + 1) * self.n
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_ct_import_ntt(self._h, host.data_ptr(), ctypes.byref(h)), "ckks_ct_import_ntt")

    # ---- packed wire format ----
    def wire_bytes(self, level: int) -> int:
        b = ctypes.c_uint64()
        _check(self.lib.ckks_wire_bytes(self._h, level, ctypes.byref(b)), "ckks_wire_bytes")
        return int(b.value)

    def export_packed(self, ct: Ciphertext, host=None):
        """Pack on the GPU and copy out: a uint8 numpy array, or into `host`
        (an 8-byte aligned CPU torch tensor of at least wire_bytes bytes)."""
        h = ct.handle(self.log_n)
        if host is None:
            out = np.zeros(self.wire_bytes(ct.level) // 8, dtype=np.uint64)
            _check(self.lib.ckks_ct_export_packed(self._h, ctypes.byref(h), out.ctypes.data), "ckks_ct_export_packed")
            return out.view(np.uint8)
        _check(self.lib.ckks_ct_export_packed(self._h, ctypes.byref(h), host.data_ptr()), "ckks_ct_export_packed")
        return host

    def import_packed(self, data, level: int, scale: float, n_limbs: int | None = None) -> Ciphertext:
        ct = self.new_ct(n_limbs or level + 1, level, scale)
        h = ct.handle(self.log_n)
        ptr = data.data_ptr() if hasattr(data, "data_ptr") else np.ascontiguousarray(data).ctypes.data
        _check(self.lib.ckks_ct_import_packed(self._h, ptr, ctypes.byref(h)), "ckks_ct_import_packed")
        return ct

    def mul_relin_host_packed(self, a_host, b_host, scale_a: float, scale_b: float, level: int, out_host,
                              rescale: int = RESCALE_NONE, chunk: int = 16) -> float:
        """ckks_mul_relin_host on packed host buffers (page-locked uint8 torch
        tensors of n x wire_bytes(level) and n x wire_bytes(level') bytes)."""
        n = int(a_host.numel() // self.wire_bytes(level))
        sc = ctypes.c_double()
        _check(self.lib.ckks_mul_relin_host_packed(self._h, a_host.data_ptr(), b_host.data_ptr(), scale_a, scale_b,
                                                   level, n, int(rescale), chunk, out_host.data_ptr(),
                                                   ctypes.byref(sc)), "ckks_mul_relin_host_packed")
        return sc.value

    def import_ct(self, arr: np.ndarray, level: int, scale: float, n_limbs: int | None = None) -> Ciphertext:
        """A new ciphertext from NTT-domain limbs uint64 [2, level+1, N]."""
        arr = np.ascontiguousarray(arr, dtype=np.uint64)
        ct = self.new_ct(n_limbs or level + 1, level, scale)
        h = ct.handle(self.log_n)
        _check(self.lib.ckks_ct_import_ntt(self._h, arr.ctypes.data, ctypes.byref(h)), "ckks_ct_import_ntt")
        return ct


def tune_dnum(w, cands=(2, 3, 4, 6), batch: int = 16, seed: int = 1, stream=None):
    """Autotune dnum for a workload's prime chain (ckks_tune_dnum): returns
    (best dnum, {dnum: ms per HMult+relin+rescale, inf where it does not fit})."""
    torch = _torch()
    lib = load_library()
    p = CkksParams()
    p.log_n, p.n_q, p.n_p, p.dnum, p.h = w.log_n, len(w.q_bits), len(w.p_bits), w.dnum, w.h
    for i, b in enumerate(w.q_bits):
        p.q_bits[i] = b
    for i, b in enumerate(w.p_bits):
        p.p_bits[i] = b
    p.log2_scale, p.sigma = w.log2_scale, w.sigma
    st = stream if stream is not None else torch.cuda.current_stream()
    cs = (ctypes.c_uint32 * len(cands))(*cands)
    ms = (ctypes.c_double * len(cands))()
    best = ctypes.c_uint32()
    _check(lib.ckks_tune_dnum(ctypes.byref(p), ctypes.c_void_p(st.cuda_stream), cs, len(cands), batch, seed,
                              ctypes.byref(best), ms), "ckks_tune_dnum")
    return best.value, {int(d): float(ms[i]) for i, d in enumerate(cands)}


class Op:
    """One operation of an uneven batch: (context, kind, a, b, out, k, rescale)."""

    def __init__(self, ctx: Context, op: int, a: Ciphertext, out: Ciphertext, b: Ciphertext | None = None,
                 k: int = 0, rescale: bool = False):
        self.ctx, self.op, self.a, self.b, self.out, self.k, self.rescale = ctx, op, a, b, out, k, rescale


def _op_array(ops):
    arr = (CkksOpDesc * len(ops))()
    keep = []
    for i, o in enumerate(ops):
        ha = o.a.handle(o.ctx.log_n)
        hb = o.b.handle(o.ctx.log_n) if o.b is not None else None
        ho = o.out.handle(o.ctx.log_n)
        keep += [ha, hb, ho]
        arr[i] = CkksOpDesc(o.op, o.ctx._h.value, ctypes.pointer(ha), ctypes.pointer(hb) if hb else None,
                            ctypes.pointer(ho), o.k, int(o.rescale))
    return arr, keep


def execute(ops) -> None:
    """Run independent operations grouped by (context, kind, level)."""
    lib = load_library()
    arr, keep = _op_array(ops)
    _check(lib.ckks_exec(arr, len(ops)), "ckks_exec")
    for i, o in enumerate(ops):
        o.out.level, o.out.scale = arr[i].out.contents.level, arr[i].out.contents.scale


class Graph:
    """A captured uneven batch: launch() replays every operation at once."""

    def __init__(self, ops, stream=None):
        import torch
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if self.stream.cuda_stream == 0:  # the legacy default stream cannot be captured
            self.stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        arr, self._keep = _op_array(ops)
        g = ctypes.c_void_p()
        _check(self.lib.ckks_exec_capture(arr, len(ops), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(g)),
               "ckks_exec_capture")
        self._g = g
        for i, o in enumerate(ops):
            o.out.level, o.out.scale = arr[i].out.contents.level, arr[i].out.contents.scale

    def launch(self) -> None:
        _check(self.lib.ckks_graph_launch(self._g, ctypes.c_void_p(self.stream.cuda_stream)), "ckks_graph_launch")

    def close(self) -> None:
        if getattr(self, "_g", None):
            self.lib.ckks_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tensor_to_u64(t) -> np.ndarray:
    """Copy a device int64 tensor to host as uint64 (same bits)."""
    return t.detach().cpu().numpy().view(np.uint64)


def u64_to_tensor(a: np.ndarray, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)
