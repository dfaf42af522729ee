"""The C-ABI library builds, loads and exports every entry point that
include/ckks.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "ckks.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ckks_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ["ckks_ctx_create", "ckks_keygen_from_seed", "ckks_encode", "ckks_decode", "ckks_encrypt",
                     "ckks_decrypt", "ckks_mul_relin", "ckks_rescale", "ckks_rotate", "ckks_mul_relin_batch",
                     "ckks_rotate_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2506_19693_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    import paper_2506_19693_gb300 as ck
    assert set(declared_symbols()) == set(ck.SIGNATURES)


def test_status_strings():
    import paper_2506_19693_gb300 as ck
    lib = ck.load_library()
    for s in range(-8, 1):
        assert lib.ckks_status_str(s)
    assert b"unknown" in lib.ckks_status_str(-99)


def test_invalid_params_rejected_without_gpu_work():
    import paper_2506_19693_gb300 as ck
    lib = ck.load_library()
    p = ck.CkksParams()
    p.log_n = 3  # below the supported ring degrees: rejected before any CUDA call
    p.n_q, p.n_p, p.dnum, p.h = 1, 1, 1, 1
    p.sigma = 3.2
    h = ctypes.c_void_p()
    assert lib.ckks_ctx_create(ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert lib.ckks_ctx_create(None, None, ctypes.byref(h)) == -1
