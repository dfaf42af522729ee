"""The benchmark's roofline arithmetic on synthetic profiles (CPU only): the
byte models of the op-level fractions, the roofs of each form, and the
binding roof as the larger fraction."""
import importlib.util
import os

import pytest

import synthetic_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"mac_per_s": 1.0e12, "bfly_fwd_loose_per_s": 2.0e12, "bfly_fwd_strict_per_s": 1.0e12,
         "bfly_inv_approx_per_s": 1.0e12, "bfly_inv_exact_per_s": 1.0e12}


def test_hmult_bytes_is_the_fused_minimum(bench):
    # 2 inputs x 2 polys x 24 limbs + key (3 digits x 2 x 32 limbs) / 64 + output 2 x 23 limbs, 512 KiB limbs
    assert bench.hmult_bytes(si.PLAIN, 64) == 512 * 1024 * (96 + 3 * 2 * 32 / 64 + 46)
    assert abs(bench.hmult_bytes(si.PLAIN, 64) / 2 ** 20 - 72.5) < 1e-9


def test_bootstrap_bytes_sums_key_switches_by_level(bench):
    w = si.BOOT
    hist = [0] * 64
    hist[20] = 32  # 2 key switches per ciphertext at level 20 for a batch of 16
    alpha = -(-len(w.q_bits) // w.dnum)
    ndig = -(-21 // alpha)
    want = 8 * w.n * 2 * (2 * 21 + ndig * 2 * (21 + len(w.p_bits)) / 16 + 2 * 20)
    assert abs(bench.bootstrap_bytes(hist, w, 16) - want) < 1e-6


def test_ntt_roof_weights_loose_and_strict_limbs(bench):
    w = si.PLAIN
    n = w.n
    # 10 forward limbs in pass A, 4 of them strict
    prof = {"ntt_fwd_pass_a": (1.0, 1, 10), "ntt_fwd_strict_limbs": (0.0, 0, 4)}
    hbm, alu, tensor = bench.kernel_work("ntt_fwd_pass_a", 10, w, 3, prof)
    per_limb = n // 2 * (w.log_n - 8)
    assert hbm == 2 * 8 * n * 10 and tensor is None
    assert dict((k, o) for o, k in alu) == {"bfly_fwd_loose_per_s": 6 * per_limb, "bfly_fwd_strict_per_s": 4 * per_limb}


def test_binding_roof_is_the_larger_fraction(bench):
    w = si.PLAIN
    # one pass-A launch over 100 loose limbs taking 1 ms
    prof = {"ntt_fwd_pass_a": (1.0, 1, 100)}
    parts = [(prof, w, 3)]
    r = bench.roofline(parts, 6000.0, "measured", PEAKS, 1700.0)
    n = w.n
    alu_frac = 100 * n // 2 * 8 / PEAKS["bfly_fwd_loose_per_s"] / 1e-3
    hbm_frac = 100 * 2 * 8 * n / 1e-3 / 6000e9
    assert r["kernel"] == "ntt_fwd_pass_a"
    assert abs(r["roofs"]["alu"]["frac"] - alu_frac) < 1e-12
    assert abs(r["roofs"]["hbm"]["frac"] - hbm_frac) < 1e-12
    assert r["bound"] == ("alu" if alu_frac > hbm_frac else "hbm")
    assert r["frac"] == max(alu_frac, hbm_frac)


def test_tensor_form_conversion_has_tensor_and_hbm_roofs_only(bench):
    w = si.PLAIN
    prof = {"bconv_tc": (2.0, 4, 4 * 192)}
    r = bench.roofline([(prof, w, 3)], 6000.0, "measured", PEAKS, 1700.0, name="bconv_tc")
    assert set(r["roofs"]) == {"hbm", "tensor"}
    flops = 4 * 192 * w.n * 64 * 2
    assert abs(r["roofs"]["tensor"]["achieved"] - flops / 2e-3 / 1e12) < 1e-9


def test_op_roofline_sums_each_class_at_its_roof(bench):
    w = si.PLAIN
    n = w.n
    prof = {"bconv": (1.0, 1, 1000), "ntt_inv_pass_b": (1.0, 1, 10)}
    op = bench.op_roofline([(prof, w, 3)], 4, 2e-3, 6000.0, PEAKS, 1700.0, 1.0e6)
    t = 1000 * n / PEAKS["mac_per_s"] + 10 * n // 2 * 8 / PEAKS["bfly_inv_approx_per_s"]
    assert abs(op["compute"]["frac"] - t / 2e-3) < 1e-12
    assert abs(op["hbm"]["frac"] - 1.0e6 * 2000 / 6000e9) < 1e-12
    assert op["ops_per_s"] == 2000


def test_cluster_ntt_work_is_one_pass_of_all_stages(bench):
    w = si.PLAIN
    n = w.n
    # 10 limbs in the one-pass cluster form, 5 of them strict
    prof = {"ntt_fwd_cluster": (1.0, 1, 10), "ntt_fwd_strict_limbs": (0.0, 0, 5)}
    hbm, alu, tensor = bench.kernel_work("ntt_fwd_cluster", 10, w, 3, prof)
    per_limb = n // 2 * w.log_n
    assert hbm == 2 * 8 * n * 10 and tensor is None
    assert dict((k, o) for o, k in alu) == {"bfly_fwd_loose_per_s": 5 * per_limb, "bfly_fwd_strict_per_s": 5 * per_limb}


def test_finish_row_pass_bytes_count_base_limbs(bench):
    """The row pass with the key-switch finish moves its input, the accumulator
    and the output (3 limbs), plus a base limb where the finish adds one; its
    butterflies are the 8 row stages."""
    w = si.PLAIN
    n = w.n
    prof = {"ntt_fwd_pass_b_finish": (1.0, 2, 12), "finish_base_limbs": (0.0, 0, 8),
            "ntt_fwd_pass_a": (1.0, 2, 12), "ntt_fwd_strict_limbs": (0.0, 0, 0)}
    hbm, alu, tensor = bench.kernel_work("ntt_fwd_pass_b_finish", 12, w, 3, prof)
    assert hbm == 8 * n * (3 * 12 + 8) and tensor is None
    assert dict((k, o) for o, k in alu) == {"bfly_fwd_loose_per_s": 12 * (n // 2) * 8, "bfly_fwd_strict_per_s": 0}
    # half of the class's launches: half of its base limbs
    hbm_half, _, _ = bench.kernel_work("ntt_fwd_pass_b_finish", 6, w, 3, prof)
    assert hbm_half == 8 * n * (3 * 6 + 4)
