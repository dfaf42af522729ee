"""Pins for the oracle's bootstrapping pieces: the special-DFT factorisation
against the dense matrix, the merged levels against their definition, the
Chebyshev/double-angle EvalMod against FP64 sine, ModRaise against exact
integers, hoisted rotations against slot semantics, and the whole circuit
against the error bound (decrypted slots within 2^-12 of the input)."""
import math

import numpy as np
import pytest

import oracle
import oracle.bootstrap as ob
import synthetic_inputs as si


def _brv_perm(n):
    lb = int(math.log2(n))
    return np.array([int(format(i, f"0{lb}b")[::-1], 2) for i in range(n)])


def _dense(diags, n):
    m = np.zeros((n, n), dtype=np.complex128)
    for d, v in diags.items():
        m[np.arange(n), (np.arange(n) + d) % n] += v
    return m


@pytest.mark.parametrize("n", [4, 16, 64])
def test_stages_times_bitreversal_equal_special_dft(n):
    U = ob.special_dft_matrix(n)
    P = np.zeros((n, n))
    P[np.arange(n), _brv_perm(n)] = 1
    M = P.astype(np.complex128)
    for s in range(int(math.log2(n))):
        M = _dense(ob.stage_diags(n, 1 << s, False), n) @ M
    assert np.max(np.abs(M - U)) < 1e-12
    # inverse stages invert
    for s in range(int(math.log2(n))):
        f = _dense(ob.stage_diags(n, 1 << s, False), n)
        b = _dense(ob.stage_diags(n, 1 << s, True), n)
        assert np.max(np.abs(b @ f - np.eye(n))) < 1e-12


def test_special_dft_is_the_encoding_map():
    # slots z = U (p_lo + i p_hi) for real coefficients p (zeta_j^(N/2) = i)
    o = oracle.Oracle(5, (55,), (61,), 1)
    n = o.n
    p = np.random.default_rng(0).normal(size=n)
    z = o.embed(p)
    U = ob.special_dft_matrix(n // 2)
    assert np.max(np.abs(U @ (p[: n // 2] + 1j * p[n // 2:]) - z)) < 1e-12


def test_diag_matmul_matches_dense_product():
    n = 32
    rng = np.random.default_rng(1)
    a = {d: rng.normal(size=n) + 1j * rng.normal(size=n) for d in (0, 3, 17)}
    b = {d: rng.normal(size=n) + 1j * rng.normal(size=n) for d in (1, 5, 31)}
    assert np.max(np.abs(_dense(ob.diag_matmul(a, b, n), n) - _dense(a, n) @ _dense(b, n))) < 1e-12


@pytest.mark.parametrize("n", [256, 2048])
def test_merged_levels_are_the_slot_transforms(n):
    plan = ob.make_plan(int(math.log2(n)) + 1, 25)
    U = ob.special_dft_matrix(n)
    P = _brv_perm(n)
    rng = np.random.default_rng(2)
    w = rng.normal(size=n) + 1j * rng.normal(size=n)
    y = w[P].copy()
    for i, lv in enumerate(plan.stc):  # undo the folded 1/(2 pi)
        y = ob.diag_apply(lv.diags if i else {d: v * 2 * np.pi for d, v in lv.diags.items()}, y)
    assert np.max(np.abs(y - U @ w)) < 1e-10 * n
    z = U @ w
    for i, lv in enumerate(plan.cts):  # undo the folded 1/(2K)
        z = ob.diag_apply(lv.diags if i else {d: v * 2 * ob.K_RANGE for d, v in lv.diags.items()}, z)
    assert np.max(np.abs(z - w[P])) < 1e-10
    # BSGS plans reproduce the diagonals: sum_b Rot(sum_a pt_ba * Rot(x, a s), g b s)
    for lv in plan.cts + plan.stc:
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        acc = np.zeros(n, dtype=np.complex128)
        for b, items in lv.plan:
            inner = sum(vec * np.roll(x, -a * lv.step) for a, vec in items)
            acc += np.roll(inner, -lv.g * b * lv.step)
        assert np.max(np.abs(acc - ob.diag_apply(lv.diags, x))) < 1e-10


def test_level_budget_is_sixteen():
    plan = ob.make_plan(12, len(si.BOOT_Q_BITS))
    assert plan.top == 24
    assert [lv.level for lv in plan.cts] == [24, 23, 22]
    assert [lv.level for lv in plan.stc] == [11, 10, 9]
    assert ob.LEVELS_CTS + ob.EVALMOD_DEPTH + ob.LEVELS_STC == 16  # tau_bs (Sec. 5.1)


def test_evalmod_function_and_double_angles_give_the_sine():
    c = ob.chebyshev_coeffs(ob.evalmod_function(), ob.CHEB_DEGREE)
    u = np.linspace(-1, 1, 20001)
    f = ob.evalmod_function()(u)
    assert np.max(np.abs(ob.chebyshev_eval_plain(c, u) - f)) < 1e-12
    v = ob.chebyshev_eval_plain(c, u)
    for _ in range(ob.DOUBLE_ANGLES):
        v = 2 * v * v - 1
    t = ob.K_RANGE * u
    assert np.max(np.abs(v - np.sin(2 * np.pi * t))) < 1e-10
    # near an integer the scaled sine reproduces t - I to (2 pi)^2 (t-I)^3 / 6
    d = 2.0 ** -10
    assert abs(np.sin(2 * np.pi * (5 + d)) / (2 * np.pi) - d) < (2 * np.pi) ** 2 * d ** 3 / 6 * 1.01


def test_round_half_away():
    assert [ob.round_half_away(x) for x in (0.5, -0.5, 1.4999999, 2.5, -2.5, 0.0, 3.0)] == [1, -1, 1, 3, -3, 0, 3]
    assert ob.round_half_away(0.49999999999999994) == 0


@pytest.fixture(scope="module")
def boot_env():
    w = si.BOOT_SMALL
    plan = ob.make_plan(w.log_n, len(w.q_bits))
    o = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    o.keygen(1)
    o.gen_rotation_keys(plan.rotation_steps())
    o.gen_galois_key(o.conj_elt())
    ev = ob.Evaluator(o, plan, ob.encode_constants(o, plan))
    return w, plan, o, ev


def test_mod_raise_adds_an_exact_small_multiple_of_q0(boot_env):
    w, plan, o, ev = boot_env
    z = si.messages(4, 1, w.slots)[0]
    delta = 2.0 ** w.log2_scale
    ct = o.encrypt(o.pt_from_int(o.encode(z, delta), 0), 0, delta, 9)
    low = o.decrypt_coeffs(ct)
    raised = ev.mod_raise(ct)
    assert raised.level == plan.top
    high = o.decrypt_coeffs(raised)
    q0 = o.q[0]
    diff = [h - l for h, l in zip(high, low)]
    assert all(d % q0 == 0 for d in diff)
    assert max(abs(d // q0) for d in diff) < ob.K_RANGE


def test_hoisted_rotations_have_rotation_semantics(boot_env):
    w, plan, o, ev = boot_env
    z = si.messages(5, 1, w.slots)[0]
    scale = 2.0 ** 50
    lvl = 12
    ct = o.encrypt(o.pt_from_int(o.encode(z, scale), lvl), lvl, scale, 3)
    steps = [1, 4, 16][: len(plan.rotation_steps())]
    o.gen_rotation_keys(steps)
    for k, r in zip(steps, o.rotate_hoisted(ct, steps)):
        assert np.max(np.abs(o.decrypt_decode(r) - np.roll(z, -k))) < 2.0 ** -30


def test_bootstrap_error_bound_small_ring(boot_env):
    w, plan, o, ev = boot_env
    z = si.messages(6, 1, w.slots)[0]
    delta = 2.0 ** w.log2_scale
    ct = o.encrypt(o.pt_from_int(o.encode(z, delta), 0), 0, delta, 11)
    out = ev.bootstrap(ct)
    assert out.level == plan.top - 16
    err = np.max(np.abs(o.decrypt_decode(out) - z))
    assert err <= 2.0 ** -12, err
    assert abs(math.log2(out.scale) - w.log2_scale) < 1e-6


@pytest.mark.parametrize("which", ["cts", "stc"])
def test_linear_level_decrypts_to_the_level_matrix(boot_env, which):
    """Readings B10 and B11 (giant steps summed over Q_l P, baby steps never
    ModDown'd, one merged ModDown-rescale): an encrypted merged level decrypts
    to the level's diagonal matrix applied to the message, to noise level."""
    w, plan, o, ev = boot_env
    i = 0 if which == "cts" else len(plan.cts)
    lv = (plan.cts + plan.stc)[i]
    pts = ev.pts[i]
    delta = 2.0 ** w.log2_scale
    z = si.messages(8, 1, w.slots)[0]
    x = o.encrypt(o.pt_from_int(o.encode(z, delta), lv.level), lv.level, delta, 13)
    out = ev.linear(x, lv, pts)
    assert (out.level, out.scale) == (lv.level - 1, delta * float(o.q[lv.level]) / float(o.q[lv.level]))
    err = np.max(np.abs(o.decrypt_decode(out) - ob.diag_apply(lv.diags, z)))
    assert err < 2.0 ** -30, err


def test_iterative_bootstrap_refines_precision(boot_env):
    """Reading B12: the second pass refreshes 2^k times the first pass's
    error, so the result decrypts to the input about 2^k times closer, at the
    single bootstrap's level, with the scale label multiplied by 2^k."""
    w, plan, o, ev = boot_env
    z = si.messages(16, 1, w.slots)[0]
    delta = 2.0 ** w.log2_scale
    ct = o.encrypt(o.pt_from_int(o.encode(z, delta), 0), 0, delta, 19)
    one = ev.bootstrap(ct)
    e1 = np.max(np.abs(o.decrypt_decode(one) - z))
    k = 14
    two = ev.bootstrap_iterative(ct, k)
    e2 = np.max(np.abs(o.decrypt_decode(two) - z))
    assert (two.level, two.scale) == (one.level, one.scale * 2.0 ** k)
    assert e2 <= 2.0 ** -36, e2
    assert e2 <= e1 * 2.0 ** -8, (e1, e2)


def test_sparse_slot_bootstrap_error_bound():
    """Reading B13: 512 slots at N = 2^12 (d = 4 copies): the sub-sum keeps the
    subring part, the 512-slot transforms refresh it, and the output decrypts to
    the input within 2^-12, still repeated with period 512."""
    w = si.BOOT_SMALL
    plan = ob.make_plan(w.log_n, len(w.q_bits), log_slots=9)
    assert plan.subsum_steps == [512, 1024]
    assert set(plan.subsum_steps) <= set(plan.rotation_steps())
    o = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    o.keygen(2)
    o.gen_rotation_keys(plan.rotation_steps())
    o.gen_galois_key(o.conj_elt())
    ev = ob.Evaluator(o, plan, ob.encode_constants(o, plan))
    z = si.messages(30, 1, 512)[0]
    delta = 2.0 ** w.log2_scale
    ct = o.encrypt(o.pt_from_int(o.encode(np.tile(z, 4), delta), 0), 0, delta, 31)
    out = ev.bootstrap(ct)
    assert out.level == plan.top - 16
    got = o.decrypt_decode(out)
    assert np.max(np.abs(got - np.tile(z, 4))) <= 2.0 ** -12


def test_sparse_subsum_is_the_trace_onto_the_subring():
    """Reading B13's sub-sum, by its algebra: the rotations by n 2^i (n 2^i < N/2)
    generate the automorphisms g = 1 mod 4n, whose fixed ring is Z[X^d],
    d = N/(2n).  Summing over them maps X^j to d X^j when d divides j and to 0
    otherwise, so the decrypted coefficients are d m_j on multiples of d and
    noise elsewhere (N = 2^12, n = 512, d = 4)."""
    w = si.BOOT_SMALL
    plan = ob.make_plan(w.log_n, len(w.q_bits), log_slots=9)
    o = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    o.keygen(3)
    o.gen_rotation_keys(plan.subsum_steps)
    n, d = 1 << w.log_n, (1 << w.log_n) // (2 * 512)
    rng = np.random.default_rng(11)
    m = rng.integers(-(1 << 30), 1 << 30, size=n)
    ct = o.encrypt(o.pt_from_int(m, 0), 0, 1.0, 12)
    for k in plan.subsum_steps:
        ct = o.add(ct, o.rotate(ct, k))
    got = np.array([float(v) for v in o.decrypt_coeffs(ct)])
    want = np.where(np.arange(n) % d == 0, d * m, 0).astype(np.float64)
    assert np.max(np.abs(got - want)) < 2.0 ** 16
    assert np.max(np.abs(got[np.arange(n) % d == 0])) > 2.0 ** 29  # the kept part is the message, not noise
