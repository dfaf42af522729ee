"""Parity at the full ring N = 2^16 on the code paths the small rings cannot
reach, against definitions computed independently of the kernels:

* the benchmark's merged product (24 + 8 primes, dnum 3, tensor-core form):
  for 2048 sampled coefficients, the GPU's result against round(X / (P q_l))
  computed from the oracle's extended accumulator X with Python big integers
  (reading C21; the kernel estimates the conversion's overflow in fixed point
  and may land one above the rounded quotient, e = 1, which is counted);
* relinearised products with the merged ModDown-rescale at EvalMod's levels
  of the bootstrapping chain (25 + 9 primes: ten conversion sources);
* one CoeffToSlot and one SlotToCoeff level of the bootstrapping circuit
  (5-stage merged levels, 16 baby x 4 giant steps, the plaintext MAC at full
  size), bit-exact against the oracle's level with the oracle's constants."""
import math

import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _crt(residues, moduli):
    M = math.prod(moduli)
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M


def _enc_pair(ctx, orc, w, level, scale, seed):
    z = si.messages(seed, 2, w.slots)
    cts, ocs = [], []
    for i in range(2):
        m = orc.encode(z[i], scale)
        cts.append(ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 1000 * seed + i))
        ocs.append(orc.encrypt(orc.pt_from_int(m, level), level, scale, 1000 * seed + i))
    return z, cts, ocs


def test_merged_product_is_rounded_division_at_bench_shape():
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    ctx = ck.Context.from_workload(w)
    try:
        ctx.set_form(True)
        ctx.keygen(1)
        orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
        orc.keygen(1)
        level = len(w.q_bits) - 1
        z, (a, b), (ao, bo) = _enc_pair(ctx, orc, w, level, 2.0 ** w.log2_scale, 131)
        out = [ctx.new_ct(level + 1)]
        ctx.mul_relin_batch([a], [b], out, rescale=ck.RESCALE_MERGED)
        assert ctx.device_error() == 0
        got = ctx.export_coeff(out[0])  # coefficient domain, [2][level][N]
        # X = KS accumulator of d2 plus P (d0, d1), over q_0..q_l, P (oracle)
        d0, d1, d2 = orc.tensor(ao, bo)
        acc = orc.keyswitch_ext(d2, level, 0)
        emods = orc.ext_mods(level)
        mods = list(range(level + 1))
        P = math.prod(int(p) for p in orc.moduli[orc.n_q:])
        qcol = np.array([int(q) for q in orc.q[: level + 1]], dtype=np.uint64)[:, None]
        xc = []
        for p, d in enumerate((d0, d1)):
            x = acc[p].copy()
            x[: level + 1] = (x[: level + 1] + orc.mul_scalars(d, mods, [P % int(q) for q in orc.q[: level + 1]])) % qcol
            xc.append(orc.intt(x, emods))
        ext_moduli = [int(orc.moduli[m]) for m in emods]
        low = [int(q) for q in orc.q[:level]]
        S = int(orc.q[level]) * P
        Qlow = math.prod(low)
        rng = np.random.default_rng(5)
        ones = 0
        for p in range(2):
            for k in rng.choice(w.n, 1024, replace=False):
                X = _crt([xc[p][t, k] for t in range(len(emods))], ext_moduli)
                want = (X + (S - 1) // 2) // S
                g = _crt([got[p][t, k] for t in range(level)], low)
                e = (g - want) % Qlow
                e = e - Qlow if e > Qlow // 2 else e
                assert e in (0, 1), (p, int(k), e)
                ones += e
        print(f"merged product at N=2^16, L=24, K=8: e=1 at {ones} of 2048 sampled coefficients")
        # the fixed-point overflow estimate errs with probability about
        # (K+1) 2^-32 per coefficient: any e = 1 here would be a 2^-20 event
        assert ones <= 1
        # the whole product also equals the oracle's (exact) merged product
        want = orc.mul_relin_rescale(ao, bo)
        assert np.array_equal(ctx.export_ct(out[0]), want.data)
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def boot_pair():
    import torch
    import oracle
    import oracle.bootstrap as ob
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT
    ctx = ck.Context.from_workload(w)
    ctx.keygen_boot(1)
    ctx.boot_setup()
    plan = ob.make_plan(w.log_n, len(w.q_bits))
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    orc.keygen(1)
    yield w, ctx, orc, plan
    ctx.close()


@pytest.mark.parametrize("tensor_form", ["uint64", "tensor", "fused"])
def test_evalmod_level_products_bit_exact_at_full_ring(boot_pair, tensor_form):
    """B9: the relinearised product with ModDown and rescale merged, at two of
    EvalMod's levels of the bootstrapping chain (nine special primes)."""
    import paper_2506_19693_gb300 as ck
    w, ctx, orc, plan = boot_pair
    ctx.set_form(tensor_form)
    try:
        for level in (21, 13):
            scale = float(orc.q[0])
            z, (a, b), (ao, bo) = _enc_pair(ctx, orc, w, level, scale, 140 + level)
            out = [ctx.new_ct(level + 1)]
            ctx.mul_relin_batch([a], [b], out, rescale=ck.RESCALE_MERGED)
            want = orc.mul_relin_rescale(ao, bo)
            assert (out[0].level, out[0].scale) == (want.level, want.scale)
            assert np.array_equal(ctx.export_ct(out[0]), want.data), level
            assert ctx.device_error() == 0
    finally:
        ctx.set_form(False)


@pytest.fixture(scope="module")
def level_consts(boot_pair):
    import oracle.bootstrap as ob
    w, ctx, orc, plan = boot_pair
    consts = ob.encode_constants(orc, plan)
    mine_c, mine_cheb = ctx.boot_export()
    ctx.boot_import(consts, plan.cheb)
    yield consts
    ctx.boot_import(list(mine_c), mine_cheb)


@pytest.mark.parametrize("index", [0, 3], ids=["coeff_to_slot_0", "slot_to_coeff_0"])
def test_linear_level_bit_exact_at_full_ring(boot_pair, level_consts, index):
    """One merged level of the special DFT (B3, B10, B11) at N = 2^16 with the
    oracle's constants: every output limb equals the oracle's level, in all
    three basis-conversion forms."""
    import oracle.bootstrap as ob
    w, ctx, orc, plan = boot_pair
    levels = plan.cts + plan.stc
    lv = levels[index]
    orc.gen_rotation_keys(sorted(lv.rotations(plan.n_slots)))
    ev = ob.Evaluator(orc, plan, level_consts, levels={index})
    scale = 2.0 ** w.log2_scale
    z = si.messages(150 + index, 1, w.slots)[0]
    m = orc.encode(z, scale)
    co = orc.encrypt(orc.pt_from_int(m, lv.level), lv.level, scale, 7700 + index)
    cg = ctx.encrypt(ctx.pt_from_int(m, lv.level), lv.level, scale, 7700 + index)
    want = ev.linear(co, lv, ev.pts[index])
    for tensor_form in ("uint64", "tensor", "fused"):
        ctx.set_form(tensor_form)
        try:
            got = ctx.boot_linear(index, [cg])[0]
            assert (got.level, got.scale) == (want.level, want.scale)
            g = ctx.export_ct(got)
            assert np.array_equal(g, want.data), (tensor_form, int(np.sum(g != want.data)))
            assert ctx.device_error() == 0
        finally:
            ctx.set_form(False)
