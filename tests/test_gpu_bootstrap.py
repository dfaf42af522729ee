"""GPU bootstrapping against the CPU oracle.

* plan: the same rotation steps and constant count as the oracle's plan;
* constants: GPU FP64 constants within FP64 rounding of the oracle's;
* bit-exact: with the oracle's constants imported, every output limb equals
  the oracle's bootstrap of the same ciphertext (N = 2^12, full 2^11 slots),
  with basis conversion on the CUDA cores and on the tensor cores;
* bound: with the GPU's own constants the decrypted slots are within 2^-12 of
  the input, at N = 2^12 and at N = 2^16 with 2^15 slots (the configuration
  bench.py times), output at level n_q - 17."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    import torch
    import oracle
    import oracle.bootstrap as ob
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT_SMALL
    ctx = ck.Context.from_workload(w)
    ctx.keygen_boot(1)
    ctx.boot_setup()
    plan = ob.make_plan(w.log_n, len(w.q_bits))
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    orc.keygen(1)
    orc.gen_rotation_keys(plan.rotation_steps())
    orc.gen_galois_key(orc.conj_elt())
    consts = ob.encode_constants(orc, plan)
    yield w, ctx, orc, plan, consts
    ctx.close()


def test_plan_matches_oracle(small):
    w, ctx, orc, plan, consts = small
    assert ctx.boot_rotation_steps() == plan.rotation_steps()
    assert ctx.boot_constant_count() == len(consts)


def test_gpu_constants_match_oracle_constants(small):
    w, ctx, orc, plan, consts = small
    got, cheb = ctx.boot_export()
    want = np.stack(consts)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-11 * scale + 2
    assert np.max(np.abs(cheb - plan.cheb)) < 1e-13


@pytest.mark.parametrize("tensor_form", ["uint64", "tensor", "fused"])
def test_bootstrap_bit_exact_with_oracle_constants(small, tensor_form):
    import oracle.bootstrap as ob
    w, ctx, orc, plan, consts = small
    ctx.set_form(tensor_form)
    z = si.messages(21, 1, w.slots)[0]
    delta = 2.0 ** w.log2_scale
    m = orc.encode(z, delta)
    co = orc.encrypt(orc.pt_from_int(m, 0), 0, delta, 77)
    cg = ctx.encrypt(ctx.pt_from_int(m, 0), 0, delta, 77)
    assert np.array_equal(ctx.export_ct(cg), co.data)
    mine_c, mine_cheb = ctx.boot_export()
    try:
        ctx.boot_import(consts, plan.cheb)
        out_g = ctx.bootstrap(cg)
        ev = ob.Evaluator(orc, plan, consts)
        out_o = ev.bootstrap(co)
        assert (out_g.level, out_g.scale) == (out_o.level, out_o.scale)
        got = ctx.export_ct(out_g)
        assert np.array_equal(got, out_o.data), int(np.sum(got != out_o.data))
        assert ctx.device_error() == 0
    finally:
        ctx.set_form(False)
        ctx.boot_import(list(mine_c), mine_cheb)


def test_bootstrap_error_bound_small_ring(small):
    w, ctx, orc, plan, consts = small
    z = si.messages(22, 2, w.slots)
    delta = 2.0 ** w.log2_scale
    cts = [ctx.encrypt(ctx.encode(z[i], 0, delta), 0, delta, 500 + i) for i in range(2)]
    outs = ctx.bootstrap_batch(cts)
    for i in range(2):
        assert outs[i].level == len(w.q_bits) - 17
        err = np.max(np.abs(ctx.decrypt_decode(outs[i]) - z[i]))
        assert err <= 2.0 ** -12, err


def test_bootstrap_error_bound_full_ring():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen_boot(1)
        ctx.boot_setup()
        z = si.messages(23, 2, w.slots)
        delta = 2.0 ** w.log2_scale
        cts = [ctx.encrypt(ctx.encode(z[i], 0, delta), 0, delta, 600 + i) for i in range(2)]
        outs = ctx.bootstrap_batch(cts)
        for i in range(2):
            assert outs[i].level == len(w.q_bits) - 17
            err = np.max(np.abs(ctx.decrypt_decode(outs[i]) - z[i]))
            assert err <= 2.0 ** -12, err
    finally:
        ctx.close()


@pytest.mark.parametrize("tensor_form", ["uint64", "tensor", "fused"])
def test_iterative_bootstrap_bit_exact_with_oracle_constants(small, tensor_form):
    """Reading B12 on the GPU: every limb of the two-pass result equals the
    oracle's, with the oracle's constants imported."""
    import oracle.bootstrap as ob
    w, ctx, orc, plan, consts = small
    ctx.set_form(tensor_form)
    z = si.messages(24, 1, w.slots)[0]
    delta = 2.0 ** w.log2_scale
    m = orc.encode(z, delta)
    co = orc.encrypt(orc.pt_from_int(m, 0), 0, delta, 78)
    cg = ctx.encrypt(ctx.pt_from_int(m, 0), 0, delta, 78)
    mine_c, mine_cheb = ctx.boot_export()
    try:
        ctx.boot_import(consts, plan.cheb)
        out_g = ctx.bootstrap_iterative_batch([cg], 14)[0]
        out_o = ob.Evaluator(orc, plan, consts).bootstrap_iterative(co, 14)
        assert (out_g.level, out_g.scale) == (out_o.level, out_o.scale)
        got = ctx.export_ct(out_g)
        assert np.array_equal(got, out_o.data), int(np.sum(got != out_o.data))
        assert ctx.device_error() == 0
    finally:
        ctx.set_form(False)
        ctx.boot_import(list(mine_c), mine_cheb)


def test_iterative_bootstrap_rejects_bad_arguments(small):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc, plan, consts = small
    delta = 2.0 ** w.log2_scale
    z = si.messages(25, 2, w.slots)
    a = ctx.encrypt(ctx.encode(z[0], 0, delta), 0, delta, 1)
    b = ctx.encrypt(ctx.encode(z[1], 0, 2 * delta), 0, 2 * delta, 2)
    with pytest.raises(ck.CkksError, match="E_SCALE|scale"):
        ctx.bootstrap_iterative_batch([a, b], 10)
    for k in (0, 31):
        with pytest.raises(ck.CkksError):
            ctx.bootstrap_iterative_batch([a], k)


def test_iterative_bootstrap_error_full_ring():
    """N = 2^16, 2^15 slots: the two-pass result is within 2^-32 of the input
    (one pass: about 2^-22), at the single bootstrap's output level."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen_boot(1)
        ctx.boot_setup()
        z = si.messages(26, 2, w.slots)
        delta = 2.0 ** w.log2_scale
        cts = [ctx.encrypt(ctx.encode(z[i], 0, delta), 0, delta, 610 + i) for i in range(2)]
        one = ctx.bootstrap_batch(cts)
        two = ctx.bootstrap_iterative_batch(cts, 16)
        for i in range(2):
            assert two[i].level == one[i].level == len(w.q_bits) - 17
            assert two[i].scale == one[i].scale * 2.0 ** 16
            e1 = np.max(np.abs(ctx.decrypt_decode(one[i]) - z[i]))
            e2 = np.max(np.abs(ctx.decrypt_decode(two[i]) - z[i]))
            assert e2 <= 2.0 ** -32 and e2 <= e1 * 2.0 ** -8, (e1, e2)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_bootstrap_error_bound_n17():
    """N = 2^17 with 2^16 slots on the eMLP-2 chain (l = 27 = 11 + 16): the
    levels are 6, 5 and 5 stages wide (32 baby steps at the widest); output at
    level 11, slots within 2^-12 of the input."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT17
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen_boot(1)
        ctx.boot_setup()
        z = si.messages(27, 2, w.slots)
        delta = 2.0 ** w.log2_scale
        cts = [ctx.encrypt(ctx.encode(z[i], 0, delta), 0, delta, 620 + i) for i in range(2)]
        outs = ctx.bootstrap_batch(cts)
        for i in range(2):
            assert outs[i].level == len(w.q_bits) - 17 == 11
            err = np.max(np.abs(ctx.decrypt_decode(outs[i]) - z[i]))
            assert err <= 2.0 ** -12, err
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_sparse_slot_bootstrap_bit_exact_and_error_bound():
    """Reading B13 at N = 2^12 with 512 slots (4 copies): the GPU plan equals the
    oracle's, the GPU constants match, the output limbs equal the oracle's with
    the oracle's constants imported, and with the GPU's own constants the slots
    come back within 2^-12, still repeated with period 512."""
    import torch
    import oracle
    import oracle.bootstrap as ob
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT_SMALL
    ctx = ck.Context.from_workload(w)
    try:
        ctx.boot_set_slots(512)
        ctx.keygen_boot(1)
        ctx.boot_setup()
        plan = ob.make_plan(w.log_n, len(w.q_bits), log_slots=9)
        assert ctx.boot_rotation_steps() == plan.rotation_steps()
        orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
        orc.keygen(1)
        orc.gen_rotation_keys(plan.rotation_steps())
        orc.gen_galois_key(orc.conj_elt())
        consts = ob.encode_constants(orc, plan)
        got, cheb = ctx.boot_export()
        want = np.stack(consts)
        assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want)) + 2
        z = si.messages(32, 1, 512)[0]
        delta = 2.0 ** w.log2_scale
        cg = ctx.encrypt(ctx.encode(np.tile(z, 4), 0, delta), 0, delta, 41)
        out = ctx.bootstrap(cg)
        assert out.level == len(w.q_bits) - 17
        assert np.max(np.abs(ctx.decrypt_decode(out) - np.tile(z, 4))) <= 2.0 ** -12
        m = orc.encode(np.tile(z, 4), delta)
        co = orc.encrypt(orc.pt_from_int(m, 0), 0, delta, 42)
        cg = ctx.encrypt(ctx.pt_from_int(m, 0), 0, delta, 42)
        ctx.boot_import(consts, plan.cheb)
        out_g = ctx.bootstrap(cg)
        out_o = ob.Evaluator(orc, plan, consts).bootstrap(co)
        assert (out_g.level, out_g.scale) == (out_o.level, out_o.scale)
        assert np.array_equal(ctx.export_ct(out_g), out_o.data)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_sparse_slot_bootstrap_full_ring():
    """N = 2^16 with 2^13 slots (4 copies): within 2^-12, output at level n_q - 17."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT
    ctx = ck.Context.from_workload(w)
    try:
        ctx.boot_set_slots(1 << 13)
        ctx.keygen_boot(1)
        ctx.boot_setup()
        z = si.messages(33, 2, 1 << 13)
        delta = 2.0 ** w.log2_scale
        cts = [ctx.encrypt(ctx.encode(np.tile(z[i], 4), 0, delta), 0, delta, 630 + i) for i in range(2)]
        outs = ctx.bootstrap_batch(cts)
        for i in range(2):
            assert outs[i].level == len(w.q_bits) - 17
            assert np.max(np.abs(ctx.decrypt_decode(outs[i]) - np.tile(z[i], 4))) <= 2.0 ** -12
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_sparse_slot_count_checks():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT_SMALL
    ctx = ck.Context.from_workload(w)
    try:
        for bad in (0, 1, 3, 768, 4096):  # not a power of two in 2 .. N/2
            with pytest.raises(ck.CkksError) as e:
                ctx.boot_set_slots(bad)
            assert ck.STATUS[e.value.status] == "CKKS_E_PARAM"
        ctx.boot_set_slots(512)
        assert 512 in ctx.boot_rotation_steps() and 1024 in ctx.boot_rotation_steps()
        ctx.boot_set_slots(512)  # the planned count again: accepted
        with pytest.raises(ck.CkksError) as e:
            ctx.boot_set_slots(1024)
        assert ck.STATUS[e.value.status] == "CKKS_E_STATE"
    finally:
        ctx.close()
