"""The key-switch finish in the forward NTT's row pass (ckks_ctx_set_fused_finish):
the last step of every ModDown, (acc - converted limbs) P^-1 + base (base read
through sigma_g for hoisted rotations), and of every merged ModDown-rescale,
(acc - converted limbs) S^-1 + base q_l^-1, computed in the output stage of the
transform that brings the converted limbs to the NTT domain.  The residues must
equal those of the separate element-wise finish, for every conversion form,
both row-pass tiles and both kinds of prime, and the result must still match
the oracle (the oracle parity tests run with the fused finish, the default).
The rescale's last step, (c - lift) q_l^-1, takes the same pass and is checked
the same way."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _ops(ck, ctx, w, steps, pairs, seed):
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    z = si.messages(seed, 2 * pairs, w.slots)
    cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, seed + 1 + i) for i in range(2 * pairs)]
    res = {}
    for on in (False, True):
        ctx.set_fused_finish(on)
        sep = [ctx.new_ct(level + 1) for _ in range(pairs)]
        ctx.mul_relin_batch(cts[:pairs], cts[pairs:], sep, rescale=ck.RESCALE_SEPARATE)
        mer = [ctx.new_ct(level + 1) for _ in range(pairs)]
        ctx.mul_relin_batch(cts[:pairs], cts[pairs:], mer, rescale=ck.RESCALE_MERGED)
        rots = [ctx.new_ct(level + 1) for _ in range(2 * len(steps))]
        ctx.rotate_hoisted(cts[:2], steps, rots)
        res[on] = [ctx.export_ct(c) for c in sep + mer + rots]
    ctx.set_fused_finish(True)
    return res, z, mer


@pytest.mark.parametrize("form", ["uint64", "tensor", "fused"])
@pytest.mark.parametrize("wl", ["SMALL", "SMALLQ", "BIGQ"])
def test_fused_finish_equals_separate_small_rings(form, wl):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = getattr(si, wl)
    ctx = ck.Context.from_workload(w)
    try:
        ctx.set_form(form)
        steps = [1, -1]
        ctx.keygen(1, rot_steps=steps)
        for rows in (16, 8):
            ctx.set_ntt_rows(rows)
            res, _, _ = _ops(ck, ctx, w, steps, 3, 40 + rows)
            assert ctx.device_error() == 0
            for i, (x, y) in enumerate(zip(res[False], res[True])):
                assert np.array_equal(x, y), (rows, i)
    finally:
        ctx.close()


@pytest.mark.parametrize("form", ["uint64", "tensor", "fused"])
def test_fused_finish_equals_separate_n65536(form):
    """N = 2^16, 24 + 8 primes, 8 pairs per batched launch, both finish tiles
    (each with the other tile for the plain transforms)."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    pairs = 8
    ctx = ck.Context.from_workload(w)
    try:
        ctx.set_form(form)
        steps = [1, 1 << 14]
        ctx.keygen(1, rot_steps=steps)
        for rows in (16, 8):
            ctx.set_ntt_rows(24 - rows)
            ctx.set_finish_rows(rows)
            res, z, mer = _ops(ck, ctx, w, steps, pairs, 61 + rows)
            assert ctx.device_error() == 0
            for i, (x, y) in enumerate(zip(res[False], res[True])):
                assert np.array_equal(x, y), (rows, i)
            err = np.max(np.abs(ctx.decrypt_decode(mer[0]) - z[0] * z[pairs]))
            assert err < 2.0 ** -30, err
    finally:
        ctx.close()


@pytest.mark.parametrize("wl", ["SMALL", "SMALLQ", "BIGQ", "PLAIN"])
def test_fused_rescale_equals_separate(wl):
    """The rescale's last step, (c - lift) q_l^-1, in the lift transform's row
    pass against k_rescale_finish, on a batch and on one ciphertext (the fused
    rescale against the oracle: test_gpu_parity.py)."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = getattr(si, wl)
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen(1)
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(77, 4, w.slots)
        outs = {}
        for on in (False, True):
            ctx.set_fused_finish(on)
            cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 80 + i) for i in range(4)]
            ctx.rescale_batch(cts[:3])
            ctx.rescale(cts[3])
            ctx.rescale(cts[3])  # and again one level down
            outs[on] = [ctx.export_ct(c) for c in cts]
        assert ctx.device_error() == 0
        for i, (x, y) in enumerate(zip(outs[False], outs[True])):
            assert np.array_equal(x, y), i
    finally:
        ctx.close()


def test_fused_finish_settings():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(si.SMALL)
    try:
        assert ck.STATUS[ctx.lib.ckks_ctx_set_fused_finish(ctx._h, 2)] == "CKKS_E_PARAM"
        ctx.set_fused_finish(False)
        ctx.set_fused_finish(True)
        assert ck.STATUS[ctx.lib.ckks_ctx_set_finish_rows(ctx._h, 12)] == "CKKS_E_PARAM"
        ctx.set_ntt_rows(8)
        assert ctx.finish_rows() == 8  # follows the NTT row tile
        ctx.set_finish_rows(16)
        assert ctx.finish_rows() == 16
        ctx.set_finish_rows(0)
        assert ctx.finish_rows() == 8
        ctx.keygen(1)
        ctx.tune_ntt(4)
        assert ctx.finish_rows() in (8, 16)
    finally:
        ctx.close()
