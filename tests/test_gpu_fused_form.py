"""The fused key-switch pipeline (CKKS_FORM_FUSED): the inverse transform's
column stages, the basis conversion and the forward transform's column stages
in one kernel per column tile.  Every limb must equal the oracle's and the
unfused uint64 form's: ModUp digits (full and partial), the plain ModDown
(separate rescale), the merged ModDown-rescale, hoisted rotations, on several
ring degrees; N = 2^17 falls back to the unfused kernels."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _pair(w, rot=(1, 2, -1)):
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    ctx.set_form("fused")
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    ctx.keygen(7, rot_steps=rot)
    orc.keygen(7)
    orc.gen_rotation_keys(rot)
    return ctx, orc


def _enc(w, ctx, orc, seed, count, level=None):
    level = len(w.q_bits) - 1 if level is None else level
    scale = 2.0 ** w.log2_scale
    z = si.messages(seed, count, w.slots)
    out = []
    for i in range(count):
        m = orc.encode(z[i], scale)
        out.append((ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 40 + i),
                    orc.encrypt(orc.pt_from_int(m, level), level, scale, 40 + i)))
    return out


@pytest.mark.parametrize("name", ["toy", "small", "mid", "n15", "n17", "smallq", "bigq"])
def test_fused_form_bit_exact_vs_oracle(name):
    import paper_2506_19693_gb300 as ck
    w = {"toy": si.TOY, "small": si.SMALL, "mid": si.MID, "n15": si.N15, "n17": si.N17,
         "smallq": si.SMALLQ, "bigq": si.BIGQ}[name]
    ctx, orc = _pair(w)
    try:
        (a, ao), (b, bo) = _enc(w, ctx, orc, 31, 2)
        p = ctx.rescale(ctx.mul_relin(a, b))
        po = orc.rescale(orc.mul_relin(ao, bo))
        assert np.array_equal(ctx.export_ct(p), po.data)
        out = [ctx.new_ct(a.level + 1)]
        ctx.mul_relin_batch([a], [b], out, rescale=ck.RESCALE_MERGED)
        assert np.array_equal(ctx.export_ct(out[0]), orc.mul_relin_rescale(ao, bo).data)
        for k in (1, -1):
            assert np.array_equal(ctx.export_ct(ctx.rotate(a, k)), orc.rotate(ao, k).data)
        outs = [ctx.new_ct(a.level + 1) for _ in range(2)]
        ctx.rotate_hoisted([a], [1, 2], outs)
        want = orc.rotate_hoisted(ao, [1, 2])
        assert np.array_equal(ctx.export_ct(outs[0]), want[0].data)
        assert np.array_equal(ctx.export_ct(outs[1]), want[1].data)
        # one level down: a partial top digit
        if a.level >= 2:
            (c, co), = _enc(w, ctx, orc, 32, 1, level=a.level - 1)
            assert np.array_equal(ctx.export_ct(ctx.rotate(c, 2)), orc.rotate(co, 2).data)
    finally:
        ctx.close()


def test_fused_form_equals_uint64_form_full_size():
    """N = 2^16, 24 + 8 primes, 16 pairs per batched launch: separate and
    merged rescale and hoisted rotations, fused against unfused."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    pairs = 16
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen(1, rot_steps=[1, 1 << 14])
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(77, 2 * pairs, w.slots)
        cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 90 + i) for i in range(2 * pairs)]
        res = {}
        for form in ("uint64", "fused"):
            ctx.set_form(form)
            out = [ctx.new_ct(level + 1) for _ in range(pairs)]
            ctx.mul_relin_batch(cts[:pairs], cts[pairs:], out, rescale=ck.RESCALE_SEPARATE)
            merged = [ctx.new_ct(level + 1) for _ in range(pairs)]
            ctx.mul_relin_batch(cts[:pairs], cts[pairs:], merged, rescale=ck.RESCALE_MERGED)
            rots = [ctx.new_ct(level + 1) for _ in range(4)]
            ctx.rotate_hoisted(cts[:2], [1, 1 << 14], rots)
            res[form] = [ctx.export_ct(c) for c in out + merged + rots]
        for i, (x, y) in enumerate(zip(res["uint64"], res["fused"])):
            assert np.array_equal(x, y), i
        err = np.max(np.abs(ctx.decrypt_decode(merged[0]) - z[0] * z[pairs]))
        assert err < 2.0 ** -30, err
    finally:
        ctx.close()
