"""Tensor-core form of basis conversion (byte-split fp16 GEMM on tcgen05 with
exact fp32 accumulation): every limb must equal the oracle's, and equal the
uint64 CUDA-core form, with no expired device wait."""
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
    ctx.set_form(True)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    ctx.keygen(7, rot_steps=rot)
    orc.keygen(7)
    orc.gen_rotation_keys(rot)
    return ctx, orc


def _enc(w, ctx, orc, seed, count):
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    z = si.messages(seed, count, w.slots)
    out = []
    for i in range(count):
        m = orc.encode(z[i], scale)
        out.append((ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 40 + i),
                    orc.encrypt(orc.pt_from_int(m, level), level, scale, 40 + i)))
    return out


@pytest.mark.parametrize("name", ["toy", "small", "mid", "n17", "smallq", "bigq"])
def test_tensor_form_bit_exact_vs_oracle(name):
    w = {"toy": si.TOY, "small": si.SMALL, "mid": si.MID, "n17": si.N17, "smallq": si.SMALLQ,
         "bigq": si.BIGQ}[name]
    ctx, orc = _pair(w)
    try:
        (a, ao), (b, bo) = _enc(w, ctx, orc, 31, 2)
        p = ctx.rescale(ctx.mul_relin(a, b))
        po = orc.rescale(orc.mul_relin(ao, bo))
        assert ctx.device_error() == 0
        assert np.array_equal(ctx.export_ct(p), po.data)
        for k in (1, -1):
            assert np.array_equal(ctx.export_ct(ctx.rotate(a, k)), orc.rotate(ao, k).data)
        outs = [ctx.new_ct(a.level + 1) for _ in range(2)]
        ctx.rotate_hoisted([a], [1, 2], outs)
        want = orc.rotate_hoisted(ao, [1, 2])
        assert np.array_equal(ctx.export_ct(outs[0]), want[0].data)
        assert np.array_equal(ctx.export_ct(outs[1]), want[1].data)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_merged_rescale_full_size_bit_exact_vs_oracle():
    """One pair at N = 2^16, L = 24 (the benchmark's ring) through the merged
    ModDown-rescale, tensor-core form, against the oracle."""
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    ctx = ck.Context.from_workload(w)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    try:
        ctx.set_form(True)
        ctx.keygen(3)
        orc.keygen(3)
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(88, 2, w.slots)
        pair = []
        for i in range(2):
            m = orc.encode(z[i], scale)
            pair.append((ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 70 + i),
                         orc.encrypt(orc.pt_from_int(m, level), level, scale, 70 + i)))
        out = [ctx.new_ct(level + 1)]
        ctx.mul_relin_batch([pair[0][0]], [pair[1][0]], out, rescale=ck.RESCALE_MERGED)
        want = orc.mul_relin_rescale(pair[0][1], pair[1][1])
        assert (out[0].level, out[0].scale) == (want.level, want.scale)
        assert np.array_equal(ctx.export_ct(out[0]), want.data)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_tensor_form_equals_uint64_form_full_size():
    """N = 2^16, 24 + 8 primes, 16 pairs per batched launch (the batched
    launch shape of the throughput benchmark, at a quarter of its batch)."""
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
        for form in (False, True):
            ctx.set_form(form)
            out = [ctx.new_ct(level + 1) for _ in range(pairs)]
            ctx.mul_relin_batch(cts[:pairs], cts[pairs:], out, rescale=ck.RESCALE_SEPARATE)
            merged = [ctx.new_ct(level + 1) for _ in range(pairs)]
            ctx.mul_relin_batch(cts[:pairs], cts[pairs:], merged, rescale=ck.RESCALE_MERGED)
            rots = [ctx.new_ct(level + 1) for _ in range(4)]
            ctx.rotate_hoisted(cts[:2], [1, 1 << 14], rots)
            res[form] = [ctx.export_ct(c) for c in out + merged + rots]
        assert ctx.device_error() == 0
        for x, y in zip(res[False], res[True]):
            assert np.array_equal(x, y)
    finally:
        ctx.close()
