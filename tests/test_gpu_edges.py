"""Edge cases of the batched calls against the CPU oracle: empty batches,
batches past the per-launch ciphertext limit (128), and every level of the
chain down to the last one (ragged gadget digits, the merged ModDown-rescale
at level 1, products and rotations at level 0), in both basis-conversion
forms.  Every limb must equal the oracle's."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

MAX_CTS = 128


def _pair(w, rot=(1, -1)):
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    ctx.keygen(5, rot_steps=rot)
    orc.keygen(5)
    orc.gen_rotation_keys(rot)
    return ctx, orc


def _enc(w, ctx, orc, seed, level, count):
    scale = 2.0 ** w.log2_scale
    z = si.messages(seed, count, w.slots)
    out = []
    for i in range(count):
        m = orc.encode(z[i], scale)
        out.append((ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 100 * seed + i),
                    orc.encrypt(orc.pt_from_int(m, level), level, scale, 100 * seed + i)))
    return out


def _same(ctx, cg, co):
    assert (cg.level, cg.scale) == (co.level, co.scale)
    got = ctx.export_ct(cg)
    assert np.array_equal(got, co.data), int(np.sum(got != co.data))


@pytest.fixture(scope="module")
def small():
    ctx, orc = _pair(si.SMALL)
    yield si.SMALL, ctx, orc
    ctx.close()


def test_empty_batches(small):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = small
    ctx.mul_relin_batch([], [], [], rescale=ck.RESCALE_MERGED)
    ctx.rotate_hoisted([], [1], [])
    ctx.rescale_batch([])
    assert ctx.device_error() == 0


@pytest.mark.parametrize("tensor_form", [False, True], ids=["uint64", "tensor"])
def test_every_level_down_to_zero(small, tensor_form):
    """SMALL: 6 ciphertext primes, 2 special primes, digits of 2 primes, so
    odd levels leave a one-prime digit."""
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = small
    ctx.set_form(tensor_form)
    try:
        top = len(w.q_bits) - 1
        for level in range(top, -1, -1):
            (a, ao), (b, bo) = _enc(w, ctx, orc, 40 + level, level, 2)
            if level >= 1:
                out = [ctx.new_ct(level + 1) for _ in range(2)]
                ctx.mul_relin_batch([a, b], [b, a], out, rescale=ck.RESCALE_MERGED)
                _same(ctx, out[0], orc.mul_relin_rescale(ao, bo))
                sep = [ctx.new_ct(level + 1)]
                ctx.mul_relin_batch([a], [b], sep, rescale=ck.RESCALE_SEPARATE)
                _same(ctx, sep[0], orc.rescale(orc.mul_relin(ao, bo)))
            plain = [ctx.new_ct(level + 1)]
            ctx.mul_relin_batch([a], [b], plain, rescale=ck.RESCALE_NONE)
            _same(ctx, plain[0], orc.mul_relin(ao, bo))
            _same(ctx, ctx.rotate(a, 1), orc.rotate(ao, 1))
            outs = [ctx.new_ct(level + 1) for _ in range(2)]
            ctx.rotate_hoisted([b], [1, -1], outs)
            want = orc.rotate_hoisted(bo, [1, -1])
            _same(ctx, outs[0], want[0])
            _same(ctx, outs[1], want[1])
        assert ctx.device_error() == 0
    finally:
        ctx.set_form(False)


def test_batches_past_the_launch_limit():
    """N = 2^12, 3 primes: 133 pairs in one call (two launches of the batched
    kernels) give the same limbs as one call per pair, and the oracle's."""
    import paper_2506_19693_gb300 as ck
    w = si.TOY
    ctx, orc = _pair(w, rot=(1,))
    try:
        n = MAX_CTS + 5
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(60, 2, w.slots)
        ms = [orc.encode(z[i], scale) for i in range(2)]
        a = [ctx.encrypt(ctx.pt_from_int(ms[0], level), level, scale, 7000 + i) for i in range(n)]
        b = [ctx.encrypt(ctx.pt_from_int(ms[1], level), level, scale, 8000 + i) for i in range(n)]
        out = [ctx.new_ct(level + 1) for _ in range(n)]
        ctx.mul_relin_batch(a, b, out, rescale=ck.RESCALE_MERGED)
        for i in range(n):
            one = [ctx.new_ct(level + 1)]
            ctx.mul_relin_batch([a[i]], [b[i]], one, rescale=ck.RESCALE_MERGED)
            assert np.array_equal(ctx.export_ct(one[0]), ctx.export_ct(out[i])), i
        for i in (0, MAX_CTS - 1, MAX_CTS, n - 1):
            ao = orc.encrypt(orc.pt_from_int(ms[0], level), level, scale, 7000 + i)
            bo = orc.encrypt(orc.pt_from_int(ms[1], level), level, scale, 8000 + i)
            _same(ctx, out[i], orc.mul_relin_rescale(ao, bo))
        rots = [ctx.new_ct(level + 1) for _ in range(n)]
        ctx.rotate_hoisted(a, [1], rots)
        for i in (0, MAX_CTS, n - 1):  # hoisted: sigma applied to the lifted digits
            ao = orc.encrypt(orc.pt_from_int(ms[0], level), level, scale, 7000 + i)
            _same(ctx, rots[i], orc.rotate_hoisted(ao, [1])[0])
        assert ctx.device_error() == 0
    finally:
        ctx.close()
