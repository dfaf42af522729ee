"""The benchmark's own launch configuration against the oracle, on sampled
outputs: N = 2^16, 24 + 8 primes, dnum = 3, 64 pairs in one batched call with
ModDown and rescale merged, and 64 inputs rotated by every power of two up to
2^14 in one hoisted call, both on the tensor-core form the benchmark times.
The oracle recomputes a few outputs one by one; the rest are checked by
decryption against slot arithmetic."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bench_pair():
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    ctx = ck.Context.from_workload(w)
    ctx.set_form(True)
    ctx.keygen(1, rot_steps=list(w.rot_steps))
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    orc.keygen(1)
    orc.gen_rotation_keys([1, 1 << 14])
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    B = w.batch
    z = si.messages(100, 2 * B, w.slots)
    seeds = si.enc_seeds(100, 2 * B)
    # sampled inputs: the oracle's integer encoding, encrypted on both sides
    # with the same seed (bit-identical ciphertexts); the rest encoded on the GPU
    sampled = (0, 5, 31, 63, B, B + 31, B + 63)
    cts, ocs = [], {}
    for i in range(2 * B):
        if i in sampled:
            m = orc.encode(z[i], scale)
            cts.append(ctx.encrypt(ctx.pt_from_int(m, level), level, scale, seeds[i]))
            ocs[i] = orc.encrypt(orc.pt_from_int(m, level), level, scale, seeds[i])
        else:
            cts.append(ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, seeds[i]))
    yield w, ctx, orc, z, cts, ocs
    ctx.close()


def test_batched_products_sampled_vs_oracle(bench_pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc, z, cts, ocs = bench_pair
    B = w.batch
    level = len(w.q_bits) - 1
    out = [ctx.new_ct(level + 1) for _ in range(B)]
    ctx.mul_relin_batch(cts[:B], cts[B:], out, rescale=ck.RESCALE_MERGED)
    assert ctx.device_error() == 0
    for i in (0, 31, 63):
        want = orc.mul_relin_rescale(ocs[i], ocs[B + i])
        assert (out[i].level, out[i].scale) == (want.level, want.scale)
        assert np.array_equal(ctx.export_ct(out[i]), want.data), i
    for i in range(0, B, 7):
        err = np.max(np.abs(ctx.decrypt_decode(out[i]) - z[i] * z[B + i]))
        assert err < 2.0 ** -30, (i, err)


def test_hoisted_rotations_sampled_vs_oracle(bench_pair):
    w, ctx, orc, z, cts, ocs = bench_pair
    B = w.batch
    level = len(w.q_bits) - 1
    steps = list(w.rot_steps)
    outs = [ctx.new_ct(level + 1) for _ in range(B * len(steps))]
    ctx.rotate_hoisted(cts[:B], steps, outs)
    assert ctx.device_error() == 0
    for i, k in ((5, 1), (63, 1 << 14)):
        want = orc.rotate_hoisted(ocs[i], [k])[0]
        got = outs[steps.index(k) * B + i]
        assert np.array_equal(ctx.export_ct(got), want.data), (i, k)
    for j in (0, 7, 14):
        for i in (0, 40):
            got = ctx.decrypt_decode(outs[j * B + i])
            assert np.max(np.abs(got - np.roll(z[i], -steps[j]))) < 2.0 ** -25, (i, j)
