"""The one-pass forward NTT on 8-CTA clusters (ckks_ctx_set_ntt_cluster, N = 2^16):
each limb is held whole in the cluster's distributed shared memory, so it
crosses HBM once.  It runs the two-pass transform's butterflies in the same
order, so every residue must equal the two-pass transform's and the oracle's,
for the loose (55-bit) and strict (61-bit) primes, and every key switch built on
it must be unchanged."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _random_limbs(moduli, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, q, size=n, dtype=np.uint64) for q in moduli])


def test_cluster_ntt_equals_two_pass_and_oracle():
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    ctx = ck.Context.from_workload(w)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    try:
        n_limbs = len(ctx.moduli)  # 24 q primes (61 and 55 bits) and 8 special 61-bit primes
        arr = _random_limbs(ctx.moduli, ctx.n, 21)
        # edge values: zeros, q - 1 everywhere on one limb, a single one
        arr[2] = 0
        arr[3] = np.uint64(ctx.moduli[3] - 1)
        arr[4] = 0
        arr[4][12345] = 1
        two = ck.u64_to_tensor(arr, ctx.device)
        ctx.ntt(two, 0)
        assert ctx.set_ntt_cluster(True) >= 1
        one = ck.u64_to_tensor(arr, ctx.device)
        ctx.ntt(one, 0)
        got = ck.tensor_to_u64(one)
        assert ctx.device_error() == 0
        assert np.array_equal(got, ck.tensor_to_u64(two))
        pick = [0, 1, 2, 3, 4, 23, 24, n_limbs - 1]
        want = orc.ntt(arr[pick], pick)
        assert np.array_equal(got[pick], want)
        # the inverse is untouched and still undoes it
        ctx.ntt(one, 0, inverse=True)
        assert np.array_equal(ck.tensor_to_u64(one), arr)
        # a transform starting at another modulus (the special primes alone)
        sp = ck.u64_to_tensor(arr[24:], ctx.device)
        ctx.ntt(sp, 24)
        assert np.array_equal(ck.tensor_to_u64(sp), got[24:])
    finally:
        ctx.close()


def test_cluster_ntt_rejected_off_n65536():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(si.N15)
    try:
        with pytest.raises(ck.CkksError):
            ctx.set_ntt_cluster(True)
        assert ctx.set_ntt_cluster(False) == 0
    finally:
        ctx.close()


@pytest.mark.parametrize("form", ["uint64", "tensor", "fused"])
def test_key_switches_unchanged_with_cluster_ntt(form):
    """N = 2^16, 24 + 8 primes, 8 pairs per batched launch: separate and merged
    rescale and hoisted rotations with and without the cluster transform."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    pairs = 8
    ctx = ck.Context.from_workload(w)
    try:
        ctx.set_form(form)
        ctx.keygen(1, rot_steps=[1, 1 << 14])
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(78, 2 * pairs, w.slots)
        cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 90 + i) for i in range(2 * pairs)]
        res = {}
        for on in (False, True):
            ctx.set_ntt_cluster(on)
            out = [ctx.new_ct(level + 1) for _ in range(pairs)]
            ctx.mul_relin_batch(cts[:pairs], cts[pairs:], out, rescale=ck.RESCALE_SEPARATE)
            merged = [ctx.new_ct(level + 1) for _ in range(pairs)]
            ctx.mul_relin_batch(cts[:pairs], cts[pairs:], merged, rescale=ck.RESCALE_MERGED)
            rots = [ctx.new_ct(level + 1) for _ in range(4)]
            ctx.rotate_hoisted(cts[:2], [1, 1 << 14], rots)
            res[on] = [ctx.export_ct(c) for c in out + merged + rots]
        assert ctx.device_error() == 0
        for i, (x, y) in enumerate(zip(res[False], res[True])):
            assert np.array_equal(x, y), i
        err = np.max(np.abs(ctx.decrypt_decode(merged[0]) - z[0] * z[pairs]))
        assert err < 2.0 ** -30, err
    finally:
        ctx.close()


def test_ntt_tuner_reports_and_keeps_parity():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen(2)
        assert ctx.ntt_config() == {"rows": 16, "cluster": False}
        ctx.set_ntt_cluster(True)
        assert ctx.ntt_config()["cluster"] is True
        arr = _random_limbs(ctx.moduli, ctx.n, 23)
        one = ck.u64_to_tensor(arr, ctx.device)
        ctx.ntt(one, 0)
        rows = ctx.tune_ntt(4)
        cfg = ctx.ntt_config()
        assert cfg["rows"] == rows and rows in (8, 16)
        two = ck.u64_to_tensor(arr, ctx.device)
        ctx.ntt(two, 0)
        assert torch.equal(one, two)
        assert ctx.device_error() == 0
    finally:
        ctx.close()
