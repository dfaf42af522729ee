"""Compressed switching keys (reading C22): b rows plus the generator state of
each digit's a row, with a regenerated inside the key inner product.  The key
values are the uncompressed keys' values, so the keys themselves, products,
rotations and bootstraps must equal the oracle's (and the uncompressed
context's) bit for bit, while the device key memory halves."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

KEY_SEED = 7
ROT = (1, 3, -1)


def _ctx(w, compressed, form=False, rot=ROT):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    ctx.set_key_compression(compressed)
    ctx.set_form(form)
    ctx.keygen(KEY_SEED, rot_steps=rot, conj=True)
    return ctx


@pytest.mark.parametrize("name", ["toy", "small", "n17"])
def test_compressed_keys_equal_oracle_keys(name):
    import oracle
    w = {"toy": si.TOY, "small": si.SMALL, "n17": si.N17}[name]
    full, comp = _ctx(w, False), _ctx(w, True)
    try:
        orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
        orc.keygen(KEY_SEED)
        orc.gen_rotation_keys([1])
        assert np.array_equal(comp.debug_key(0), orc.key_data(0))
        g = orc.galois_elt(1)
        assert np.array_equal(comp.debug_key(g), orc.key_data(g))
        # 5 keys (relinearisation, 3 rotations, conjugation) each lose their a rows;
        # the compressed key generation holds one more limb set of scratch
        half = full.n_digits * (full.n_q + full.n_p) * full.n
        diff = full.device_bytes() - comp.device_bytes()
        assert 5 * (half - 16) * 8 - (full.n_q + full.n_p) * full.n * 8 <= diff <= 5 * (half - 16) * 8
    finally:
        full.close()
        comp.close()


@pytest.mark.parametrize("form", [False, True])
def test_compressed_products_and_rotations_bit_exact(form):
    import oracle
    import paper_2506_19693_gb300 as ck
    w = si.SMALL
    ctx = _ctx(w, True, form)
    try:
        orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
        orc.keygen(KEY_SEED)
        orc.gen_rotation_keys(list(ROT))
        orc.gen_galois_key(orc.conj_elt())
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(70, 4, w.slots)
        cts, ocs = [], []
        for i in range(4):
            m = orc.encode(z[i], scale)
            cts.append(ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 700 + i))
            ocs.append(orc.encrypt(orc.pt_from_int(m, level), level, scale, 700 + i))
        out = [ctx.new_ct(level + 1) for _ in range(2)]
        ctx.mul_relin_batch(cts[:2], cts[2:], out, rescale=ck.RESCALE_MERGED)
        for i in range(2):
            want = orc.mul_relin_rescale(ocs[i], ocs[2 + i])
            assert (out[i].level, out[i].scale) == (want.level, want.scale)
            assert np.array_equal(ctx.export_ct(out[i]), want.data), i
        rot = [ctx.new_ct(level + 1) for _ in range(2 * len(ROT))]
        ctx.rotate_hoisted(cts[:2], list(ROT), rot)
        for j, k in enumerate(ROT):
            for i in range(2):
                want = orc.rotate_hoisted(ocs[i], [k])[0]
                assert np.array_equal(ctx.export_ct(rot[j * 2 + i]), want.data), (i, k)
        one = ctx.rotate(cts[3], -1)
        assert np.array_equal(ctx.export_ct(one), orc.rotate(ocs[3], -1).data)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_compressed_bootstrap_equals_uncompressed():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.BOOT_SMALL
    outs = []
    for compressed in (False, True):
        ctx = ck.Context.from_workload(w)
        try:
            ctx.set_key_compression(compressed)
            ctx.keygen_boot(1)
            ctx.boot_setup()
            delta = 2.0 ** w.log2_scale
            z = si.messages(71, 1, w.slots)[0]
            ct = ctx.encrypt(ctx.encode(z, 0, delta), 0, delta, 72)
            out = ctx.bootstrap(ct)
            assert np.max(np.abs(ctx.decrypt_decode(out) - z)) <= 2.0 ** -12
            outs.append(ctx.export_ct(out))
            assert ctx.device_error() == 0
        finally:
            ctx.close()
    assert np.array_equal(outs[0], outs[1])


def test_key_compression_after_keygen_is_refused():
    import paper_2506_19693_gb300 as ck
    ctx = _ctx(si.TOY, False)
    try:
        with pytest.raises(ck.CkksError) as e:
            ctx.set_key_compression(True)
        assert ck.STATUS[e.value.status] == "CKKS_E_STATE"
    finally:
        ctx.close()


def test_compressed_full_size_batch_equals_full_keys():
    """N = 2^16, 24 + 8 primes, dnum = 3: 16 merged products and 4 inputs x 3
    hoisted rotations with compressed keys equal the full-key context's limbs."""
    import paper_2506_19693_gb300 as ck
    w = si.PLAIN
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    res = []
    for compressed in (False, True):
        ctx = _ctx(w, compressed, form=True)
        try:
            z = si.messages(74, 32, w.slots)
            cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 740 + i) for i in range(32)]
            out = [ctx.new_ct(level + 1) for _ in range(16)]
            ctx.mul_relin_batch(cts[:16], cts[16:], out, rescale=ck.RESCALE_MERGED)
            rot = [ctx.new_ct(level + 1) for _ in range(4 * len(ROT))]
            ctx.rotate_hoisted(cts[:4], list(ROT), rot)
            assert ctx.device_error() == 0
            assert np.max(np.abs(ctx.decrypt_decode(out[5]) - z[5] * z[21])) < 2.0 ** -30
            res.append([ctx.export_ct(c) for c in out + rot])
        finally:
            ctx.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)
