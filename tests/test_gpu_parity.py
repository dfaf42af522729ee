"""GPU parity: every C-ABI call against the CPU oracle on identical seeded
inputs.  Integer work (limbs, keys, transforms) must match bit for bit;
FP64 encode/decode within the bounds derived in the design notes."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

KEY_SEED = 7
ROT_STEPS = (1, 2, 3, -1, 5)


def _pair(w, rot=ROT_STEPS, conj=True):
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    ctx.keygen(KEY_SEED, rot_steps=rot, conj=conj)
    orc.keygen(KEY_SEED)
    orc.gen_rotation_keys(rot)
    if conj:
        orc.gen_galois_key(orc.conj_elt())
    return ctx, orc


@pytest.fixture(scope="module", params=["toy", "small", "mid", "n15", "n17", "smallq", "bigq"])
def pair(request):
    w = {"toy": si.TOY, "small": si.SMALL, "mid": si.MID, "n15": si.N15, "n17": si.N17,
         "smallq": si.SMALLQ, "bigq": si.BIGQ}[request.param]
    ctx, orc = _pair(w)
    yield w, ctx, orc
    ctx.close()


def _enc_both(w, ctx, orc, seed, level=None, count=1):
    level = len(w.q_bits) - 1 if level is None else level
    scale = 2.0 ** w.log2_scale
    z = si.messages(seed, count, w.slots)
    out = []
    for i in range(count):
        m = orc.encode(z[i], scale)
        co = orc.encrypt(orc.pt_from_int(m, level), level, scale, 1000 * seed + i)
        cg = ctx.encrypt(ctx.pt_from_int(m, level), level, scale, 1000 * seed + i)
        out.append((z[i], cg, co))
    return out


def _noise_bound(w):
    """Slot-error bound for a fresh or once key-switched ciphertext: 2^-20 at
    scales of 2^40 and above; at a smaller scale the same noise, about 2^20
    below the scale at these ring sizes, is a larger fraction of the message."""
    return 2.0 ** -min(20.0, w.log2_scale - 20.0)


def _same(ctx, cg, co):
    assert cg.level == co.level
    assert cg.scale == co.scale
    got = ctx.export_ct(cg)
    if not np.array_equal(got, co.data):
        bad = np.argwhere(got != co.data)
        raise AssertionError(f"{len(bad)} limbs words differ, first at {bad[0].tolist()}")


def test_prime_chain_and_roots_match(pair):
    w, ctx, orc = pair
    assert ctx.moduli == orc.moduli
    assert ctx.psi == orc.psi
    assert (ctx.n_digits, ctx.alpha) == (orc.n_digits, orc.alpha)


def test_ntt_forward_inverse_bit_exact(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    rng = np.random.default_rng(1)
    nm = len(ctx.moduli)
    a = np.stack([rng.integers(0, m, size=ctx.n, dtype=np.uint64) for m in ctx.moduli])
    t = ck.u64_to_tensor(a, ctx.device)
    ctx.ntt(t, 0)
    want = orc.ntt(a, list(range(nm)))
    assert np.array_equal(ck.tensor_to_u64(t), want)
    ctx.ntt(t, 0, inverse=True)
    assert np.array_equal(ck.tensor_to_u64(t), a)


def test_secret_and_keys_bit_exact(pair):
    w, ctx, orc = pair
    assert np.array_equal(ctx.debug_secret().astype(np.int64), orc.secret())
    assert np.array_equal(ctx.debug_key(0), orc.key_data(0))
    g = orc.galois_elt(1)
    assert np.array_equal(ctx.debug_key(g), orc.key_data(g))


def test_encrypt_decrypt_bit_exact(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    for lvl in (len(w.q_bits) - 1, 0):
        (z, cg, co), = _enc_both(w, ctx, orc, 3, level=lvl)
        _same(ctx, cg, co)
        assert np.array_equal(ck.tensor_to_u64(ctx.decrypt(cg)), orc.decrypt(co))


def test_elementwise_ops_bit_exact(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    (za, a, ao), (zb, b, bo) = _enc_both(w, ctx, orc, 4, count=2)
    _same(ctx, ctx.add(a, b), orc.add(ao, bo))
    _same(ctx, ctx.sub(a, b), orc.sub(ao, bo))
    _same(ctx, ctx.mul_int(a, -3), orc.mul_int(ao, -3))
    level = a.level
    m = orc.encode(zb, 2.0 ** 30)
    pt_o = orc.pt_from_int(m, level)
    pt_g = ctx.pt_from_int(m, level)
    assert np.array_equal(ck.tensor_to_u64(pt_g), pt_o)
    _same(ctx, ctx.mul_plain(a, pt_g, 2.0 ** 30), orc.mul_plain(ao, pt_o, 2.0 ** 30))
    _same(ctx, ctx.add_plain(a, pt_g), orc.add_plain(ao, pt_o))


def test_mul_relin_and_rescale_bit_exact(pair):
    w, ctx, orc = pair
    (za, a, ao), (zb, b, bo) = _enc_both(w, ctx, orc, 5, count=2)
    pg, po = ctx.mul_relin(a, b), orc.mul_relin(ao, bo)
    _same(ctx, pg, po)
    ctx.rescale(pg)
    po = orc.rescale(po)
    _same(ctx, pg, po)
    # a second product at the lower level exercises the partial top digit
    pg2 = ctx.rescale(ctx.mul_relin(pg, pg))
    po2 = orc.rescale(orc.mul_relin(po, po))
    _same(ctx, pg2, po2)


@pytest.mark.parametrize("tensor_form", ["uint64", "tensor", "fused"])
def test_merged_moddown_rescale_bit_exact(pair, tensor_form):
    """Reading C21 (ModDown and rescale in one conversion) against the oracle,
    at the top level and again one level down (partial top digit)."""
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    ctx.set_form(tensor_form)
    try:
        (za, a, ao), (zb, b, bo) = _enc_both(w, ctx, orc, 6, count=2)
        out = [ctx.new_ct(a.level + 1) for _ in range(2)]
        ctx.mul_relin_batch([a, b], [b, a], out, rescale=ck.RESCALE_MERGED)
        po = orc.mul_relin_rescale(ao, bo)
        _same(ctx, out[0], po)
        _same(ctx, out[1], orc.mul_relin_rescale(bo, ao))
        out2 = [ctx.new_ct(out[0].level + 1)]
        ctx.mul_relin_batch([out[0]], [out[1]], out2, rescale=ck.RESCALE_MERGED)
        _same(ctx, out2[0], orc.mul_relin_rescale(po, orc.mul_relin_rescale(bo, ao)))
        assert ctx.device_error() == 0
    finally:
        ctx.set_form(False)


def test_rotations_and_conjugation_bit_exact(pair):
    w, ctx, orc = pair
    (z, a, ao), = _enc_both(w, ctx, orc, 6)
    for k in ROT_STEPS:
        _same(ctx, ctx.rotate(a, k), orc.rotate(ao, k))
    _same(ctx, ctx.conjugate(a), orc.conjugate(ao))
    # at a lower level (fewer digits)
    low = ctx.rescale(ctx.mul_int(a, 1))
    lowo = orc.rescale(orc.mul_int(ao, 1))
    _same(ctx, ctx.rotate(low, 2), orc.rotate(lowo, 2))


def test_batched_calls_equal_single_calls(pair):
    w, ctx, orc = pair
    items = _enc_both(w, ctx, orc, 8, count=4)
    a = [it[1] for it in items[:2]]
    b = [it[1] for it in items[2:]]
    out = [ctx.new_ct(a[0].level + 1) for _ in range(2)]
    ctx.mul_relin_batch(a, b, out, rescale=True)
    for i in range(2):
        want = orc.rescale(orc.mul_relin(items[i][2], items[2 + i][2]))
        _same(ctx, out[i], want)
    rots = [ctx.new_ct(a[0].level + 1) for _ in range(2)]
    ctx.rotate_batch(a, [1, -1], rots)
    _same(ctx, rots[0], orc.rotate(items[0][2], 1))
    _same(ctx, rots[1], orc.rotate(items[1][2], -1))


def test_hoisted_rotations_bit_exact(pair):
    w, ctx, orc = pair
    (za, a, ao), (zb, b, bo) = _enc_both(w, ctx, orc, 13, count=2)
    steps = [1, 2, -1]
    outs = [ctx.new_ct(a.level + 1) for _ in range(2 * len(steps))]
    ctx.rotate_hoisted([a, b], steps, outs)
    for i, co in enumerate((ao, bo)):
        want = orc.rotate_hoisted(co, steps)
        for j in range(len(steps)):
            _same(ctx, outs[j * 2 + i], want[j])
    got = ctx.decrypt_decode(outs[0])
    assert np.max(np.abs(got - np.roll(za, -1))) < _noise_bound(w)


def test_public_key_and_public_key_encryption_bit_exact(pair):
    """Reading C5, pk form: the public key and Enc_pk at the top level and at
    level 0 equal the oracle's limb for limb, and decrypt to the message."""
    w, ctx, orc = pair
    ctx.keygen_public()
    orc.gen_public_key()
    assert np.array_equal(ctx.public_key(), orc.public_key())
    scale = 2.0 ** w.log2_scale
    z = si.messages(15, 1, w.slots)[0]
    m = orc.encode(z, scale)
    for lvl in (len(w.q_bits) - 1, 0):
        cg = ctx.encrypt_pk(ctx.pt_from_int(m, lvl), lvl, scale, 555 + lvl)
        co = orc.encrypt_pk(orc.pt_from_int(m, lvl), lvl, scale, 555 + lvl)
        _same(ctx, cg, co)
    # the mask multiplies the key's error: about sqrt(N/2) sigma per coefficient
    got = ctx.decrypt_decode(ctx.encrypt_pk(ctx.pt_from_int(m, len(w.q_bits) - 1), len(w.q_bits) - 1, scale, 9))
    assert np.max(np.abs(got - z)) < 2.0 ** 6 * _noise_bound(w)
    assert ctx.device_error() == 0


def test_public_key_statuses():
    import paper_2506_19693_gb300 as ck
    ctx, orc = _pair(si.TOY, rot=(1,), conj=False)
    try:
        level = len(si.TOY.q_bits) - 1
        pt = ctx.pt_from_int(np.zeros(ctx.n, dtype=np.int64), level)
        with pytest.raises(ck.CkksError):
            ctx.encrypt_pk(pt, level, 1.0, 1)
        with pytest.raises(ck.CkksError):
            ctx.public_key()
        ctx.keygen_public()
        ctx.encrypt_pk(pt, level, 1.0, 1)
        ctx.keygen(KEY_SEED, rot_steps=[1])  # a new secret discards the public key
        with pytest.raises(ck.CkksError):
            ctx.encrypt_pk(pt, level, 1.0, 1)
    finally:
        ctx.close()


def test_encode_matches_oracle_within_fp64_rounding(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    scale = 2.0 ** w.log2_scale
    z = si.messages(9, 1, w.slots)[0]
    level = len(w.q_bits) - 1
    pt = ctx.encode(z, level, scale)
    ctx.ntt(pt, 0, inverse=True)
    got = ck.tensor_to_u64(pt)
    want = orc.encode(z, scale)
    q0 = orc.q[0]
    # |m| < q0 / 2 here, so limb 0 determines the integer coefficient
    m_gpu = np.array([int(v) if v <= q0 // 2 else int(v) - q0 for v in got[0]], dtype=object)
    diff = np.array([int(a) - int(b) for a, b in zip(m_gpu, want)], dtype=np.float64)
    # two FP64 length-N FFTs of inputs |z| <= sqrt(2): each output's error is
    # below log2(N) * 2^-52 * sqrt(2) * N/2 * scale / N, plus 1 for rounding.
    bound = w.log_n * 2.0 ** -52 * scale + 1
    assert np.max(np.abs(diff)) <= bound, (np.max(np.abs(diff)), bound)
    for l in range(1, level + 1):
        ql = orc.q[l]
        assert [int(x) for x in got[l]] == [int(v) % ql for v in m_gpu]


def test_decode_matches_oracle(pair):
    w, ctx, orc = pair
    (z, a, ao), = _enc_both(w, ctx, orc, 10)
    got = ctx.decrypt_decode(a)
    want = orc.decrypt_decode(ao)
    assert np.max(np.abs(got - want)) <= 2.0 ** -40 * 8
    assert np.max(np.abs(got - z)) < _noise_bound(w)


def test_toy_mult_error_bound():
    ctx, orc = _pair(si.TOY, rot=(1,), conj=False)
    try:
        (za, a, ao), (zb, b, bo) = _enc_both(si.TOY, ctx, orc, 11, count=2)
        p = ctx.rescale(ctx.mul_relin(a, b))
        err = np.max(np.abs(ctx.decrypt_decode(p) - za * zb))
        assert err <= 2.0 ** -25, err
    finally:
        ctx.close()


def test_error_statuses():
    import paper_2506_19693_gb300 as ck
    ctx, orc = _pair(si.TOY, rot=(1,), conj=False)
    try:
        (za, a, ao), (zb, b, bo) = _enc_both(si.TOY, ctx, orc, 12, count=2)
        low = ctx.rescale(ctx.mul_int(a, 1))
        with pytest.raises(ck.CkksError) as e:
            ctx.add(low, b)
        assert e.value.status == -2
        with pytest.raises(ck.CkksError) as e:
            ctx.rotate(a, 7)
        assert e.value.status == -4
        zero = ctx.rescale(ctx.rescale(ctx.mul_int(a, 1)))
        with pytest.raises(ck.CkksError) as e:
            ctx.rescale(zero)
        assert e.value.status == -2
        with pytest.raises(ck.CkksError) as e:
            ctx.encode(np.full(si.TOY.slots, 1e3), 0, 2.0 ** 60)  # m_0 = 1e3 * 2^60 > 2^62
        assert e.value.status == -3
    finally:
        ctx.close()
