"""The boundary's buffer and exchange calls, and the tensor-core kernel's
failure path, through the C ABI on the GPU.

* ckks_ct_alloc / ckks_ct_free: a library-owned ciphertext buffer that the
  other calls accept like a caller-owned one;
* ckks_ct_export / ckks_ct_import: coefficient-domain host copies, equal to
  the oracle's inverse NTT of the NTT-domain limbs, and a bit-exact round trip;
* the bounded mbarrier wait of the tensor-core conversion made to run out
  (before any matrix multiply is issued): the status reads CKKS_E_TIMEOUT,
  and the next conversion on the same context is bit-exact again."""
import ctypes

import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.SMALL
    ctx = ck.Context.from_workload(w)
    ctx.keygen(3)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    orc.keygen(3)
    yield w, ctx, orc
    ctx.close()


def test_alloc_encrypt_export_free(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    m = orc.encode(si.messages(3, 1, w.slots)[0], scale)
    h = ctx.ct_alloc(level + 1)
    try:
        assert h.data and h.n_limbs == level + 1 and h.level == level and h.is_ntt == 1
        assert not ctx.export_coeff(h).any()  # zero-filled
        pt = ctx.pt_from_int(m, level)
        assert ctx.lib.ckks_encrypt(ctx._h, ctypes.c_void_p(pt.data_ptr()), level, scale, 77, ctypes.byref(h)) == 0
        want = orc.encrypt(orc.pt_from_int(m, level), level, scale, 77)
        ntt = np.zeros((2, level + 1, ctx.n), dtype=np.uint64)
        assert ctx.lib.ckks_ct_export_ntt(ctx._h, ctypes.byref(h), ntt.ctypes.data) == 0
        assert np.array_equal(ntt, want.data)
        coeff = ctx.export_coeff(h)
        mods = list(range(level + 1))
        for p in range(2):
            assert np.array_equal(coeff[p], orc.intt(want.data[p], mods))
        # the library-owned buffer works as an operand of the other calls
        out = ctx.new_ct(level + 1)
        hh = (ck.CkksCt * 1)(h)
        ho = ctx._handles([out])
        assert ctx.lib.ckks_mul_int_batch(ctx._h, hh, 3, ho, 1) == 0
        out.level, out.scale = ho[0].level, ho[0].scale
        assert np.array_equal(ctx.export_ct(out), orc.mul_int(want, 3).data)
    finally:
        ctx.ct_free(h)
    assert not h.data
    ctx.ct_free(h)  # freeing an emptied handle is a no-op


def test_coefficient_domain_import_round_trip(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    level = 3
    rng = np.random.default_rng(8)
    arr = np.stack([np.stack([rng.integers(0, ctx.q[t], size=ctx.n, dtype=np.uint64) for t in range(level + 1)])
                    for _ in range(2)])
    ct = ctx.new_ct(level + 2, level, 1.0)
    ctx.import_coeff(arr, ct)
    mods = list(range(level + 1))
    for p in range(2):
        assert np.array_equal(ctx.export_ct(ct)[p], orc.ntt(arr[p], mods))
    assert np.array_equal(ctx.export_coeff(ct), arr)
    bad = arr.copy()
    bad[1, 2, 5] = np.uint64(ctx.q[2])  # not a residue: refused before any copy
    with pytest.raises(ck.CkksError) as e:
        ctx.import_coeff(bad, ct)
    assert e.value.status == -1
    assert np.array_equal(ctx.export_coeff(ct), arr)


def test_tensor_core_wait_expiry_is_reported_and_recovered(pair):
    import paper_2506_19693_gb300 as ck
    w, ctx, orc = pair
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    z = si.messages(4, 2, w.slots)
    a, b = (ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 90 + i) for i in range(2))
    ref = [ctx.new_ct(level + 1)]
    ctx.mul_relin_batch([a], [b], ref, rescale=ck.RESCALE_MERGED)  # uint64 form
    assert ctx.device_error() == 0
    ctx.debug_tc_expire(2_000_000)  # the wait gives up after 2 ms
    assert ctx.device_error() == -7  # CKKS_E_TIMEOUT, flag cleared by the read
    assert ctx.device_error() == 0
    ctx.set_form(True)
    try:
        out = [ctx.new_ct(level + 1)]
        ctx.mul_relin_batch([a], [b], out, rescale=ck.RESCALE_MERGED)
        assert ctx.device_error() == 0
        assert np.array_equal(ctx.export_ct(out[0]), ctx.export_ct(ref[0]))
    finally:
        ctx.set_form(False)
