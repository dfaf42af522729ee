"""Packed wire format: every limb holds its N residues in bits(q_t) bits
(residue k at bits [k b, k b + b) of little-endian words), polynomial 0 then
polynomial 1.  The GPU packing must equal this definition written with Python
integers, unpacking must invert it, and the host-streamed multiply on packed
buffers must return exactly the packed device-batch products."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _pack_ref(limbs, moduli):
    """The definition: [2][l+1][N] uint64 residues -> bytes."""
    out = bytearray()
    for poly in limbs:
        for t, limb in enumerate(poly):
            b = int(moduli[t]).bit_length()
            big = 0
            for k, v in enumerate(limb.tolist()):
                big |= int(v) << (k * b)
            out += big.to_bytes(len(limb) * b // 8, "little")
    return np.frombuffer(bytes(out), dtype=np.uint8)


def _ctx(w):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    ctx.keygen(3)
    return ctx


@pytest.mark.parametrize("name", ["toy", "small"])
def test_pack_matches_definition_and_round_trips(name):
    w = {"toy": si.TOY, "small": si.SMALL}[name]
    ctx = _ctx(w)
    try:
        scale = 2.0 ** w.log2_scale
        for level in (len(w.q_bits) - 1, 0):
            z = si.messages(50 + level, 1, w.slots)[0]
            ct = ctx.encrypt(ctx.encode(z, level, scale), level, scale, 5)
            raw = ctx.export_ct(ct)
            got = ctx.export_packed(ct)
            assert got.size == ctx.wire_bytes(level)
            assert np.array_equal(got, _pack_ref(raw, ctx.moduli))
            back = ctx.import_packed(got.view(np.uint64), level, scale)
            assert np.array_equal(ctx.export_ct(back), raw)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


@pytest.mark.parametrize("name,pairs,chunk", [("small", 5, 2), ("plain", 12, 4)])
def test_packed_host_products_equal_device_batch(name, pairs, chunk):
    import torch
    import paper_2506_19693_gb300 as ck
    w = {"small": si.SMALL, "plain": si.PLAIN}[name]
    ctx = _ctx(w)
    try:
        ctx.set_form(True)
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(60, 2 * pairs, w.slots)
        cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 100 + i) for i in range(2 * pairs)]
        want = [ctx.new_ct(level + 1) for _ in range(pairs)]
        ctx.mul_relin_batch(cts[:pairs], cts[pairs:], want, rescale=ck.RESCALE_MERGED)
        wi, wo = ctx.wire_bytes(level), ctx.wire_bytes(level - 1)
        ha = torch.empty(pairs * wi, dtype=torch.uint8, pin_memory=True)
        hb = torch.empty(pairs * wi, dtype=torch.uint8, pin_memory=True)
        ho = torch.zeros(pairs * wo, dtype=torch.uint8, pin_memory=True)
        for i in range(pairs):
            ctx.export_packed(cts[i], ha[i * wi:(i + 1) * wi])
            ctx.export_packed(cts[pairs + i], hb[i * wi:(i + 1) * wi])
        sc = ctx.mul_relin_host_packed(ha, hb, scale, scale, level, ho, rescale=ck.RESCALE_MERGED, chunk=chunk)
        assert sc == want[0].scale
        for i in range(pairs):
            assert np.array_equal(ho[i * wo:(i + 1) * wo].numpy(), ctx.export_packed(want[i])), i
        assert ctx.device_error() == 0
    finally:
        ctx.close()
