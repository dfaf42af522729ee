"""ckks_mul_relin_host: pairs in page-locked host memory streamed through the
GPU in chunks (copies overlapping compute) give, bit for bit, the products
of the device-resident batched call, for every rescale mode, a ragged last
chunk and staging slots reused more than once."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _host(cts, level, torch):
    n = cts[0].data.shape[-1]
    h = torch.empty((len(cts), 2, level + 1, n), dtype=torch.int64, pin_memory=True)
    for i, c in enumerate(cts):
        h[i].copy_(c.data[:, : level + 1])
    return h


@pytest.mark.parametrize("w,pairs,chunk", [(si.SMALL, 5, 2), (si.PLAIN, 7, 3)], ids=["n4096", "n65536"])
@pytest.mark.parametrize("mode", [0, 1, 2], ids=["none", "separate", "merged"])
def test_host_streamed_products_equal_device_batch(w, pairs, chunk, mode):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    try:
        ctx.set_form(True)
        ctx.keygen(4)
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(50, 2 * pairs, w.slots)
        cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 300 + i) for i in range(2 * pairs)]
        a, b = cts[:pairs], cts[pairs:]
        ref = [ctx.new_ct(level + 1) for _ in range(pairs)]
        ctx.mul_relin_batch(a, b, ref, rescale=mode)
        out_level = level - (1 if mode else 0)
        host_out = torch.zeros((pairs, 2, out_level + 1, ctx.n), dtype=torch.int64, pin_memory=True)
        sc = ctx.mul_relin_host(_host(a, level, torch), _host(b, level, torch), scale, scale, level, host_out,
                                rescale=mode, chunk=chunk)
        assert sc == ref[0].scale
        for i in range(pairs):
            assert ref[i].level == out_level
            assert np.array_equal(host_out[i].numpy().view(np.uint64), ctx.export_ct(ref[i]))
        assert ctx.device_error() == 0
    finally:
        ctx.close()
