"""ckks_rescale_noalloc: the rescale for callers that cannot let the library
allocate device memory (a capped or pool-managed device budget, or a path
that cannot take an allocation's implicit synchronisation).  It keeps its
workspace in a fixed array inside the library instead of the context's
growable scratch buffer, so it must give exactly the limbs ckks_rescale gives.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.  It builds its own contexts,
so it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _random_ct(ctx, level, seed):
    rng = np.random.default_rng(seed)
    arr = np.stack([np.stack([rng.integers(0, ctx.q[i], size=ctx.n, dtype=np.uint64) for i in range(level + 1)])
                    for _ in range(2)])
    return arr


# N = 2^17 leaves room for one lifted limb per pass (the chunk loop at G = 1)
@pytest.mark.parametrize("w", [si.TOY, si.PLAIN, si.N17], ids=["n4096", "n65536_L24", "n131072_g1"])
def test_rescale_noalloc_equals_rescale_on_two_calls_in_a_row(w):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    try:
        level = len(w.q_bits) - 1
        arr = _random_ct(ctx, level, 5)
        ref = ctx.import_ct(arr, level, 2.0 ** 80, n_limbs=level + 1)
        tst = ctx.import_ct(arr, level, 2.0 ** 80, n_limbs=level + 1)
        for call in range(2):  # two calls in a row reuse the same fixed workspace
            ctx.rescale(ref)
            ctx.rescale_noalloc(tst)
            assert (tst.level, tst.scale) == (ref.level, ref.scale)
            assert np.array_equal(ctx.export_ct(tst), ctx.export_ct(ref)), f"call {call}"
        # and once more on a fresh input, after the array holds earlier contents
        arr2 = _random_ct(ctx, level, 6)
        a = ctx.import_ct(arr2, level, 1.0)
        b = ctx.import_ct(arr2, level, 1.0)
        assert np.array_equal(ctx.export_ct(ctx.rescale_noalloc(a)), ctx.export_ct(ctx.rescale(b)))
    finally:
        ctx.close()


def test_rescale_noalloc_rejects_level_zero():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(si.TOY)
    try:
        ct = ctx.import_ct(_random_ct(ctx, 0, 7), 0, 1.0)
        with pytest.raises(ck.CkksError) as e:
            ctx.rescale_noalloc(ct)
        assert e.value.status == -2
    finally:
        ctx.close()
