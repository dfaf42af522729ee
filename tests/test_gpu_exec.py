"""Uneven batches: operations on ciphertexts of two ring degrees and many
levels run through the grouped executor and through a captured CUDA graph
must give exactly the limbs of the same operations issued one by one (which
the parity tests tie to the oracle); the autotuner must not change results."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctxs = []
    for w in (si.SMALL, si.MID):
        c = ck.Context.from_workload(w)
        c.keygen(3, rot_steps=[1, 2, 4, 8, -1])
        ctxs.append((w, c))
    return ctxs


def _batch(ctxs, n_ops, seed):
    import paper_2506_19693_gb300 as ck
    rng = np.random.default_rng(seed)
    ops, refs = [], []
    for i in range(n_ops):
        w, c = ctxs[rng.integers(0, len(ctxs))]
        top = len(w.q_bits) - 1
        level = int(rng.integers(1, top + 1))
        scale = 2.0 ** w.log2_scale
        z = si.messages(seed * 1000 + i, 2, w.slots)
        a = c.encrypt(c.encode(z[0], level, scale), level, scale, 7000 + i)
        kind = int(rng.integers(0, 3))
        out = c.new_ct(level + 1)
        if kind == 0:
            b = c.encrypt(c.encode(z[1], level, scale), level, scale, 8000 + i)
            ops.append(ck.Op(c, ck.OP_MUL_RELIN, a, out, b=b, rescale=True))
            refs.append((c, lambda c=c, a=a, b=b: c.rescale(c.mul_relin(a, b))))
        elif kind == 1:
            k = int(rng.choice([1, 2, 4, 8, -1]))
            ops.append(ck.Op(c, ck.OP_ROTATE, a, out, k=k))
            refs.append((c, lambda c=c, a=a, k=k: c.rotate(a, k)))
        else:
            ops.append(ck.Op(c, ck.OP_RESCALE, a, out))
            refs.append((c, lambda c=c, a=a: c.rescale(c.mul_int(a, 1))))
    return ops, refs


def _check(ops, refs):
    for op, (c, f) in zip(ops, refs):
        want = f()
        assert (op.out.level, op.out.scale) == (want.level, want.scale)
        assert np.array_equal(c.export_ct(op.out), c.export_ct(want))


def test_executor_graph_and_tuner_match_single_calls():
    import torch
    import paper_2506_19693_gb300 as ck
    ctxs = _setup()
    try:
        ops, refs = _batch(ctxs, 30, 1)
        ck.execute(ops)
        _check(ops, refs)
        for op in ops:
            op.out.data.fill_(-1)
        g = ck.Graph(ops)
        for op in ops:
            op.out.data.fill_(0)
        g.launch()
        g.launch()  # replays are idempotent: inputs are never written
        torch.cuda.synchronize()
        _check(ops, refs)
        g.close()
        for w, c in ctxs:
            assert c.tune(len(w.q_bits) - 1, 4) in (2, 4, 8, 16, 32)
        for op in ops:
            op.out.data.fill_(0)
        ck.execute(ops)
        _check(ops, refs)
    finally:
        for _, c in ctxs:
            c.close()


def test_executor_rejects_aliasing_and_bad_ops():
    import paper_2506_19693_gb300 as ck
    ctxs = _setup()
    try:
        w, c = ctxs[0]
        lvl = len(w.q_bits) - 1
        a = c.encrypt(c.encode(si.messages(9, 1, w.slots)[0], lvl, 2.0 ** 55), lvl, 2.0 ** 55, 1)
        with pytest.raises(ck.CkksError):
            ck.execute([ck.Op(c, ck.OP_ROTATE, a, a, k=1)])
        with pytest.raises(ck.CkksError):
            ck.execute([ck.Op(c, 99, a, c.new_ct(lvl + 1))])
    finally:
        for _, c in ctxs:
            c.close()


def test_ntt_row_tiles_agree_and_tuner_picks_one():
    """Both NTT row-pass tiles (16 and 8 rows per CTA) give the same limbs; the
    tuner keeps one of them."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.MID
    ctx = ck.Context.from_workload(w)
    try:
        ctx.keygen(2)
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(70, 4, w.slots)
        cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 70 + i) for i in range(4)]
        outs = {}
        for rows in (16, 8):
            ctx.set_ntt_rows(rows)
            out = [ctx.new_ct(level + 1) for _ in range(2)]
            ctx.mul_relin_batch(cts[:2], cts[2:], out, rescale=ck.RESCALE_MERGED)
            outs[rows] = [ctx.export_ct(o) for o in out]
        for x, y in zip(outs[16], outs[8]):
            assert np.array_equal(x, y)
        assert ctx.tune_ntt(8) in (8, 16)
    finally:
        ctx.close()


def test_dnum_tuner_times_every_fitting_candidate():
    import math
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    best, ms = ck.tune_dnum(si.SMALL, cands=(1, 2, 3), batch=4)
    # n_q = 6: dnum 1 -> alpha 6, 2 -> 3, 3 -> 2 special primes; all fit 16 sources
    assert best in (1, 2, 3)
    assert all(math.isfinite(v) and v > 0 for v in ms.values())
    best, ms = ck.tune_dnum(si.PLAIN, cands=(1, 3), batch=2)
    assert best == 3 and math.isinf(ms[1])  # alpha 24 does not fit a 16-source conversion
