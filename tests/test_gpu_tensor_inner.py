"""The key-switch inner product as a byte-split tensor-core GEMM (ckks_ks_inner_tc)
against the same product on the CUDA cores (ckks_ks_inner_u64) and against its
definition, out[p][o][t][k] = sum_j d[p][j][t][k] key[j][o][t][k] mod q_t, by
Python integers on sampled entries.  Inputs are uniform residues, with the
largest residue q - 1 and zero planted in some coefficients."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

P = 128


def _inputs(ctx, torch, ndig, L, seed):
    g = torch.Generator(device=ctx.device)
    g.manual_seed(seed)
    n = ctx.n
    d = torch.empty((P, ndig, L, n), dtype=torch.int64, device=ctx.device)
    key = torch.empty((ndig, 2, L, n), dtype=torch.int64, device=ctx.device)
    for t in range(L):
        q = int(ctx.moduli[t])
        d[:, :, t] = torch.randint(0, q, (P, ndig, n), device=ctx.device, generator=g)
        key[:, :, t] = torch.randint(0, q, (ndig, 2, n), device=ctx.device, generator=g)
        d[:3, :, t, :5] = q - 1      # the largest products
        key[:, :, t, :3] = q - 1
        d[5, :, t, 7] = 0
    return d, key


def _check_definition(ctx, d, key, out, L, ndig, seed, count=96):
    rng = np.random.default_rng(seed)
    samples = [(0, 0, 0, 0), (2, 1, L - 1, 4), (5, 0, 0, 7)]
    samples += [(int(rng.integers(P)), int(rng.integers(2)), int(rng.integers(L)), int(rng.integers(ctx.n)))
                for _ in range(count)]
    for p, o, t, k in samples:
        q = int(ctx.moduli[t])
        want = sum(int(d[p, j, t, k]) * int(key[j, o, t, k]) for j in range(ndig)) % q
        assert int(out[p, o, t, k]) == want, (p, o, t, k)


@pytest.mark.parametrize("ndig", [1, 2, 3, 4])
def test_tensor_inner_product_small_ring(ndig):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.SMALL
    ctx = ck.Context.from_workload(w)
    try:
        L = len(ctx.moduli)  # 61- and 55-bit primes
        d, key = _inputs(ctx, torch, ndig, L, 3 + ndig)
        out_tc = torch.zeros((P, 2, L, ctx.n), dtype=torch.int64, device=ctx.device)
        out_u = torch.zeros_like(out_tc)
        ctx.ks_inner(d, key, out_tc, "tensor")
        ctx.ks_inner(d, key, out_u, "uint64")
        torch.cuda.synchronize()
        assert ctx.device_error() == 0
        assert torch.equal(out_tc, out_u)
        _check_definition(ctx, d.cpu(), key.cpu(), out_tc.cpu(), L, ndig, ndig)
    finally:
        ctx.close()


@pytest.mark.parametrize("L", [8, 32], ids=["n65536_L8", "n65536_L32"])
def test_tensor_inner_product_full_size(L):
    """N = 2^16, 3 digits, 128 ciphertexts; 32 limbs is every prime (24 + 8)."""
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.PLAIN
    ctx = ck.Context.from_workload(w)
    try:
        ndig = 3
        d, key = _inputs(ctx, torch, ndig, L, 11)
        out_tc = torch.zeros((P, 2, L, ctx.n), dtype=torch.int64, device=ctx.device)
        ctx.ks_inner(d, key, out_tc, "tensor")
        out_u = torch.zeros_like(out_tc)
        ctx.ks_inner(d, key, out_u, "uint64")
        torch.cuda.synchronize()
        assert ctx.device_error() == 0
        assert torch.equal(out_tc, out_u)
        _check_definition(ctx, d, key, out_tc, L, ndig, 12, count=48)
    finally:
        ctx.close()


def test_tensor_inner_product_rejects_other_batches():
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(si.SMALL)
    try:
        n = ctx.n
        d = torch.zeros((64, 3, 4, n), dtype=torch.int64, device=ctx.device)
        key = torch.zeros((3, 2, 4, n), dtype=torch.int64, device=ctx.device)
        out = torch.zeros((64, 2, 4, n), dtype=torch.int64, device=ctx.device)
        with pytest.raises(ck.CkksError):
            ctx.ks_inner(d, key, out, "tensor")  # the MMA rows are 128 ciphertexts
        ctx.ks_inner(d, key, out, "uint64")
        d5 = torch.zeros((P, 5, 4, n), dtype=torch.int64, device=ctx.device)
        with pytest.raises(ck.CkksError):
            ctx.ks_inner(d5, key, out, "uint64")
    finally:
        ctx.close()
