"""The tensor-core NTT stage prototype (ckks_ntt_tc): the forward transform's
first four column stages as one exact byte-split GEMM on tcgen05 per limb
(16 x 16 block matrix over Z_q), the other stages on the CUDA cores.  Every
residue must equal the uint64 transform's (ckks_ntt) and the oracle's."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _random_limbs(ctx, n_polys, n_limbs, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([rng.integers(0, ctx.moduli[t], size=ctx.n, dtype=np.uint64)
                               for t in range(n_limbs)]) for _ in range(n_polys)])


@pytest.mark.parametrize("w", [si.N15, si.PLAIN], ids=["n32768", "n65536_L24"])
def test_tensor_stage_ntt_equals_uint64_ntt(w):
    import torch
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    ctx = ck.Context.from_workload(w)
    try:
        n_limbs = len(ctx.moduli)  # every q and p modulus: 55- and 61-bit primes
        n_polys = 3
        arr = _random_limbs(ctx, n_polys, n_limbs, 11)
        t = ck.u64_to_tensor(arr.reshape(n_polys * n_limbs, ctx.n), ctx.device)
        ctx.ntt_tc(t, n_polys, n_limbs)
        got = ck.tensor_to_u64(t).reshape(n_polys, n_limbs, ctx.n)
        assert ctx.device_error() == 0
        for p in range(n_polys):
            ref = ck.u64_to_tensor(arr[p], ctx.device)
            ctx.ntt(ref, 0)
            assert np.array_equal(got[p], ck.tensor_to_u64(ref)), p
    finally:
        ctx.close()


def test_tensor_stage_ntt_matches_oracle():
    import torch
    import oracle
    import paper_2506_19693_gb300 as ck
    torch.cuda.set_device(0)
    w = si.N15
    ctx = ck.Context.from_workload(w)
    orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    try:
        n_limbs = len(ctx.moduli)
        arr = _random_limbs(ctx, 1, n_limbs, 12)
        t = ck.u64_to_tensor(arr[0], ctx.device)
        ctx.ntt_tc(t, 1, n_limbs)
        assert np.array_equal(ck.tensor_to_u64(t), orc.ntt(arr[0], list(range(n_limbs))))
    finally:
        ctx.close()
