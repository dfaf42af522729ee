import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


@pytest.fixture(scope="session")
def toy_oracle():
    from oracle import Oracle
    import synthetic_inputs as si
    w = si.TOY
    o = Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    o.keygen(7)
    o.gen_rotation_keys([1, 2, 3, -1, 5, o.n // 4])
    o.gen_galois_key(o.conj_elt())
    return o


@pytest.fixture(scope="session")
def tiny_oracle():
    """N = 2^5 ring with four q-primes, two special primes and two digits:
    small enough for big-integer brute force."""
    from oracle import Oracle
    o = Oracle(5, (50, 45, 45, 45), (55, 55), 2, h=8, sigma=3.2)
    o.keygen(3)
    o.gen_rotation_keys([1, 3])
    return o
