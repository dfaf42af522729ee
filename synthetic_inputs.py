"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds workload definitions (ring degree, prime bit sizes, digit
count, scale, batch size) and seeded message generators only: none of the
scheme's arithmetic lives here.  Both the CPU oracle and the CUDA library get
their messages and seeds from here; each side then draws its own secret,
errors and masks from the seed with its own implementation of the
counter-based SplitMix64 generator.

The paper's datasets (MNIST and the other Table 2 sets) are not available;
messages are uniform in [-1, 1] (real and imaginary parts), the distribution
the scheme's error bounds are quoted on, and the MLP inputs are uniform in
[0, 1] with 784 features per sample.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    log_n: int
    q_bits: tuple
    p_bits: tuple
    dnum: int
    log2_scale: float
    h: int = 64
    sigma: float = 3.2
    batch: int = 1
    rot_steps: tuple = field(default_factory=tuple)

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def slots(self) -> int:
        return self.n // 2


# Toy ring (not secure): N = 2^12, 2048 slots, scale 2^40.  q0 ~ 2^50 holds the
# message after the last rescale; q1, q2 ~ 2^40 match the scale so that a
# rescale returns it to ~2^40; one special prime of 51 bits (>= every q_i).
TOY = Workload("toy_n4096_q50_40_40_p51", 12, (50, 40, 40), (51,), 3, 40.0,
               batch=1, rot_steps=(1,))

# N = 2^16, 24 ciphertext primes (q0 ~ 2^61, 23 x ~2^55), 8 special primes of
# 61 bits, dnum = 3 (8 primes per digit), scale 2^55, 64 ciphertext pairs and
# rotations by every power of two up to 2^14.
PLAIN = Workload("n65536_L24_dnum3_b64", 16, (61,) + (55,) * 23, (61,) * 8, 3, 55.0,
                 batch=64, rot_steps=tuple(1 << k for k in range(15)))

# Small versions of the same shapes that the CPU oracle finishes in seconds
# while still spanning several NTT tiles and more than one digit.
SMALL = Workload("n4096_L6_dnum3", 12, (61,) + (55,) * 5, (61,) * 2, 3, 55.0,
                 batch=3, rot_steps=(1, 2, 4, -1))
MID = Workload("n8192_L8_dnum3", 13, (61,) + (55,) * 7, (61,) * 3, 3, 55.0,
               batch=2, rot_steps=(1, 8))
# Every prime below 2^32 (the smallest sizes the parameter check admits are 20
# bits; these are 31 and 28): the word-size edge of the reductions and of the
# merged rescale's overflow estimate.  Not secure; scale 2^26.
SMALLQ = Workload("n4096_q31_28x3_p31x2_dnum2", 12, (31, 28, 28, 28), (31, 31), 2, 26.0,
                  batch=2, rot_steps=(1, -1))
# The largest primes the parameter check admits (62 bits: strict forward
# butterflies, the inverse with exact quotients) mixed with 60 and 55 bits.
BIGQ = Workload("n4096_q62_60_62_55_p62x2_dnum2", 12, (62, 60, 62, 55), (62, 62), 2, 50.0,
                batch=2, rot_steps=(1, -1))
# N = 2^15, the other ring degree of the uneven batch, on a short chain of the
# same prime sizes (the primes are shared with N = 2^16: all = 1 mod 2^17)
N15 = Workload("n32768_L6_dnum3", 15, (61,) + (55,) * 5, (61,) * 2, 3, 55.0,
               batch=2, rot_steps=(1, 1 << 13))


# Bootstrapping chain (25 ciphertext primes = base + 24 levels, Table 3's l = 24):
# q0 ~ 2^60 (message ratio Delta/q0 = 2^-10), q1..q8 ~ 2^50 for the user's
# 8 levels (Table 3's tau_ReBoot = 8), q9..q11 ~ 2^50 for SlotToCoeff,
# q12..q21 ~ 2^60 for EvalMod (scale ~ q0 stays put), q22..q24 ~ 2^60 for
# CoeffToSlot; 9 special primes of 61 bits (alpha = ceil(25/3)), dnum = 3.
BOOT_Q_BITS = (60,) + (50,) * 11 + (60,) * 13
BOOT = Workload("n65536_boot_L24_dnum3_b16", 16, BOOT_Q_BITS, (61,) * 9, 3, 50.0, batch=16)
BOOT_SMALL = Workload("n4096_boot_L24_dnum3", 12, BOOT_Q_BITS, (61,) * 9, 3, 50.0, batch=2)


# N = 2^17 (Table 3's eMLP-2/3 ring): a short chain the CPU oracle handles in
# seconds (4 ciphertext primes, 2 special), and the bootstrapping chain of
# eMLP-2, l = 27 = 11 + 16: q0 ~ 2^60, q1..q14 ~ 2^50 (11 user levels plus
# SlotToCoeff), q15..q27 ~ 2^60 (EvalMod and CoeffToSlot), 10 special primes
# of 61 bits (alpha = ceil(28/3)), dnum = 3, Delta = 2^50 (Table 3's 2^59
# would need q0 >= 2^69 for the same message ratio, beyond a 64-bit word).
N17 = Workload("n131072_L4_dnum2", 17, (60,) + (55,) * 3, (61,) * 2, 2, 55.0,
               batch=2, rot_steps=(1, -1, 1 << 15))
BOOT17_Q_BITS = (60,) + (50,) * 14 + (60,) * 13
BOOT17 = Workload("n131072_boot_L27_dnum3_b8", 17, BOOT17_Q_BITS, (61,) * 10, 3, 50.0, batch=8)
# eMLP-3 (Table 3: l = 29 = 13 + 16): two more user levels on the same plan
BOOT17_L29 = Workload("n131072_boot_L29_dnum3", 17, (60,) + (50,) * 16 + (60,) * 13, (61,) * 10, 3, 50.0,
                      batch=8)


def rng(seed: int, stream: str) -> np.random.Generator:
    """An independent numpy generator per (seed, stream name)."""
    tag = int.from_bytes(stream.encode()[:8].ljust(8, b"\0"), "little")
    return np.random.default_rng([seed, tag])


def messages(seed: int, count: int, n_slots: int, real_only: bool = False) -> np.ndarray:
    """`count` vectors of `n_slots` complex slots, real and imaginary parts
    uniform in [-1, 1]."""
    g = rng(seed, "msg")
    re = g.uniform(-1.0, 1.0, size=(count, n_slots))
    if real_only:
        return re.astype(np.complex128)
    im = g.uniform(-1.0, 1.0, size=(count, n_slots))
    return re + 1j * im


def enc_seeds(seed: int, count: int) -> list[int]:
    """Per-ciphertext encryption seeds (64-bit)."""
    g = rng(seed, "encseed")
    return [int(x) for x in g.integers(0, 2 ** 63 - 1, size=count, dtype=np.int64)]
