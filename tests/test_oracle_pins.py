"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- published values, brute force on tiny rings, exact big-integer
arithmetic (Python ints, sympy), closed forms and group laws."""
import math
import os

import numpy as np
import pytest

import oracle
import synthetic_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def negacyclic_mul_int(a, b, n):
    """Schoolbook product in Z[X]/(X^n + 1) over Python integers."""
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return out


def centred(x, m):
    x %= m
    return x - m if x > m // 2 else x


# ---------------------------------------------------------------- C4
def test_splitmix64_known_answers():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for seed, idx, hexv in rows:
        assert oracle.splitmix_draw(int(seed), int(idx)) == int(hexv, 16)


def test_secret_is_ternary_with_exact_hamming_weight(toy_oracle):
    s = toy_oracle.secret()
    assert set(np.unique(s)).issubset({-1, 0, 1})
    assert int(np.count_nonzero(s)) == toy_oracle.h


def test_error_distribution_matches_rounded_gaussian(toy_oracle):
    e = np.concatenate([toy_oracle.enc_error(seed) for seed in range(8)]).astype(np.float64)
    assert np.max(np.abs(e)) <= math.floor(6 * 3.2)
    assert abs(np.mean(e)) < 0.1
    # variance of a rounded N(0, 3.2^2) is 3.2^2 + 1/12
    assert abs(np.std(e) - math.sqrt(3.2 ** 2 + 1 / 12)) < 0.1


# ---------------------------------------------------------------- C1, C2
@pytest.mark.parametrize("log_n", [16, 17])
def test_prime_chain_is_prime_ntt_friendly_and_complete(log_n):
    sympy = pytest.importorskip("sympy")
    bits = [61, 55, 55, 55, 40, 61, 61]
    primes = oracle.gen_primes(bits, log_n)
    step = 1 << max(17, log_n + 1)  # 2N divides q - 1
    assert len(set(primes)) == len(primes)
    for b, q in zip(bits, primes):
        assert sympy.isprime(q)
        assert q % step == 1
        assert q < (1 << b)
    # completeness: no skipped candidate of the scan is prime
    for b in (55, 61):
        chosen = [q for bb, q in zip(bits, primes) if bb == b]
        m = 1
        seen = []
        while len(seen) < len(chosen):
            t = (1 << b) + 1 - m * step
            if sympy.isprime(t):
                seen.append(t)
            m += 1
        assert seen == chosen


def test_psi_is_primitive_2n_root_from_smallest_nonresidue():
    sympy = pytest.importorskip("sympy")
    try:
        from sympy.functions.combinatorial.numbers import legendre_symbol
    except ImportError:
        from sympy.ntheory import legendre_symbol
    for q in oracle.gen_primes([50, 55, 61]):
        for log_n in (4, 12, 16):
            n = 1 << log_n
            psi = _oracle_psi(q, n)
            assert pow(psi, n, q) == q - 1       # order exactly 2N
            g = 2
            while legendre_symbol(g, q) != -1:
                g += 1
            assert psi == pow(g, (q - 1) // (2 * n), q)
    for q in oracle.gen_primes([55, 60], 17):  # N = 2^17 takes primes = 1 mod 2^18
        n = 1 << 17
        psi = _oracle_psi(q, n)
        assert pow(psi, n, q) == q - 1


def _oracle_psi(q, n):
    lib = oracle._load()
    return int(lib.oc_find_psi(q, n))


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("log_n", [2, 3, 5, 7])
def test_ntt_equals_brute_force_evaluation(log_n):
    o = oracle.Oracle(log_n, (50, 40), (51,), 2)
    n = o.n
    rng = np.random.default_rng(log_n)
    for mi in range(3):
        q, psi = o.moduli[mi], o.psi[mi]
        a = rng.integers(0, min(q, 2 ** 62), size=n, dtype=np.uint64) % np.uint64(q)
        got = o.ntt(a, [mi])
        al = [int(x) for x in a]
        for j in range(n):
            x = pow(psi, 2 * brv(j, log_n) + 1, q)
            want = sum(al[k] * pow(x, k, q) for k in range(n)) % q
            assert int(got[j]) == want


def test_ntt_product_is_negacyclic_convolution():
    o = oracle.Oracle(6, (55,), (61,), 1)
    n = o.n
    rng = np.random.default_rng(1)
    q = o.q[0]
    a = rng.integers(0, q, size=n, dtype=np.uint64)
    b = rng.integers(0, q, size=n, dtype=np.uint64)
    prod = o.intt((o.ntt(a, [0]) .astype(object) * o.ntt(b, [0]).astype(object) % q).astype(np.uint64), [0])
    want = [x % q for x in negacyclic_mul_int([int(x) for x in a], [int(x) for x in b], n)]
    assert [int(x) for x in prod] == want
    assert [int(x) for x in o.negacyclic_schoolbook(a, b, 0)] == want


@pytest.mark.parametrize("log_n", [4, 12])
def test_intt_inverts_ntt(log_n):
    o = oracle.Oracle(log_n, (61, 55), (61,), 2)
    rng = np.random.default_rng(2)
    a = np.stack([rng.integers(0, m, size=o.n, dtype=np.uint64) for m in o.moduli])
    mods = [0, 1, 2]
    assert np.array_equal(o.intt(o.ntt(a, mods), mods), a)


# ---------------------------------------------------------------- CRT, BConv (C8)
def test_crt_round_trip(tiny_oracle):
    o = tiny_oracle
    Q = math.prod(o.q)
    rng = np.random.default_rng(3)
    xs = [int(v) for v in rng.integers(-2 ** 62, 2 ** 62, size=o.n)]
    xs = [(v * 2 ** 120 + 12345) % Q - Q // 2 for v in xs]
    res = np.array([[x % q for x in xs] for q in o.q], dtype=np.uint64)
    assert o.crt_centred(res, o.n_q - 1) == xs


def test_bconv_is_exact_crt_plus_small_multiple_of_source_modulus(tiny_oracle):
    sympy = pytest.importorskip("sympy")
    from sympy.ntheory.modular import crt
    o = tiny_oracle
    src, dst = [1, 2, 3], [0, 4, 5]
    QD = math.prod(o.moduli[i] for i in src)
    rng = np.random.default_rng(4)
    x = np.stack([rng.integers(0, o.moduli[i], size=o.n, dtype=np.uint64) for i in src])
    y = o.bconv(x, src, dst)
    for k in range(o.n):
        exact = int(crt([o.moduli[i] for i in src], [int(x[r, k]) for r in range(3)])[0])
        # y_t = exact + u * Q_D (mod t) for one u in [0, |D|)
        us = []
        for t, mi in enumerate(dst):
            m = o.moduli[mi]
            us.append([u for u in range(len(src)) if (exact + u * QD) % m == int(y[t, k])])
        common = set(us[0]).intersection(*map(set, us[1:]))
        assert len(common) == 1


# ---------------------------------------------------------------- encoding (C3)
def test_encoding_is_the_canonical_embedding_by_brute_force():
    o = oracle.Oracle(4, (55,), (61,), 1)
    n = o.n
    z = si.messages(5, 1, n // 2)[0]
    m = o.embed_inverse(z)
    for j in range(n // 2):
        root = complex(math.cos(math.pi * pow(5, j, 2 * n) / n), math.sin(math.pi * pow(5, j, 2 * n) / n))
        val = sum(m[k] * root ** k for k in range(n))
        assert abs(val - z[j]) < 1e-12
    assert np.allclose(o.embed(m), z, atol=1e-12)


def test_encode_decode_error_bound(toy_oracle):
    o = toy_oracle
    z = si.messages(6, 1, o.n // 2)[0]
    scale = 2.0 ** 40
    m = o.encode(z, scale)
    back = o.decode_coeffs(m, scale)
    # rounding error <= 0.5 per coefficient: slot error <= N/2 / scale
    assert np.max(np.abs(back - z)) <= (o.n / 2) / scale


# ---------------------------------------------------------------- encryption (C5)
def test_decrypt_of_encrypt_is_message_plus_small_error(tiny_oracle):
    o = tiny_oracle
    n = o.n
    rng = np.random.default_rng(7)
    m = rng.integers(-2 ** 40, 2 ** 40, size=n).astype(np.int64)
    level = o.n_q - 1
    ct = o.encrypt(o.pt_from_int(m, level), level, 1.0, 99)
    s = [int(v) for v in o.secret()]
    c0 = o.crt_centred(o.intt(ct.data[0], list(range(level + 1))), level)
    c1 = o.crt_centred(o.intt(ct.data[1], list(range(level + 1))), level)
    Q = math.prod(o.q)
    dec = [centred(a + b, Q) for a, b in zip(c0, negacyclic_mul_int(c1, s, n))]
    err = [d - int(v) for d, v in zip(dec, m)]
    assert max(abs(e) for e in err) <= 19
    assert err == [int(v) for v in o.enc_error(99)]


def _centred_poly(o, res, level):
    return o.crt_centred(o.intt(res, list(range(level + 1))), level)


def test_public_key_relation_by_big_integers(tiny_oracle):
    """pk = (b, a) with b + a s = e small over Q (C5, pk form)."""
    o = tiny_oracle
    n, level = o.n, o.n_q - 1
    o.gen_public_key()
    pk = o.public_key()
    s = [int(v) for v in o.secret()]
    Q = math.prod(o.q)
    b = _centred_poly(o, pk[0], level)
    a = _centred_poly(o, pk[1], level)
    e = [centred(x + y, Q) for x, y in zip(b, negacyclic_mul_int(a, s, n))]
    assert max(abs(v) for v in e) <= 19 and any(e)
    assert max(abs(v) for v in a) > Q // 8  # a is spread over Z_Q, not small


@pytest.mark.parametrize("level", [3, 1])
def test_public_key_encryption_by_big_integers(tiny_oracle, level):
    """ct = (v b + m + e0, v a + e1) over q_0..q_level with the mask v the
    library draws, e0 and e1 small; so c0 + c1 s = m + v e + e0 + e1 s."""
    o = tiny_oracle
    n = o.n
    o.gen_public_key()
    pk = o.public_key()
    rng = np.random.default_rng(11)
    m = rng.integers(-2 ** 30, 2 ** 30, size=n).astype(np.int64)
    ct = o.encrypt_pk(o.pt_from_int(m, level), level, 1.0, 123)
    v = [int(x) for x in o.pk_mask(123)]
    assert set(v) <= {-1, 0, 1}
    Ql = math.prod(o.q[: level + 1])
    c0 = _centred_poly(o, ct.data[0], level)
    c1 = _centred_poly(o, ct.data[1], level)
    b = _centred_poly(o, np.ascontiguousarray(pk[0][: level + 1]), level)
    a = _centred_poly(o, np.ascontiguousarray(pk[1][: level + 1]), level)
    e0 = [centred(x - y - int(mm), Ql) for x, y, mm in zip(c0, negacyclic_mul_int(v, b, n), m)]
    e1 = [centred(x - y, Ql) for x, y in zip(c1, negacyclic_mul_int(v, a, n))]
    assert max(abs(x) for x in e0) <= 19 and max(abs(x) for x in e1) <= 19
    assert any(e0) and any(e1) and e0 != e1  # both errors present, from separate streams
    s = [int(x) for x in o.secret()]
    dec = [centred(x + y, Ql) for x, y in zip(c0, negacyclic_mul_int(c1, s, n))]
    noise = [d - int(mm) for d, mm in zip(dec, m)]
    assert max(abs(x) for x in noise) <= 19 * (n + 1 + 8)


def test_public_key_mask_distribution():
    """P(0) = 1/2, P(+1) = P(-1) = 1/4, within five standard deviations."""
    o = oracle.Oracle(12, (50,), (51,), 1, h=64, sigma=3.2)
    v = np.concatenate([o.pk_mask(seed) for seed in range(4)])
    n = len(v)
    for val, p in ((0, 0.5), (1, 0.25), (-1, 0.25)):
        cnt = int(np.sum(v == val))
        assert abs(cnt - p * n) <= 5 * math.sqrt(n * p * (1 - p)), (val, cnt)


def test_public_key_encryption_decodes(toy_oracle):
    o = toy_oracle
    o.gen_public_key()
    scale = 2.0 ** 40
    z = si.messages(21, 1, o.n // 2)[0]
    level = o.n_q - 1
    ct = o.encrypt_pk(o.pt_from_int(o.encode(z, scale), level), level, scale, 77)
    # noise v e + e0 + e1 s: at most a few thousand per coefficient, over 2^40
    assert np.max(np.abs(o.decrypt_decode(ct) - z)) < 2.0 ** -20


# ---------------------------------------------------------------- keys (C7)
def test_switching_key_relation_by_big_integers(tiny_oracle):
    o = tiny_oracle
    n, ext = o.n, o.n_q + o.n_p
    s = [int(v) for v in o.secret()]
    s2 = negacyclic_mul_int(s, s, n)
    key = o.key_data(0)
    P = math.prod(o.p)
    for j in range(o.n_digits):
        lo, hi = j * o.alpha, min((j + 1) * o.alpha, o.n_q)
        errs = []
        for t in range(ext):
            m = o.moduli[t]
            b = [int(v) for v in o.intt(key[j, 0, t], [t])]
            a = [int(v) for v in o.intt(key[j, 1, t], [t])]
            as_ = negacyclic_mul_int(a, s, n)
            gadget = 1 if lo <= t < hi else 0
            errs.append([centred(bb + x - gadget * P * y, m) for bb, x, y in zip(b, as_, s2)])
        assert all(abs(v) <= 19 for v in errs[0])
        assert all(e == errs[0] for e in errs)        # one small integer error over all limbs


@pytest.mark.parametrize("level", [3, 2, 1, 0])
def test_keyswitch_decrypts_to_product_with_new_secret(tiny_oracle, level):
    o = tiny_oracle
    n = o.n
    rng = np.random.default_rng(10 + level)
    d = np.stack([rng.integers(0, o.q[i], size=n, dtype=np.uint64) for i in range(level + 1)])
    u0, u1 = o.keyswitch(d, level, 0)
    mods = list(range(level + 1))
    Ql = math.prod(o.q[: level + 1])
    s = [int(v) for v in o.secret()]
    s2 = negacyclic_mul_int(s, s, n)
    dc = o.crt_centred(o.intt(d, mods), level)
    a0 = o.crt_centred(o.intt(u0, mods), level)
    a1 = o.crt_centred(o.intt(u1, mods), level)
    lhs = [x + y for x, y in zip(a0, negacyclic_mul_int(a1, s, n))]
    rhs = negacyclic_mul_int(dc, s2, n)
    noise = [centred(x - y, Ql) for x, y in zip(lhs, rhs)]
    # |noise| <= sum_j |digit_j| * |e_j| * N / P + rounding: far below Q_l
    assert max(abs(v) for v in noise) < 2 ** 20


# ---------------------------------------------------------------- rescale (C10)
def test_rescale_is_exact_rounded_division(tiny_oracle):
    o = tiny_oracle
    level = o.n_q - 1
    rng = np.random.default_rng(12)
    data = np.stack([np.stack([rng.integers(0, o.q[i], size=o.n, dtype=np.uint64)
                               for i in range(level + 1)]) for _ in range(2)])
    ct = oracle.OCt(data, level, 2.0 ** 90)
    out = o.rescale(ct)
    ql = o.q[level]
    Qlow = math.prod(o.q[:level])
    for pol in range(2):
        c = o.crt_centred(o.intt(data[pol], list(range(level + 1))), level)
        want = [(x + ql // 2) // ql if x >= 0 else -((-x + ql // 2) // ql) for x in c]
        got = o.crt_centred(o.intt(out.data[pol], list(range(level))), level - 1)
        assert [centred(g - w, Qlow) for g, w in zip(got, want)] == [0] * o.n
    assert out.scale == 2.0 ** 90 / ql


def _crt(residues, moduli):
    """The integer in [0, prod moduli) with the given residues (Python ints)."""
    M = math.prod(moduli)
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M


def _merged_is_rounded_division(o, seed):
    """The oracle's merged ModDown-rescale of random residues X over
    q_0..q_l, P equals round(X / (P q_l)) by Python big integers, on every
    coefficient (the integer X is the CRT representative in [0, Q_l P))."""
    level, K = o.n_q - 1, o.n_p
    ext = list(range(level + 1)) + [o.n_q + k for k in range(K)]
    moduli = [int(o.moduli[m]) for m in ext]
    rng = np.random.default_rng(seed)
    x = np.stack([rng.integers(0, m, size=o.n, dtype=np.uint64) for m in moduli])
    out = o.moddown_rescale(o.ntt(x, ext), level)
    y = o.intt(out, list(range(level)))
    div = int(o.q[level]) * math.prod(int(o.moduli[o.n_q + k]) for k in range(K))
    Qlow = math.prod(int(q) for q in o.q[:level])
    for k in range(o.n):
        X = _crt([x[t, k] for t in range(len(ext))], moduli)
        Y = _crt([y[t, k] for t in range(level)], [int(q) for q in o.q[:level]])
        assert (Y - (X + (div - 1) // 2) // div) % Qlow == 0, k


def test_merged_moddown_rescale_is_rounded_division(tiny_oracle):
    """Reading C21: the merged step's result is round(X / S), S = P q_l."""
    _merged_is_rounded_division(tiny_oracle, 21)


def test_merged_moddown_rescale_is_rounded_division_with_eight_special_primes():
    """The same at the benchmark's gadget shape: K = 8 special primes of 61 bits
    (S spans nine primes, about 2^540), 61- and 55-bit ciphertext primes, on a
    2^6 ring, four independent draws."""
    from oracle import Oracle
    o = Oracle(6, (61, 55, 55, 55, 55), (61,) * 8, 2, h=8, sigma=3.2)
    for seed in range(4):
        _merged_is_rounded_division(o, 40 + seed)


def test_merged_mul_relin_rescale_matches_separate_steps(toy_oracle):
    """Reading C21 against C9 then C10: the merged step rounds the exact
    quotient, the separate one the quotient of ModDown's floor, so the two
    differ by at most 2 per coefficient; the merged product decrypts within 2^-25."""
    o = toy_oracle
    scale = 2.0 ** 40
    level = o.n_q - 1
    z = si.messages(31, 2, o.n // 2)
    cts = [o.encrypt(o.pt_from_int(o.encode(z[i], scale), level), level, scale, 60 + i) for i in range(2)]
    merged = o.mul_relin_rescale(cts[0], cts[1])
    separate = o.rescale(o.mul_relin(cts[0], cts[1]))
    assert (merged.level, merged.scale) == (separate.level, separate.scale)
    Qlow = math.prod(int(q) for q in o.q[:level])
    for pol in range(2):
        a = o.crt_centred(o.intt(merged.data[pol], list(range(level))), level - 1)
        b = o.crt_centred(o.intt(separate.data[pol], list(range(level))), level - 1)
        assert max(abs(centred(p - q, Qlow)) for p, q in zip(a, b)) <= 2
    err = np.max(np.abs(o.decrypt_decode(merged) - z[0] * z[1]))
    assert err <= 2.0 ** -25, err


# ---------------------------------------------------------------- automorphisms (C11)
def test_automorphism_group_law(tiny_oracle):
    o = tiny_oracle
    rng = np.random.default_rng(13)
    x = rng.integers(0, o.q[0], size=(1, o.n), dtype=np.uint64)
    for g, h in [(5, 25), (3, 2 * o.n - 1), (2 * o.n - 1, 2 * o.n - 1)]:
        lhs = o.automorph_coeff(o.automorph_coeff(x, [0], h), [0], g)
        rhs = o.automorph_coeff(x, [0], (g * h) % (2 * o.n))
        assert np.array_equal(lhs, rhs)
    assert o.galois_elt(o.n // 2) == 1
    assert o.galois_elt(-1) == pow(5, o.n // 2 - 1, 2 * o.n)


def test_rotation_and_conjugation_slot_semantics(toy_oracle):
    o = toy_oracle
    z = si.messages(14, 1, o.n // 2)[0]
    scale = 2.0 ** 40
    level = o.n_q - 1
    ct = o.encrypt(o.pt_from_int(o.encode(z, scale), level), level, scale, 5)
    for k in (1, 2, 3, -1, 5):
        got = o.decrypt_decode(o.rotate(ct, k))
        assert np.max(np.abs(got - np.roll(z, -k))) < 2 ** -20
    r12 = o.decrypt_decode(o.rotate(o.rotate(ct, 1), 2))
    assert np.max(np.abs(r12 - np.roll(z, -3))) < 2 ** -19
    got = o.decrypt_decode(o.conjugate(ct))
    assert np.max(np.abs(got - np.conj(z))) < 2 ** -20


# ---------------------------------------------------------------- Eq. add/sub/mult
def test_slotwise_operations_and_mult_error_bound(toy_oracle):
    o = toy_oracle
    z = si.messages(15, 2, o.n // 2)
    scale = 2.0 ** 40
    level = o.n_q - 1
    a = o.encrypt(o.pt_from_int(o.encode(z[0], scale), level), level, scale, 21)
    b = o.encrypt(o.pt_from_int(o.encode(z[1], scale), level), level, scale, 22)
    assert np.max(np.abs(o.decrypt_decode(o.add(a, b)) - (z[0] + z[1]))) < 2 ** -28
    assert np.max(np.abs(o.decrypt_decode(o.sub(a, b)) - (z[0] - z[1]))) < 2 ** -28
    prod = o.rescale(o.mul_relin(a, b))
    assert prod.level == level - 1
    err = np.max(np.abs(o.decrypt_decode(prod) - z[0] * z[1]))
    assert err <= 2 ** -25, err
    pm = o.rescale(o.mul_plain(a, o.pt_from_int(o.encode(z[1], scale), level), scale))
    assert np.max(np.abs(o.decrypt_decode(pm) - z[0] * z[1])) <= 2 ** -25
    assert np.max(np.abs(o.decrypt_decode(o.mul_int(a, 2)) - 2 * z[0])) < 2 ** -27


def test_tensor_decrypts_under_s_squared(tiny_oracle):
    o = tiny_oracle
    n, level = o.n, o.n_q - 1
    rng = np.random.default_rng(16)
    ma = rng.integers(-2 ** 30, 2 ** 30, size=n)
    mb = rng.integers(-2 ** 30, 2 ** 30, size=n)
    a = o.encrypt(o.pt_from_int(ma, level), level, 1.0, 1)
    b = o.encrypt(o.pt_from_int(mb, level), level, 1.0, 2)
    d = o.tensor(a, b)
    mods = list(range(level + 1))
    Q = math.prod(o.q)
    s = [int(v) for v in o.secret()]
    s2 = negacyclic_mul_int(s, s, n)
    dc = [o.crt_centred(o.intt(d[i], mods), level) for i in range(3)]
    dec = [centred(x + y + w, Q) for x, y, w in
           zip(dc[0], negacyclic_mul_int(dc[1], s, n), negacyclic_mul_int(dc[2], s2, n))]
    ea, eb = [int(v) for v in o.enc_error(1)], [int(v) for v in o.enc_error(2)]
    want = negacyclic_mul_int([int(x) + y for x, y in zip(ma, ea)], [int(x) + y for x, y in zip(mb, eb)], n)
    assert [centred(x - y, Q) for x, y in zip(dec, want)] == [0] * n


def test_ring_2_17_product_and_rotations_decrypt_to_slot_math():
    """N = 2^17 (Table 3's eMLP-2/3 ring; primes = 1 mod 2^18): the merged
    product and rotations by 1 and 2^15 decrypt to the slot-wise product and
    the cyclic shifts of the 2^16 slots."""
    import synthetic_inputs as si
    w = si.N17
    o = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    assert all(q % (1 << 18) == 1 for q in o.moduli)
    o.keygen(3)
    o.gen_rotation_keys([1, 1 << 15])
    z = si.messages(1, 2, w.slots)
    sc, lv = 2.0 ** w.log2_scale, len(w.q_bits) - 1
    a, b = (o.encrypt(o.pt_from_int(o.encode(z[i], sc), lv), lv, sc, 1 + i) for i in range(2))
    assert np.max(np.abs(o.decrypt_decode(o.mul_relin_rescale(a, b)) - z[0] * z[1])) < 2.0 ** -30
    for k in (1, 1 << 15):
        assert np.max(np.abs(o.decrypt_decode(o.rotate(a, k)) - np.roll(z[0], -k))) < 2.0 ** -30
