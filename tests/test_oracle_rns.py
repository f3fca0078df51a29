"""Pins of the oracle's RNS layer: primes (O1), roots (O2), the NTT (O3), Philox (O5).

Each check compares the oracle with something other than itself: a library primality test, brute
force over small moduli, the O(N^2) evaluation definition, schoolbook negacyclic products, and
numpy's own Philox4x64-10.
"""
import numpy as np
import pytest

import oracle
from tiny_ckks import brv, negacyclic_mul, primitive_2n_roots

CHAINS = {
    "C1 N=4096 [36,36,36|37]": (12, [36, 36, 36, 37]),
    "C2 N=8192 [31,26x6|31]": (13, [31, 26, 26, 26, 26, 26, 26, 31]),
    "C4 N=16384 [60,40,40|60]": (14, [60, 40, 40, 60]),
}


@pytest.mark.parametrize("name", sorted(CHAINS))
def test_primes_definition(name):
    sympy = pytest.importorskip("sympy")
    log_n, bits = CHAINS[name]
    m = 2 << log_n
    qs = oracle.gen_primes(log_n, bits)
    assert len(set(qs)) == len(qs)
    for k, (q, b) in enumerate(zip(qs, bits)):
        assert sympy.isprime(q)
        assert q % m == 1
        assert q.bit_length() == b
        # largest: every larger candidate of this size is composite or already taken
        c = q + m
        while c < (1 << b):
            assert (not sympy.isprime(c)) or c in qs[:k], (name, k, c)
            c += m


def test_c2_chain_shape():
    qs = oracle.gen_primes(13, [31, 26, 26, 26, 26, 26, 26, 31])
    # the special prime is the second-largest 31-bit prime == 1 mod 2N (the first is q_0)
    assert qs[7] < qs[0]
    assert sorted(qs[1:7], reverse=True) == qs[1:7]


def test_primality_matches_library():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(0)
    cands = [int(x) for x in rng.integers(2, 1 << 62, size=300, dtype=np.uint64)]
    cands += [2, 3, 4, 561, 1105, 3215031751, 2152302898747, 3474749660383, 341550071728321,
              3825123056546413051, (1 << 61) - 1, (1 << 62) - 57]
    for c in cands:
        assert oracle.is_prime(c) == sympy.isprime(c), c


@pytest.mark.parametrize("log_n,q", [(3, 17), (4, 97), (4, 193), (5, 193), (5, 449), (6, 7681), (6, 12289),
                                     (8, 12289), (10, 12289)])
def test_min_psi_brute_force(log_n, q):
    n = 1 << log_n
    psi = oracle.min_psi(q, log_n)
    assert pow(psi, n, q) == q - 1
    # no smaller x is a primitive 2N-th root
    for x in range(2, psi):
        assert pow(x, n, q) != q - 1
    assert psi == primitive_2n_roots(q, n)[0]


@pytest.mark.parametrize("name", sorted(CHAINS))
def test_min_psi_config_primes(name):
    log_n, bits = CHAINS[name]
    n = 1 << log_n
    for q in oracle.gen_primes(log_n, bits):
        psi = oracle.min_psi(q, log_n)
        assert pow(psi, n, q) == q - 1
        # minimal among all N primitive roots psi0^k, k odd (enumerated independently here)
        if log_n <= 12:
            sq = psi * psi % q
            cur = psi
            for _ in range(n - 1):
                cur = cur * sq % q
                assert cur >= psi


@pytest.mark.parametrize("log_n", [3, 4, 5, 6, 7, 8])
def test_fast_ntt_equals_definition(log_n):
    n = 1 << log_n
    for bits in (20, 36, 60):
        q = oracle.gen_primes(log_n, [bits])[0]
        psi = oracle.min_psi(q, log_n)
        a = np.random.default_rng(log_n * 100 + bits).integers(0, q, size=n, dtype=np.uint64)
        ref = np.zeros(n, dtype=np.uint64)
        for j in range(n):  # independent Python evaluation of the definition
            w = pow(psi, 2 * brv(j, log_n) + 1, q)
            ref[j] = sum(int(a[i]) * pow(w, i, q) for i in range(n)) % q
        assert np.array_equal(oracle.ntt_naive(a, q, psi), ref)
        assert np.array_equal(oracle.ntt(a, q, psi), ref)


@pytest.mark.parametrize("log_n", [3, 4, 5, 6])
def test_ntt_product_is_schoolbook(log_n):
    """P1: pointwise product of transforms = schoolbook negacyclic product, every config prime."""
    n = 1 << log_n
    primes = [oracle.gen_primes(log_n, [b])[0] for b in (26, 31, 36, 37, 40, 60)]
    for q in primes:
        psi = oracle.min_psi(q, log_n)
        rng = np.random.default_rng(q % 1000)
        a = rng.integers(0, q, size=n, dtype=np.uint64)
        b = rng.integers(0, q, size=n, dtype=np.uint64)
        fa, fb = oracle.ntt(a, q, psi), oracle.ntt(b, q, psi)
        prod = np.array([int(x) * int(y) % q for x, y in zip(fa, fb)], dtype=np.uint64)
        got = oracle.intt(prod, q, psi)
        ref = negacyclic_mul([int(x) for x in a], [int(x) for x in b], q)
        assert [int(x) for x in got] == ref


@pytest.mark.parametrize("log_n", [10, 12, 13, 14, 15, 16])
def test_ntt_roundtrip(log_n):
    """P2: INTT(NTT(a)) = a, and X * a maps to a pointwise product by the evaluation points."""
    n = 1 << log_n
    for bits in (31, 50, 60):
        q = oracle.gen_primes(log_n, [bits])[0]
        psi = oracle.min_psi(q, log_n)
        a = np.random.default_rng(bits).integers(0, q, size=n, dtype=np.uint64)
        fa = oracle.ntt(a, q, psi)
        assert np.array_equal(oracle.intt(fa, q, psi), a)
        if log_n <= 12:
            # multiplication by X: coefficient shift with the wrapped term negated (X^N = -1)
            xa = np.concatenate([np.array([(q - int(a[-1])) % q], dtype=np.uint64), a[:-1]])
            fxa = oracle.ntt(xa, q, psi)
            for j in range(0, n, 97):
                w = pow(psi, 2 * brv(j, log_n) + 1, q)
                assert int(fxa[j]) == int(fa[j]) * w % q


def _numpy_philox(ctr, key):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64))
    st = bg.state
    c = [int(x) for x in ctr]
    # numpy increments the 256-bit counter before each block: start one below
    v = (c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)) - 1
    v %= 1 << 256
    st["state"]["counter"] = np.array([(v >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    st["buffer_pos"] = 4
    bg.state = st
    return [int(x) for x in bg.random_raw(4)]


def test_philox_matches_numpy():
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([2**64 - 1] * 4, [2**64 - 1] * 2), ([5, 3, 0, 0], [0x7E5EA1, 2])]
    for _ in range(50):
        cases.append(([int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.uint64)],
                      [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.uint64)]))
    for ctr, key in cases:
        assert oracle.philox4x64(ctr, key) == _numpy_philox(ctr, key), (ctr, key)


def test_philox_known_answer():
    """Known-answer vector of Philox4x64-10 for a zero counter and key (Salmon et al., SC'11)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.json")
    kat = json.load(open(path))
    for case in kat["cases"]:
        got = oracle.philox4x64([int(x, 16) for x in case["ctr"]], [int(x, 16) for x in case["key"]])
        assert got == [int(x, 16) for x in case["out"]]
