"""Pins of the oracle's hybrid key switching (reading A26: digits of alpha data primes, K special
primes, balanced fast base conversions in ModUp and ModDown).

Independent references: the one-prime key switch (alpha = 1, K = 1, itself pinned by big integers in
test_oracle_ckks.py) must come out bit for bit; the base conversion is characterised in big integers
(congruence to the input modulo the digit's primes and the size bound of a balanced conversion); the
key-switch output satisfies the key-switching equation c0 + c1 s = x s' + e with e inside the bound
that the definitions give; decryptions match FP64; hoisting is exact; trimmed keys are sub-arrays.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleCKKS
from oracle.ckks import P as ptr
from paper_2104_03152_gb300 import inputs


def _centred(v: int, m: int) -> int:
    v %= m
    return v - m if v > m // 2 else v


def _compose(o, rows: np.ndarray, chain_idx) -> list[int]:
    """Coefficient-domain residues (rows modulo the chain primes chain_idx) to centred integers."""
    qs = [o.q[i] for i in chain_idx]
    M = math.prod(qs)
    out = []
    for k in range(o.N):
        x = 0
        for r, q in enumerate(qs):
            Mr = M // q
            x += int(rows[r][k]) * pow(Mr % q, -1, q) * Mr
        out.append(_centred(x, M))
    return out


def test_alpha1_k1_is_the_one_prime_key_switch():
    """With alpha = 1 and one special prime the hybrid functions reproduce O6-O18 bit for bit."""
    o = OracleCKKS(11, [36, 36, 36, 37], 2.0 ** 30).keygen()
    o.gen_galois_keys([1, 5])
    L, N = o.L, o.N
    lib = oracle.lib()
    rlk = np.zeros((L, 2, L + 1, N), dtype=np.uint64)
    lib.orc_keygen_relin_hyb(o._ctx, o.key_seed, ptr(o.s), 1, L, ptr(rlk))
    assert np.array_equal(rlk, o.rlk.data)
    gk = np.zeros_like(rlk)
    lib.orc_keygen_galois_hyb(o._ctx, o.key_seed, ptr(o.s), o.galois_elt(5), 1, L, ptr(gk))
    assert np.array_equal(gk, o.galois[5].data)
    x = np.ascontiguousarray(inputs.random_limbs(o.q[:3], N, 7, polys=1)[0])
    d = np.zeros((3, 4, N), dtype=np.uint64)
    lib.orc_modup_hyb(o._ctx, ptr(x), 3, 1, ptr(d))
    assert np.array_equal(d, o.modup_poly(x, 3))
    out = np.zeros((2, 3, N), dtype=np.uint64)
    lib.orc_keyswitch_hyb(o._ctx, ptr(x), 3, 1, ptr(o.rlk.data), L, ptr(out))
    assert np.array_equal(out, o.keyswitch(x, 3, o.rlk))
    ct = oracle.Ct(np.ascontiguousarray(inputs.random_limbs(o.q[:3], N, 8, polys=2)), 3, 1.0)
    rot = np.zeros_like(ct.data)
    lib.orc_rotate_hyb(o._ctx, ptr(ct.data), 3, 1, o.galois_elt(1), ptr(o.galois[1].data), L, ptr(rot))
    assert np.array_equal(rot, o.rotate(ct, 1).data)


@pytest.fixture(scope="module")
def tiny():
    # four 24-bit data primes in digits of two, two 26-bit special primes
    return OracleCKKS(4, [24, 24, 24, 24, 26, 26], 2.0 ** 10, n_special=2, alpha=2).keygen()


@pytest.mark.parametrize("level", [4, 3])
def test_modup_is_a_balanced_base_conversion(tiny, level):
    """Every digit, composed over all its limbs, is an integer polynomial congruent to the input
    modulo the digit's primes, of size at most |G_j| Q_j / 2, and equal to sum_i y_i Q_j / q_i."""
    o = tiny
    x = np.ascontiguousarray(inputs.random_limbs(o.q[:level], o.N, 11, polys=1)[0])
    D = o.modup_poly(x, level)
    assert D.shape == (o.digits(level), level + o.K, o.N)
    chain = list(range(level)) + [o.L + k for k in range(o.K)]
    X = _compose(o, o.intt_rows(x, list(range(level))), list(range(level)))
    for j in range(o.digits(level)):
        G = list(range(j * o.alpha, min((j + 1) * o.alpha, level)))
        Qj = math.prod(o.q[i] for i in G)
        Dj = _compose(o, o.intt_rows(D[j], chain), chain)
        for k in range(o.N):
            assert (Dj[k] - X[k]) % Qj == 0
            assert abs(Dj[k]) <= len(G) * Qj // 2
        # the defining sum, in exact integers, from the coefficient residues of the digit's primes
        xi = o.intt_rows(x[G], G)
        for k in range(o.N):
            tot = 0
            for r, i in enumerate(G):
                hat = Qj // o.q[i]
                y = int(xi[r][k]) * pow(hat % o.q[i], -1, o.q[i]) % o.q[i]
                tot += _centred(y, o.q[i]) * hat
            assert Dj[k] == tot


@pytest.mark.parametrize("level", [5, 4, 2])
def test_keyswitch_equation_and_noise_bound(level):
    """KS_s'(x) = (c0, c1) with c0 + c1 s = x s' + e (mod Q_level), e small: |e| <= sum_j |D_j| |e_j|_1 / P
    + (K/2)(1 + |s|_1), with |D_j| <= alpha Q_j / 2 and CBD errors |e_j| <= 21 (here s' = s^2, the
    relinearization key)."""
    o = OracleCKKS(10, [30, 30, 30, 30, 30, 34, 34], 2.0 ** 20, n_special=2, alpha=2).keygen()
    N = o.N
    x = np.ascontiguousarray(inputs.random_limbs(o.q[:level], N, 21 + level, polys=1)[0])
    c0, c1 = o.keyswitch(x, level, o.rlk)
    idx = list(range(level))
    diff = np.zeros((level, N), dtype=np.uint64)
    for i in idx:
        q = o.q[i]
        s = o.s[i].astype(object)
        lhs = (c0[i].astype(object) + c1[i].astype(object) * s) % q
        rhs = (x[i].astype(object) * s * s) % q
        diff[i] = np.array((lhs - rhs) % q, dtype=np.uint64)
    e = _compose(o, o.intt_rows(diff, idx), idx)
    Pspec = math.prod(o.q[o.L:])
    Qmax = max(math.prod(o.q[j * o.alpha:min((j + 1) * o.alpha, level)]) for j in range(o.digits(level)))
    bound = o.digits(level) * (o.alpha * Qmax // 2) * 21 * N / Pspec + o.K / 2 * (1 + N)
    worst = max(abs(v) for v in e)
    assert worst <= bound, (worst, bound)


@pytest.fixture(scope="module")
def c4h():
    """N = 4096, five data primes [50, 40, 40, 40, 40] in digits of two, special primes [60, 60]."""
    o = OracleCKKS(12, [50, 40, 40, 40, 40, 60, 60], 2.0 ** 40, n_special=2, alpha=2).keygen()
    o.gen_galois_keys([1, 7, 100])
    return o


def test_hybrid_ops_match_fp64(c4h):
    o = c4h
    x, y = inputs.uniform_slots(o.slots, 1), inputs.uniform_slots(o.slots, 2)
    cx, cy = o.encrypt_values(x, 3), o.encrypt_values(y, 4)
    assert np.max(np.abs(o.decrypt_values(o.mul(cx, cy)) - x * y)) < 1e-5
    for st in (1, 7, 100):
        assert np.max(np.abs(o.decrypt_values(o.rotate(cx, st)) - np.roll(x, -st))) < 1e-5
    for lv in (3, 2, 1):  # a partial last digit at level 3 and 1
        low = o.mod_switch(cx, lv)
        assert np.max(np.abs(o.decrypt_values(o.rotate(low, 7)) - np.roll(x, -7))) < 1e-4
        if lv >= 2:
            prod = o.mul(o.mod_switch(cx, lv), o.mod_switch(cy, lv))
            assert np.max(np.abs(o.decrypt_values(prod) - x * y)) < 1e-4


def test_hybrid_hoisting_is_exact(c4h):
    """The balanced conversions commute with the automorphism, so rotations from one shared ModUp
    equal the plain rotations bit for bit."""
    o = c4h
    ct = o.encrypt_values(inputs.uniform_slots(o.slots, 5), 6)
    for lv in (5, 3):
        c = o.mod_switch(ct, lv)
        digits = o.modup(c)
        for st in (1, 7, 100):
            assert np.array_equal(o.rotate_from_digits(c, digits, st).data, o.rotate(c, st).data), (lv, st)


def test_hybrid_key_trimming(c4h):
    """A key trimmed to level 3 holds the full key's first ceil(3/alpha) digits on limbs q_0..q_2 and
    the special primes, unchanged."""
    o = c4h
    full = o.galois[7].data
    t = OracleCKKS(12, [50, 40, 40, 40, 40, 60, 60], 2.0 ** 40, n_special=2, alpha=2).keygen()
    k3 = t.gen_galois_key(7, 3).data
    assert k3.shape == (2, 2, 3 + 2, o.N)
    keep = [0, 1, 2, o.L, o.L + 1]
    assert np.array_equal(k3, full[:2][:, :, keep])
