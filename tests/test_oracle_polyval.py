"""Pins of the oracle's power and polynomial evaluation (§3: a minimum-depth circuit for x^k, a
minimal circuit for sum_i a_i x^i).

Independent references: the depth lower bound ceil(log2 k) of a product of k factors, the closed form
of encoding a constant (the general encoder applied to a constant vector), and decrypt(op(Enc(x)))
against numpy's FP64 polynomial evaluation on the same values."""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleCKKS
from paper_2104_03152_gb300 import inputs

# (coefficients a_0..a_d, lowest-degree first): the paper's unary benchmark 2x^2 + x, a degree-3
# sigmoid approximation, and polynomials with gaps, negative terms and a constant
POLYS = [
    [0.0, 1.0, 2.0],
    [0.5, 0.197, 0.0, -0.004],
    [-0.25, 0.0, 0.0, 0.0, 0.0, 1.5],
    [1.0, -0.5, 0.25, -0.125, 0.0625, 0.0, 0.0, 0.3],
    [0.0, 0.0, 0.0, 0.0, 1.0],
]


@pytest.fixture(scope="module")
def deep():
    """N = 4096, six 30-bit data primes and a 40-bit special prime, scale 2^30."""
    return OracleCKKS(12, [40, 30, 30, 30, 30, 30, 40], 2.0 ** 30).keygen()


def _depth(products):
    d = {1: 0}
    for i, a, b in products:
        assert a in d and b in d, "an operand is used before it is computed"
        assert a + b == i
        d[i] = max(d[a], d[b]) + 1
    return d


def test_power_products_reach_the_depth_lower_bound():
    for k in range(1, 300):
        prods = oracle.power_products([k])
        d = _depth(prods)
        assert d[k] == math.ceil(math.log2(k)), k
        # squarings up to the top bit, then one product per further set bit
        assert len(prods) == (k.bit_length() - 1) + bin(k).count("1") - 1, k
    prods = oracle.power_products(range(1, 33))
    d = _depth(prods)
    assert len(prods) == 31 and all(d[i] == math.ceil(math.log2(i)) for i in range(1, 33))


def test_const_pt_is_the_encoding_of_a_constant_vector(deep):
    for a, scale in ((0.75, 2.0 ** 30), (-3.1, 2.0 ** 33), (1e-3, 2.0 ** 40)):
        pt = deep.const_pt(a, scale, 4)
        ref = deep.encode(np.full(deep.slots, a), scale=scale, level=4)
        assert np.array_equal(pt.data, ref.data), a
    with pytest.raises(OverflowError):
        deep.const_pt(4.0, 2.0 ** 61, 2)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8, 11, 16, 31])
def test_power_decrypts_to_xk(deep, k):
    x = inputs.uniform_slots(deep.slots, 40 + k)
    ct = deep.encrypt(deep.encode(x), 500 + k)
    r = deep.power(ct, k)
    assert r.level == deep.L - math.ceil(math.log2(k))
    err = float(np.max(np.abs(deep.decrypt_values(r) - x ** k)))
    assert err < 1e-3, (k, err)


def test_power_of_two_is_repeated_squaring(deep):
    x = inputs.uniform_slots(deep.slots, 3)
    ct = deep.encrypt(deep.encode(x), 77)
    sq = ct
    for _ in range(3):
        sq = deep.square(sq)
    r = deep.power(ct, 8)
    assert np.array_equal(r.data, sq.data) and r.scale == sq.scale


@pytest.mark.parametrize("coeffs", POLYS, ids=[f"deg{len(c) - 1}_{i}" for i, c in enumerate(POLYS)])
def test_polyval_decrypts_to_fp64_polynomial(deep, coeffs):
    x = inputs.uniform_slots(deep.slots, 9)
    ct = deep.encrypt(deep.encode(x), 91)
    r = deep.polyval(ct, coeffs)
    d = len(coeffs) - 1
    assert r.level == deep.L - (math.ceil(math.log2(d)) + 1) if d > 1 else deep.L - 1
    assert r.scale == deep.scale
    ref = np.polynomial.polynomial.polyval(x, coeffs)
    err = float(np.max(np.abs(deep.decrypt_values(r) - ref)))
    assert err < 1e-3, err


def test_polyval_from_a_lower_level_and_a_drifted_scale(deep):
    """Input one level down whose scale is no longer the context scale (after a product): the result
    still lands at the context scale, and a fresh encoding at that scale adds to it."""
    x = inputs.uniform_slots(deep.slots, 12)
    ct = deep.mul(deep.encrypt(deep.encode(x), 5), deep.encrypt(deep.encode(np.ones(deep.slots)), 6))
    assert ct.scale != deep.scale
    coeffs = [0.1, -1.0, 0.5, 2.0]
    r = deep.polyval(ct, coeffs)
    assert r.level == ct.level - 3 and r.scale == deep.scale
    z = deep.add_plain(r, deep.encode(np.full(deep.slots, 0.5), level=r.level))
    ref = np.polynomial.polynomial.polyval(x, coeffs) + 0.5
    assert float(np.max(np.abs(deep.decrypt_values(z) - ref))) < 1e-3


@pytest.fixture(scope="module")
def uneven():
    """Primes of unequal sizes [50, 40, 30, 40 | 50] at scale 2^35: the scale after a rescale depends
    on which prime was divided by, so choosing a wrong prime for a coefficient's scale, or leaving out
    a term's own scale, moves the decrypted value by a factor near 2^10 instead of near 1 + 1e-5."""
    return OracleCKKS(12, [50, 40, 30, 40, 50], 2.0 ** 35).keygen()


@pytest.mark.parametrize("coeffs", [[0.0, 1.0, 2.0], [0.5, 0.197, 0.0, -0.004], [0.1, -1.0, 0.5, 2.0],
                                    [0.0, 0.0, 0.0, 0.0, 1.0]])
def test_polyval_scale_bookkeeping_on_unequal_primes(uneven, coeffs):
    x = inputs.uniform_slots(uneven.slots, 9)
    ct = uneven.encrypt(uneven.encode(x), 91)
    r = uneven.polyval(ct, coeffs)
    assert r.scale == uneven.scale
    err = float(np.max(np.abs(uneven.decrypt_values(r) - np.polynomial.polynomial.polyval(x, coeffs))))
    assert err < 1e-4, err
    for k in (2, 3, 4):
        p = uneven.power(ct, k)
        assert float(np.max(np.abs(uneven.decrypt_values(p) - x ** k))) < 1e-4, k


def test_polyval_rejects_constants_and_exhausted_levels(deep):
    ct = deep.encrypt(deep.encode(inputs.uniform_slots(deep.slots, 1)), 1)
    with pytest.raises(ValueError):
        deep.polyval(ct, [1.0, 0.0, 0.0])
    with pytest.raises(ValueError):
        deep.polyval(deep.mod_switch(ct, 2), [0.0, 1.0, 1.0])
    with pytest.raises(ValueError):
        deep.power(ct, 0)
