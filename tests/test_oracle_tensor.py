"""Pins of the oracle's CKKSTensor (§2.3): every tensor operation decrypts to numpy's result on the
same values (broadcasting, axes, reductions and products as numpy defines them), batched and not."""
import numpy as np
import pytest

from oracle import OracleCKKS, OracleTensor

TOL = 1e-3


@pytest.fixture(scope="module")
def o():
    """N = 2048, five 30-bit data primes and a 40-bit special prime, scale 2^30."""
    o = OracleCKKS(11, [40, 30, 30, 30, 30, 40], 2.0 ** 30).keygen()
    o.gen_galois_keys([1, 2, 4])
    return o


def _vals(shape, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


def _close(t, ref, tol=TOL):
    got = t.decrypt()
    assert got.shape == np.shape(ref), (got.shape, np.shape(ref))
    err = float(np.max(np.abs(got - ref)))
    assert err < tol, err


def test_roundtrip_and_layout(o):
    x = _vals((3, 4), 1)
    t = OracleTensor.encrypt(o, x, seed=10)
    assert t.shape == (3, 4) and len(t.cts) == 12
    _close(t, x)
    xb = _vals((8, 3), 2)
    tb = OracleTensor.encrypt(o, xb, batch=True, seed=20)
    assert tb.shape == (8, 3) and len(tb.cts) == 3
    # ciphertext i holds column i of the batched values in slots [0, 8)
    assert np.max(np.abs(o.decrypt_values(tb.cts[1], 8) - xb[:, 1])) < TOL
    _close(tb, xb)


def test_elementwise_with_broadcasting(o):
    x, y = _vals((3, 4), 3), _vals((4,), 4)
    a, b = OracleTensor.encrypt(o, x, seed=1), OracleTensor.encrypt(o, y, seed=100)
    _close(a.add(b), x + y)
    _close(a.sub(b), x - y)
    _close(a.mul(b), x * y)
    _close(a.negate(), -x)
    _close(a.square(), x * x)
    xb, yb = _vals((8, 2, 3), 5), _vals((8, 1, 3), 6)
    ab, bb = OracleTensor.encrypt(o, xb, batch=True, seed=200), OracleTensor.encrypt(o, yb, batch=True, seed=300)
    _close(ab.mul(bb), xb * yb)
    _close(ab.add(bb), xb + yb)


def test_plain_operands(o):
    x = _vals((3, 4), 7)
    a = OracleTensor.encrypt(o, x, seed=1)
    w = _vals((3, 4), 8)
    _close(a.add(0.25), x + 0.25)
    _close(a.sub(w), x - w)
    _close(a.mul(w), x * w)           # constant polynomial per ciphertext
    _close(a.mul(-1.5), x * -1.5)
    xb = _vals((8, 3), 9)
    ab = OracleTensor.encrypt(o, xb, batch=True, seed=50)
    wb = _vals((8, 3), 10)
    _close(ab.mul(wb), xb * wb)        # varies along the batched axis: encoded per ciphertext
    _close(ab.mul(wb[0]), xb * wb[0])  # constant along it: constant polynomials
    _close(ab.add(wb), xb + wb)


def test_power_polyval(o):
    x = _vals((2, 3), 11)
    a = OracleTensor.encrypt(o, x, seed=1)
    _close(a.power(3), x ** 3)
    c = [0.5, 0.197, 0.0, -0.004]
    _close(a.polyval(c), np.polynomial.polynomial.polyval(x, c))


def test_reductions(o):
    x = _vals((3, 4), 12)
    a = OracleTensor.encrypt(o, x, seed=1)
    _close(a.sum(0), x.sum(0))
    _close(a.sum(1), x.sum(1))
    _close(a.sum(), x.sum())
    xb = _vals((8, 2, 3), 13)
    ab = OracleTensor.encrypt(o, xb, batch=True, seed=60)
    _close(ab.sum(2), xb.sum(2))
    s0 = ab.sum(0)
    assert s0.shape == (2, 3) and not s0.batch
    _close(s0, xb.sum(0))
    _close(ab.sum(), xb.sum())
    x6 = _vals((6, 2), 14)  # B = 6: the slots [6, 8) are zero and join the rotate-and-add
    a6 = OracleTensor.encrypt(o, x6, batch=True, seed=70)
    _close(a6.sum(0), x6.sum(0))
    dirty = a6.polyval([0.5, 1.0])
    with pytest.raises(ValueError):
        dirty.sum(0)


def test_products(o):
    u, v = _vals((5,), 15), _vals((5,), 16)
    tu, tv = OracleTensor.encrypt(o, u, seed=1), OracleTensor.encrypt(o, v, seed=10)
    _close(tu.dot(tv), np.dot(u, v))
    A, B = _vals((2, 3), 17), _vals((3, 4), 18)
    tA, tB = OracleTensor.encrypt(o, A, seed=100), OracleTensor.encrypt(o, B, seed=200)
    _close(tA.dot(tB), A @ B)
    M = _vals((3, 5), 19)
    _close(tA.mm_plain(M), A @ M)
    xb = _vals((8, 3), 20)
    tb = OracleTensor.encrypt(o, xb, batch=True, seed=300)
    _close(tb.mm_plain(M), xb @ M)  # a linear layer over 8 samples batched in the slots


def test_rearrangement_and_levels(o):
    x = _vals((2, 3, 4), 21)
    a = OracleTensor.encrypt(o, x, seed=1)
    _close(a.transpose((2, 0, 1)), x.transpose((2, 0, 1)))
    _close(a.reshape((6, 4)), x.reshape(6, 4))
    y = _vals((2, 3, 4), 22)
    b = OracleTensor.encrypt(o, y, seed=100).mul(1.0)  # one level down, rescaled
    assert b.level == a.level - 1
    _close(a.mul(b), x * y)
