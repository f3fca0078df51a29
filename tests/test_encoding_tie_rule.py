"""The checker the GPU encoding tests use (assert_encoding_agrees) must itself reject what it is there to
catch: a coefficient moved by one away from a .5 tie, a coefficient moved by two, a P limb that carries
another integer than the data limbs, and a wrong scale. The mistakes are planted in oracle encodings on
the CPU."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_encoding_agrees, encode_tie_bound
from paper_2104_03152_gb300 import inputs

BITS = [31, 26, 26, 26, 31]


@pytest.fixture(scope="module")
def o():
    return oracle.OracleCKKS(11, BITS, 2.0 ** 26)


def _shift(o, limbs, idx, i, delta):
    """limbs (NTT form, rows modulo the chain primes idx) with coefficient i moved by delta."""
    c = o.intt_rows(limbs, idx)
    for r, l in enumerate(idx):
        q = o.q[l]
        c[r, i] = np.uint64((int(c[r, i]) + delta) % q)
    out = c.copy()
    for r, l in enumerate(idx):
        row = np.ascontiguousarray(out[r])
        oracle.lib().orc_ntt_limb(o._ctx, oracle.ckks.P(row), l)
        out[r] = row
    return out


def test_identical_encoding_passes(o):
    z = inputs.uniform_slots(o.slots, 1)
    pt = o.encode(z, level=3)
    assert assert_encoding_agrees(o, pt.data, z, o.scale, 3) == 0
    ext = o.encode_ext(z, 3)
    assert assert_encoding_agrees(o, ext, z, o.scale, 3) == 0


def test_off_by_one_away_from_a_tie_fails(o):
    z = inputs.uniform_slots(o.slots, 2)
    pt, pre = o.encode(z, level=3, want_pre=True)
    frac = np.abs(pre - np.floor(pre) - 0.5)
    i = int(np.argmax(frac))  # the coefficient farthest from a tie
    bad = _shift(o, pt.data, [0, 1, 2], i, 1)
    with pytest.raises(AssertionError, match="not near a .5 tie"):
        assert_encoding_agrees(o, bad, z, o.scale, 3)


def test_off_by_one_at_a_tie_passes(o):
    # one non-zero slot x: coefficient 0 is scale (2/N) x, here exactly 2^16 + 1/2, a tie that the oracle
    # rounds away from zero and an FFT a hair below it would round down
    x = (2.0 ** 16 + 0.5) * o.N / 2.0 / o.scale
    z = np.zeros(o.slots)
    z[0] = x
    pt, pre = o.encode(z, level=3, want_pre=True)
    assert pre[0] == 2.0 ** 16 + 0.5
    good = _shift(o, pt.data, [0, 1, 2], 0, -1)
    assert assert_encoding_agrees(o, good, z, o.scale, 3) == 1
    with pytest.raises(AssertionError, match="not near a .5 tie"):  # coefficient 1 is no tie
        assert_encoding_agrees(o, _shift(o, good, [0, 1, 2], 1, 1), z, o.scale, 3)


def test_off_by_two_fails(o):
    z = inputs.uniform_slots(o.slots, 4)
    pt = o.encode(z, level=3)
    bad = _shift(o, pt.data, [0, 1, 2], 5, 2)
    with pytest.raises(AssertionError, match="more than one"):
        assert_encoding_agrees(o, bad, z, o.scale, 3)


def test_p_limb_of_another_integer_fails(o):
    z = inputs.uniform_slots(o.slots, 5)
    ext = o.encode_ext(z, 3)
    bad = ext.copy()
    bad[3:] = _shift(o, ext[3:], [o.L], 7, 1)
    with pytest.raises(AssertionError):
        assert_encoding_agrees(o, bad, z, o.scale, 3)


def test_wrong_scale_fails(o):
    z = inputs.uniform_slots(o.slots, 6)
    pt = o.encode(z, scale=2.0 ** 25, level=3)
    with pytest.raises(AssertionError):
        assert_encoding_agrees(o, pt.data, z, o.scale, 3)
