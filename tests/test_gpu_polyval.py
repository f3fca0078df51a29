"""power / polyval (§3) on the GPU through the C ABI versus the CPU oracle, bit-exact on identical
keys and ciphertexts, plus the batched entry points against the single calls and the error cases.

Chains: six 30-bit data primes at N = 4096 (64-bit words, up to degree 16), unequal primes
[50, 40, 30, 40 | 50] (the scale bookkeeping), C2's [31, 26 x 6 | 31] at N = 8192 (32-bit words), and
the paper's unary-operation context N = 8192 with a 200-bit modulus [60, 40, 40 | 60] at 2^40."""
import math

import numpy as np
import pytest

import paper_2104_03152_gb300 as tk
from gpu_common import Pair, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu

CHAINS = {
    "deep": (12, [40, 30, 30, 30, 30, 30, 40], 2.0 ** 30),
    "uneven": (12, [50, 40, 30, 40, 50], 2.0 ** 35),
    "C2": (13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26),
    "table": (13, [60, 40, 40, 60], 2.0 ** 40),
}
POLYS = [
    [0.0, 1.0, 2.0],                                  # the paper's unary benchmark 2x^2 + x
    [0.5, 0.197, 0.0, -0.004],                        # degree-3 sigmoid approximation
    [-0.25, 0.0, 0.0, 0.0, 0.0, 1.5],
    [1.0, -0.5, 0.25, -0.125, 0.0625, 0.0, 0.0, 0.3],
    [0.0, 0.0, 0.0, 0.0, 1.0],
]


@pytest.fixture(scope="module", params=sorted(CHAINS))
def pair(request):
    return Pair(*CHAINS[request.param])


def _enc(pair, seed):
    o = pair.o
    x = inputs.uniform_slots(o.slots, seed)
    pt = o.encode(x)
    return x, o.encrypt(pt, 700 + seed), pair.g.encrypt(pair.import_pt(pt), 700 + seed)


def test_power_parity(pair):
    x, oc, gc = _enc(pair, 1)
    for k in (1, 2, 3, 4, 5, 7, 8, 13, 16):
        if pair.o.L < math.ceil(math.log2(k)) + 1:
            with pytest.raises(tk.TcksError) as e:
                gc.power(k)
            assert e.value.name == "LEVEL_EXHAUSTED"
            continue
        assert_ct_equal(gc.power(k), pair.o.power(oc, k), f"x^{k}")


def test_polyval_parity(pair):
    x, oc, gc = _enc(pair, 2)
    for coeffs in POLYS:
        d = len(coeffs) - 1
        if pair.o.L < math.ceil(math.log2(d)) + 2:
            with pytest.raises(tk.TcksError) as e:
                gc.polyval(coeffs)
            assert e.value.name == "LEVEL_EXHAUSTED"
            continue
        ref = pair.o.polyval(oc, coeffs)
        got = gc.polyval(coeffs)
        assert_ct_equal(got, ref, str(coeffs))
        err = float(np.max(np.abs(pair.g.decrypt_values(got) - np.polynomial.polynomial.polyval(x, coeffs))))
        # 1e-3 at scales >= 2^30; C2's 2^26 leaves about 16x the noise (the oracle itself reaches 9e-3)
        assert err < (1e-3 if pair.o.scale >= 2.0 ** 30 else 2e-2), (coeffs, err)


def test_polyval_many_terms_and_a_lower_input():
    """Degree 12 with every coefficient non-zero (12 terms: two passes of the combination kernel), and
    an input one level down whose scale is no longer the context scale."""
    pair = Pair(*CHAINS["deep"])
    x, oc, gc = _enc(pair, 3)
    coeffs = [0.01 * (-1) ** i * (i + 1) for i in range(13)]
    assert_ct_equal(gc.polyval(coeffs), pair.o.polyval(oc, coeffs), "degree 12")
    one = pair.o.encode(np.ones(pair.o.slots))
    om = pair.o.mul(oc, pair.o.encrypt(one, 9))
    gm = gc.mul(pair.g.encrypt(pair.import_pt(one), 9))
    assert_ct_equal(gm, om, "input")
    c3 = [0.1, -1.0, 0.5, 2.0]
    assert_ct_equal(gm.polyval(c3), pair.o.polyval(om, c3), "lower input")


def test_batched_equals_single(pair):
    cts = [_enc(pair, 10 + i)[2] for i in range(5)]
    coeffs = [0.5, 0.197, 0.0, -0.004] if pair.o.L >= 4 else [0.0, 1.0, 2.0]
    outs = tk.polyval_batch(cts, coeffs)
    for c, r in zip(cts, outs):
        assert np.array_equal(r.export(), c.polyval(coeffs).export())
    k = 3 if pair.o.L >= 3 else 2
    p = tk.power_batch(cts, k)
    for c, r in zip(cts, p):
        assert np.array_equal(r.export(), c.power(k).export())
    assert tk.polyval_batch([], coeffs) == []


def test_errors_launch_nothing():
    pair = Pair(*CHAINS["deep"])
    _, _, gc = _enc(pair, 4)
    low = pair.g.ct_import(gc.export(), gc.info()[1])
    low.mod_switch_(3)
    cases = [
        (lambda: gc.polyval([1.0, 0.0]), "INVALID_ARG"),
        (lambda: gc.polyval([]), "INVALID_ARG"),
        (lambda: gc.power(0), "INVALID_ARG"),
        (lambda: low.polyval([0.0, 0.0, 0.0, 0.0, 1.0]), "LEVEL_EXHAUSTED"),
        (lambda: low.power(5), "LEVEL_EXHAUSTED"),
        (lambda: gc.polyval([0.0, 1e30]), "VALUE_OVERFLOW"),
        (lambda: gc.polyval([1e30, 1.0]), "VALUE_OVERFLOW"),
        (lambda: tk.polyval_batch([gc, low], [0.0, 1.0]), "LEVEL_MISMATCH"),
    ]
    pair.g.synchronize()
    before = tk.launch_count()
    for fn, name in cases[:5]:
        with pytest.raises(tk.TcksError) as e:
            fn()
        assert e.value.name == name
    assert tk.launch_count() == before
    for fn, name in cases[5:]:
        with pytest.raises(tk.TcksError) as e:
            fn()
        assert e.value.name == name
