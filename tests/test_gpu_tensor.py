"""CKKSTensor (§2.3) on the GPU through the C ABI (ciphertext arrays) versus the oracle's tensor,
bit-exact ciphertext by ciphertext after every operation, on a 64-bit chain and on C2's 32-bit chain;
plus the array ABI's argument errors."""
import ctypes

import numpy as np
import pytest

import paper_2104_03152_gb300 as tk
from gpu_common import Pair
from oracle import OracleTensor

pytestmark = pytest.mark.gpu

CHAINS = {
    "w64": (11, [40, 30, 30, 30, 30, 40], 2.0 ** 30),
    "C2": (13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26),
}


@pytest.fixture(scope="module", params=sorted(CHAINS))
def pair(request):
    return Pair(*CHAINS[request.param], galois=[1, 2, 4])


def _vals(shape, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


def _same(g: tk.CKKSTensor, r: OracleTensor, what=""):
    assert g.shape == r.shape and g.grid == r.grid and g.batch == r.batch, what
    n, lv, sc = g.info()
    assert n == len(r.cts) and lv == r.level and sc == r.cts[0].scale, what
    assert np.array_equal(g.export(), np.stack([c.data for c in r.cts])), what


def _enc(pair, x, batch=False, seed=0):
    return tk.CKKSTensor.encrypt(pair.g, x, batch, seed), OracleTensor.encrypt(pair.o, x, batch, seed)


def test_encrypt_decrypt(pair):
    x = _vals((3, 4), 1)
    g, r = _enc(pair, x, seed=10)
    _same(g, r, "encrypt")
    assert np.max(np.abs(g.decrypt() - x)) < 1e-3
    xb = _vals((8, 3), 2)
    gb, rb = _enc(pair, xb, True, 20)
    _same(gb, rb, "encrypt batched")
    assert np.max(np.abs(gb.decrypt() - xb)) < 1e-3


def test_elementwise_and_plain(pair):
    x, y, w = _vals((3, 4), 3), _vals((4,), 4), _vals((3, 4), 5)
    (ga, ra), (gb, rb) = _enc(pair, x, seed=1), _enc(pair, y, seed=100)
    for what, g, r in [("add", ga.add(gb), ra.add(rb)), ("sub", ga.sub(gb), ra.sub(rb)),
                       ("mul", ga.mul(gb), ra.mul(rb)), ("neg", ga.negate(), ra.negate()),
                       ("square", ga.square(), ra.square()), ("add plain", ga.add(w), ra.add(w)),
                       ("sub scalar", ga.sub(0.25), ra.sub(0.25)), ("mul plain", ga.mul(w), ra.mul(w)),
                       ("power", ga.power(3), ra.power(3)),
                       ("polyval", ga.polyval([0.5, 0.197, 0.0, -0.004]), ra.polyval([0.5, 0.197, 0.0, -0.004]))]:
        _same(g, r, what)
    xb, yb, wb = _vals((8, 2, 3), 6), _vals((8, 1, 3), 7), _vals((8, 2, 3), 8)
    (gx, rx), (gy, ry) = _enc(pair, xb, True, 200), _enc(pair, yb, True, 300)
    _same(gx.mul(gy), rx.mul(ry), "batched mul")
    _same(gx.mul(wb), rx.mul(wb), "batched mul plain (encoded)")
    _same(gx.mul(wb[0]), rx.mul(wb[0]), "batched mul plain (constants)")
    _same(gx.add(wb), rx.add(wb), "batched add plain")


def test_reductions_products_rearrangement(pair):
    x = _vals((3, 4), 9)
    ga, ra = _enc(pair, x, seed=1)
    for ax in (0, 1, None):
        _same(ga.sum(ax), ra.sum(ax), f"sum {ax}")
    xb = _vals((8, 2, 3), 10)
    gb, rb = _enc(pair, xb, True, 60)
    for ax in (0, 2, None):
        _same(gb.sum(ax), rb.sum(ax), f"batched sum {ax}")
    assert np.max(np.abs(gb.sum(0).decrypt() - xb.sum(0))) < 1e-2
    A, B, M = _vals((2, 3), 11), _vals((3, 4), 12), _vals((3, 5), 13)
    (gA, rA), (gB, rB) = _enc(pair, A, seed=100), _enc(pair, B, seed=200)
    _same(gA.dot(gB), rA.dot(rB), "matmul")
    _same(gA.mm_plain(M), rA.mm_plain(M), "mm_plain")
    assert np.max(np.abs(gA.mm_plain(M).decrypt() - A @ M)) < 1e-2
    _same(gb.sum(2).mm_plain(M[:2, :]), rb.sum(2).mm_plain(M[:2, :]), "batched linear layer")
    x3 = _vals((2, 3, 4), 14)
    g3, r3 = _enc(pair, x3, seed=300)
    _same(g3.transpose((2, 0, 1)), r3.transpose((2, 0, 1)), "transpose")
    _same(g3.reshape((6, 4)), r3.reshape((6, 4)), "reshape")
    low_g, low_r = g3.mul(1.0), r3.mul(1.0)
    _same(g3.mul(low_g), r3.mul(low_r), "level matching")


def test_array_errors(pair):
    g = pair.g
    t = tk.CKKSTensor.encrypt(g, _vals((4,), 1), seed=1)
    L = tk.lib()
    h = ctypes.c_void_p()
    idx = np.array([0, 9], dtype=np.uint32)
    w = np.ones(2)
    assert L.tcks_cta_combine(t.h, tk._p(idx), tk._p(w), 2, 1, 0, ctypes.byref(h)) == -1  # index out of range
    idx = np.array([0, 1], dtype=np.uint32)
    w = np.array([1.0, 0.5])
    assert L.tcks_cta_combine(t.h, tk._p(idx), tk._p(w), 2, 1, 0, ctypes.byref(h)) != 0  # non-integer, mode 0
    w = np.array([1e300, 1.0])
    assert tk.lib().tcks_cta_combine(t.h, tk._p(idx), tk._p(w), 2, 1, 1, ctypes.byref(h)) != 0  # overflow
    u = tk.CKKSTensor.encrypt(g, _vals((3,), 2), seed=2)
    assert L.tcks_cta_binary(tk.TCKS_CTA_ADD, t.h, u.h, ctypes.byref(h)) != 0  # different lengths
    v = tk.CKKSTensor.encrypt(g, _vals((4,), 3), seed=3).mul(2.0)
    with pytest.raises(tk.TcksError) as e:
        tk.check(L.tcks_cta_binary(tk.TCKS_CTA_ADD, t.h, v.h, ctypes.byref(h)))
    assert e.value.name == "LEVEL_MISMATCH"
    with pytest.raises(tk.TcksError) as e:
        tk.check(L.tcks_cta_sum_slots(t.h, 64, ctypes.byref(h)))  # no key for steps 8..32
    assert e.value.name == "NO_GALOIS_KEY"
    assert L.tcks_cta_encrypt(g.h, tk._p(np.zeros(1)), 0, 1, 0, 0, ctypes.byref(h)) != 0  # empty
