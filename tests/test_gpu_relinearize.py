"""Enc x enc without automatic relinearization (§2.1: the context relinearizes after a product only
when asked to): tcks_mul returns the three-component product (d0, d1, d2), tcks_relinearize turns it
into the two-component ciphertext. Bit-exact against the oracle on identical keys and ciphertexts,
with and without the automatic rescale; the operations defined on three components (element-wise
ops, plain products, rescale, mod-switch, decryption, export) match the oracle's; the others refuse
them."""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import Pair, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu

CHAINS = {
    "C1": (12, [36, 36, 36, 37], 2.0 ** 30),
    "C2": (13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26),
    "C4": (14, [60, 40, 40, 60], 2.0 ** 40),
}


@pytest.fixture(scope="module", params=sorted(CHAINS))
def pair(request):
    log_n, bits, scale = CHAINS[request.param]
    p = Pair(log_n, bits, scale, flags=0, galois=[1])
    x, y = inputs.uniform_slots(p.o.slots, 61), inputs.uniform_slots(p.o.slots, 62)
    cx, cy = p.o.encrypt_values(x, 63), p.o.encrypt_values(y, 64)
    return p, x, y, cx, cy


def test_mul_then_relinearize(pair):
    p, x, y, cx, cy = pair
    o, g = p.o, p.g
    g.set_flags(0)
    prod = p.import_ct(cx).mul(p.import_ct(cy))
    assert prod.size == 3
    ref3 = o.mul(cx, cy, relin=False, rescale=False)
    assert_ct_equal(prod, ref3, "three-component product")
    assert np.array_equal(g.decrypt(prod).export(), o.decrypt(ref3).data)
    prod.relinearize_()
    assert prod.size == 2
    assert_ct_equal(prod, o.relinearize_ct(ref3), "relinearized")
    g.set_flags(tk.TCKS_AUTO_RELIN)
    try:
        assert np.array_equal(prod.export(), p.import_ct(cx).mul(p.import_ct(cy)).export())
    finally:
        g.set_flags(0)
    prod.relinearize_()  # a two-component ciphertext is left as it is
    assert_ct_equal(prod, o.relinearize_ct(ref3), "relinearized twice")


def test_mul_auto_rescale_without_relin(pair):
    p, x, y, cx, cy = pair
    o, g = p.o, p.g
    g.set_flags(tk.TCKS_AUTO_RESCALE)
    try:
        prod = p.import_ct(cx).mul(p.import_ct(cy))
    finally:
        g.set_flags(0)
    ref = o.mul(cx, cy, relin=False, rescale=True)
    assert prod.size == 3
    assert_ct_equal(prod, ref, "rescaled three-component product")
    prod.relinearize_()
    assert_ct_equal(prod, o.relinearize_ct(ref), "rescaled, then relinearized")


def test_three_component_elementwise(pair):
    p, x, y, cx, cy = pair
    o, g = p.o, p.g
    ref3 = o.mul(cx, cy, relin=False, rescale=False)
    g3 = g.ct_import(ref3.data, ref3.scale)
    assert g3.size == 3 and np.array_equal(g3.export(), ref3.data)
    two = o.mul_plain(cx, o.encode(inputs.uniform_slots(o.slots, 65)))  # a two-component operand at the same scale
    two = oracle.Ct(two.data, two.level, ref3.scale)
    g2 = p.import_ct(two)
    assert_ct_equal(g3.add(g2), o.add(ref3, two), "add 3 + 2")
    assert_ct_equal(g2.add(g3), o.add(two, ref3), "add 2 + 3")
    assert_ct_equal(g3.sub(g2), o.sub(ref3, two), "sub 3 - 2")
    assert_ct_equal(g2.sub(g3), o.sub(two, ref3), "sub 2 - 3")
    assert_ct_equal(g3.add(g3), o.add(ref3, ref3), "add 3 + 3")
    assert_ct_equal(g3.negate(), o.negate(ref3), "negate")
    pt = o.encode(inputs.uniform_slots(o.slots, 66))
    assert_ct_equal(g3.mul_plain(p.import_pt(pt)), o.mul_plain(ref3, pt), "mul_plain")
    small = min(1.0, 2.0 ** 40 / ref3.scale)  # keeps |scale m_i| below 2^62 at the product's scale
    pts = o.encode(inputs.uniform_slots(o.slots, 67) * small, scale=ref3.scale)
    assert_ct_equal(g3.add_plain(p.import_pt(pts)), o.add_plain(ref3, pts), "add_plain")
    assert_ct_equal(g3.sub_plain(p.import_pt(pts)), o.sub_plain(ref3, pts), "sub_plain")
    low = g.ct_import(ref3.data, ref3.scale).mod_switch_(o.L - 1)
    assert_ct_equal(low, oracle.Ct(np.ascontiguousarray(ref3.data[:, :o.L - 1]), o.L - 1, ref3.scale), "mod switch")
    assert_ct_equal(g.ct_import(ref3.data, ref3.scale).rescale_(), o.rescale(ref3), "rescale")


def test_three_component_refused(pair):
    p, x, y, cx, cy = pair
    o, g = p.o, p.g
    ref3 = o.mul(cx, cy, relin=False, rescale=False)
    g3 = g.ct_import(ref3.data, ref3.scale)
    g2 = p.import_ct(cx)
    for name, call in (("rotate", lambda: g3.rotate(1)), ("mul", lambda: g3.mul(g2)), ("mul", lambda: g2.mul(g3)),
                       ("sum", lambda: g3.sum(4)), ("serialize", lambda: g3.serialize()),
                       ("dot_plain", lambda: g3.dot_plain(np.ones(4), 4))):
        with pytest.raises(tk.TcksError) as e:
            call()
        assert e.value.name == "INVALID_ARG", name
    assert g3.size == 3 and np.array_equal(g3.export(), ref3.data)  # untouched
