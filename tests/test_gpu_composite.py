"""Composite operations on the GPU versus the oracle: sum, dot, dot_plain (§3.1), vector x plain
matrix (§3.1), im2col convolution (§3.2). Bit-exact where both sides hold identical plaintexts."""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import Pair, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p40():
    """N=4096 with 40-bit primes and scale 2^40 (rescale keeps the scale near 2^40)."""
    p = Pair(12, [55, 40, 40, 56], 2.0 ** 40)
    p.add_galois(p.o.sum_steps())
    return p


def test_sum_dot_parity(p40):
    o, g = p40.o, p40.g
    n = 300
    x = np.zeros(o.slots)
    y = np.zeros(o.slots)
    x[:n], y[:n] = inputs.uniform_slots(n, 5), inputs.uniform_slots(n, 6)
    cx, cy = o.encrypt_values(x, 31), o.encrypt_values(y, 32)
    gx, gy = p40.import_ct(cx), p40.import_ct(cy)
    assert_ct_equal(gx.sum(n), o.sum(cx, n), "sum")
    assert_ct_equal(gx.dot(gy, n), o.dot(cx, cy, n), "dot")
    w = y[:n]
    # dot_plain encodes w on each side: bit-exact when the two encodings agree (checked first)
    assert np.array_equal(g.encode(w, level=cx.level).export(), o.encode(w, level=cx.level).data)
    got = gx.dot_plain(w)
    assert_ct_equal(got, o.dot_plain(cx, w, n), "dot_plain")
    assert np.max(np.abs(g.decrypt_values(got) - x @ y)) < 1e-6


@pytest.mark.parametrize("n,m", [(16, 8), (64, 10), (256, 64)])
def test_vecmat_parity(n, m):
    p = Pair(12, [55, 40, 40, 56], 2.0 ** 40)
    o, g = p.o, p.g
    p.add_galois(o.vecmat_steps(n))
    v = np.zeros(o.slots)
    v[:n] = inputs.uniform_slots(n, 7)
    ct = o.encrypt_values(v, 41)
    M = inputs.random_matrix(n, m, 8, 0.5)
    diags = o.encode_matrix(M, ct.level)
    ref = o.vecmat(ct, diags, n, m)
    limbs = np.ascontiguousarray(np.stack([d.data for d in diags]))
    gm = g.matrix_import(limbs, n, m, diags[0].scale)
    got = p.import_ct(ct).vecmat_plain(gm)
    assert_ct_equal(got, ref, "vecmat")
    # the GPU's own encoding of the diagonals matches the oracle's
    gm2 = g.matrix_encode(M, level=ct.level)
    assert_ct_equal(p.import_ct(ct).vecmat_plain(gm2), ref, "vecmat (GPU-encoded matrix)")
    out = g.decrypt_values(got)
    assert np.max(np.abs(out[:m] - v[:n] @ M)) < 1e-5
    assert np.max(np.abs(out[m:])) < 1e-5


@pytest.mark.parametrize("n,m", [(16, 8), (64, 10), (256, 64)])
def test_vecmat_double_hoisted_parity(n, m):
    """TCKS_DOUBLE_HOIST: the ModDown once after the rotation sum, bit-exact against the oracle's
    double-hoisted product, with the diagonals imported from the oracle or encoded on the GPU, one
    ciphertext or a batch."""
    p = Pair(12, [55, 40, 40, 56], 2.0 ** 40)
    o, g = p.o, p.g
    p.add_galois(o.vecmat_steps(n))
    M = inputs.random_matrix(n, m, 8, 0.5)
    cts = []
    for i in range(3):
        v = np.zeros(o.slots)
        v[:n] = inputs.uniform_slots(n, 70 + i)
        cts.append((v, o.encrypt_values(v, 410 + i)))
    level = cts[0][1].level
    ext = o.encode_matrix_ext(M, level)
    gm = g.matrix_import_ext(ext, n, m, o.scale)
    gm2 = g.matrix_encode(M, level=level)
    plain_only = g.matrix_import(np.ascontiguousarray(ext[:, :level]), n, m, o.scale)
    g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_DOUBLE_HOIST)
    try:
        refs = [o.vecmat_dh(ct, ext, n, m) for _, ct in cts]
        for (v, ct), ref in zip(cts, refs):
            got = p.import_ct(ct).vecmat_plain(gm)
            assert_ct_equal(got, ref, "vecmat (double hoisted)")
            assert_ct_equal(p.import_ct(ct).vecmat_plain(gm2), ref, "vecmat (double hoisted, GPU-encoded)")
            out = g.decrypt_values(got)
            assert np.max(np.abs(out[:m] - v[:n] @ M)) < 1e-5
        outs = gm.vecmat_batch([p.import_ct(ct) for _, ct in cts])
        for got, ref in zip(outs, refs):
            assert_ct_equal(got, ref, "vecmat batch (double hoisted)")
        with pytest.raises(tk.TcksError) as e:
            p.import_ct(cts[0][1]).vecmat_plain(plain_only)
        assert e.value.name == "UNSUPPORTED"
        g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_DOUBLE_HOIST | tk.TCKS_MERGED_RESCALE)
        for (v, ct) in cts:  # the ModDown and the rescale in one rounding
            assert_ct_equal(p.import_ct(ct).vecmat_plain(gm), o.vecmat_dh(ct, ext, n, m, merged=True),
                            "vecmat (double hoisted, merged rescale)")
    finally:
        g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE)


@pytest.mark.parametrize("n,m", [(16, 4), (64, 10), (256, 64), (32, 4), (16, 8)])
def test_vecmat_rect_parity(n, m):
    """Rectangular (hybrid) diagonals: with the oracle's encodings imported, bit-exact against the
    oracle's rectangular schedule with either key-switch schedule, single and batched; the
    rotate-and-add chains after the sum have two, three and one steps (the steps alternate between
    the output and a scratch, an odd chain takes its first in place). Diagonals
    encoded on the GPU decrypt to the same v M (their every slot is non-zero, so the FFT and the
    oracle's direct sum round an encoding coefficient differently at near ties far more often than
    for the square form, reading A9)."""
    p = Pair(12, [55, 40, 40, 56], 2.0 ** 40)
    o, g = p.o, p.g
    p.add_galois(o.vecmat_rect_steps(n, m))
    M = inputs.random_matrix(n, m, 9, 0.5)
    cts = []
    for i in range(2):
        v = np.zeros(o.slots)
        v[:n] = inputs.uniform_slots(n, 80 + i)
        cts.append((v, o.encrypt_values(v, 510 + i)))
    level = cts[0][1].level
    diags = o.encode_matrix_rect(M, level)
    ext = o.encode_matrix_rect_ext(M, level)
    gm = g.matrix_import_rect(ext, n, m, o.scale)
    genc = g.matrix_encode_rect(M, level=level)
    for flags, kw in ((tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE, {"diags": diags}),
                      (tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_DOUBLE_HOIST, {"diags_ext": ext}),
                      (tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_DOUBLE_HOIST | tk.TCKS_MERGED_RESCALE,
                       {"diags_ext": ext, "merged": True})):
        g.set_flags(flags)
        try:
            refs = [o.vecmat_rect(ct, n, m, **kw) for _, ct in cts]
            for (v, ct), ref in zip(cts, refs):
                got = p.import_ct(ct).vecmat_plain(gm)
                assert_ct_equal(got, ref, f"vecmat rect {list(kw)}")
                assert np.max(np.abs(g.decrypt_values(got)[:m] - v[:n] @ M)) < 1e-5
                own = g.decrypt_values(p.import_ct(ct).vecmat_plain(genc))
                assert np.max(np.abs(own[:m] - v[:n] @ M)) < 1e-5
            for got, ref in zip(gm.vecmat_batch([p.import_ct(ct) for _, ct in cts]), refs):
                assert_ct_equal(got, ref, "vecmat rect batch")
        finally:
            g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE)


@pytest.mark.parametrize("chain", ["40-bit", "narrow"])
def test_rotate_sum_hoisted_parity(chain):
    """The hoisted rotation sum (one ModUp, one ModDown) bit-exact against the oracle, 64-bit and 32-bit
    words, and within the key-switch noise of the plain sum of rotations."""
    if chain == "40-bit":
        p = Pair(12, [55, 40, 40, 56], 2.0 ** 40)
    else:
        p = Pair(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26)
    o, g = p.o, p.g
    steps = [64 * b for b in range(1, 8)]
    p.add_galois(steps)
    z = inputs.uniform_slots(o.slots, 33)
    ct = o.encrypt_values(z, 90)
    ref = o.rotsum_dh(ct, steps)
    got = p.import_ct(ct).rotate_sum_hoisted(steps)
    assert_ct_equal(got, ref, "rotate_sum_hoisted")
    plain = z + sum(np.roll(z, -s) for s in steps)
    # scale 2^40 vs 2^26: the fresh-encryption noise of the 8 summed copies, about 4e-4 per slot each at 2^26
    assert np.max(np.abs(g.decrypt_values(got) - plain)) < (1e-6 if chain == "40-bit" else 1e-2)
    with pytest.raises(tk.TcksError) as e:
        p.import_ct(ct).rotate_sum_hoisted([0])
    assert e.value.name == "INVALID_ARG"


def test_conv_parity():
    p = Pair(13, [40, 30, 30, 41], 2.0 ** 30)
    o, g = p.o, p.g
    img = inputs.mnist_like_image(3)
    v, W = oracle.OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    p.add_galois(o.conv_steps(49, W))
    ct = o.encrypt_values(v, 51)
    ker = inputs.cnn_weights(4)["conv_w"][1]
    kpt = o.encode(o.kernel_slots(ker, W), level=ct.level)
    ref = o.conv2d_im2col_pt(ct, kpt, 49, W)
    assert_ct_equal(p.import_ct(ct).conv2d_im2col_pt(p.import_pt(kpt), 49, W), ref, "conv (imported kernel)")
    assert_ct_equal(p.import_ct(ct).conv2d_im2col(ker, W), ref, "conv (GPU-encoded kernel)")
    out = g.decrypt_values(p.import_ct(ct).conv2d_im2col(ker, W))
    want = np.array([np.sum(img[3 * (w // 8):3 * (w // 8) + 7, 3 * (w % 8):3 * (w % 8) + 7] * ker.reshape(7, 7))
                     for w in range(64)])
    assert np.max(np.abs(out[:64] - want)) < 1e-3
