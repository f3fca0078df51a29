"""Pins of the oracle's CKKS layer (encoding, keys, homomorphic ops, schedules).

Independent references used here: a numpy-FFT derivation of the canonical embedding, the closed form
of encoding a constant, a big-integer (non-RNS) re-derivation of every exact op for tiny N
(tests/tiny_ckks.py), exact algebraic invariants of automorphisms, a worst-case key-switch noise
bound, and decrypt(op(Enc(x))) against FP64 arithmetic on the same values.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleCKKS
from paper_2104_03152_gb300 import inputs
from tiny_ckks import TinyCKKS, primitive_2n_roots


@pytest.fixture(scope="module")
def c1():
    """Config C1 chain: N=4096, [36,36,36 | 37], scale 2^30."""
    o = OracleCKKS(12, [36, 36, 36, 37], 2.0 ** 30).keygen()
    o.gen_galois_keys([1, 2, 5, 100, 2047] + o.sum_steps())
    return o


def fft_encode(z, n, scale):
    """Canonical-embedding inverse via numpy: slot j sits at index t_j = (5^j mod 2N - 1)/4 of a size
    N/2 transform (zeta^(5^j) = zeta * omega^t_j, omega = zeta^4); w_k zeta^k = (1/n) sum_t y_t
    omega^(-tk) (numpy's forward FFT / n); m_k = Re w_k, m_{k+N/2} = Im w_k."""
    half = n // 2
    y = np.zeros(half, dtype=np.complex128)
    g = 1
    for j in range(half):
        y[(g - 1) // 4] = z[j] if j < len(z) else 0.0
        g = g * 5 % (2 * n)
    wz = np.fft.fft(y) / half
    k = np.arange(half)
    w = wz * np.exp(-1j * np.pi * k / n)
    return scale * np.concatenate([w.real, w.imag])


def fft_decode(p, n, scale, n_out):
    half = n // 2
    w = (p[:half] + 1j * p[half:]) / scale
    k = np.arange(half)
    out = np.fft.ifft(w * np.exp(1j * np.pi * k / n)) * half  # sum_k (w_k zeta^k) omega^(+tk)
    z = np.zeros(n_out)
    g = 1
    for j in range(n_out):
        z[j] = out[(g - 1) // 4].real
        g = g * 5 % (2 * n)
    return z


# ------------------------------------------------------------------------------ encoding ----

def test_encode_constant_closed_form(c1):
    """P6: a constant vector encodes to coefficient 0 = round(scale * c), every other coefficient 0."""
    for c in (0.5, -1.25, 3.0):
        pt, pre = c1.encode(np.full(c1.slots, c), want_pre=True)
        coeffs = c1.crt_compose(c1.intt_limbs(pt.data, pt.level), pt.level)
        assert coeffs[0] == round(c * 2 ** 30)
        assert all(x == 0 for x in coeffs[1:])


def test_encode_matches_fft_derivation(c1):
    z = inputs.uniform_slots(c1.slots, 1)
    pt, pre = c1.encode(z, want_pre=True)
    ref = fft_encode(z, c1.N, 2.0 ** 30)
    assert np.max(np.abs(pre - ref)) / 2 ** 30 < 1e-12
    # a short, zero-padded input
    z2 = inputs.uniform_slots(37, 2)
    _, pre2 = c1.encode(z2, want_pre=True)
    assert np.max(np.abs(pre2 - fft_encode(z2, c1.N, 2.0 ** 30))) / 2 ** 30 < 1e-12


def test_decode_matches_fft_and_roundtrip(c1):
    z = inputs.uniform_slots(c1.slots, 3)
    pt = c1.encode(z)
    dec = c1.decode(pt)
    coeffs = np.array(c1.crt_compose(c1.intt_limbs(pt.data, pt.level), pt.level), dtype=np.float64)
    assert np.max(np.abs(dec - fft_decode(coeffs, c1.N, 2.0 ** 30, c1.slots))) < 1e-12
    # rounding each coefficient moves a slot by at most N/2 * 0.5 / scale
    assert np.max(np.abs(dec - z)) < c1.N / 4 / 2 ** 30


def test_encode_overflow_and_sizes(c1):
    with pytest.raises(OverflowError):
        c1.encode(np.full(4, 1e10), scale=2.0 ** 40)
    with pytest.raises(ValueError):
        c1.encode(np.zeros(c1.slots + 1))


# -------------------------------------------------------------------------- keys / sampler ----

def test_sampler_distributions(c1):
    """s ternary, pk and key 'a' parts uniform, errors CBD(21): checked through the keys themselves."""
    s_coeff = c1.intt_limbs(c1.s[:1], 1)[0]
    q0 = c1.q[0]
    vals = np.array([int(v) if int(v) <= q0 // 2 else int(v) - q0 for v in s_coeff])
    assert set(np.unique(vals)) <= {-1, 0, 1}
    frac = [np.mean(vals == t) for t in (-1, 0, 1)]
    assert all(abs(f - 1 / 3) < 0.04 for f in frac)
    # pk0 + pk1 * s = e (CBD, |e| <= 21, variance 10.5)
    d = c1.decrypt(oracle.Ct(c1.pk[:, :1].copy(), 1, 1.0))
    e = c1.crt_compose(c1.intt_limbs(d.data, 1), 1)
    e = np.array(e)
    assert np.max(np.abs(e)) <= 21
    assert abs(np.var(e) - 10.5) < 1.5
    a = c1.pk[1, 0].astype(np.float64)
    assert abs(np.mean(a) / q0 - 0.5) < 0.02


def test_key_trimming_is_subset():
    o = OracleCKKS(10, [30, 30, 30, 30, 31], 2.0 ** 25).keygen()
    full = o.gen_galois_key(3, 4).data.copy()
    trim = o.gen_galois_key(3, 2).data
    # trimmed key = digits j < 2, limbs q_0, q_1 and P of the full key
    assert np.array_equal(trim[:, :, :2], full[:2, :, :2])
    assert np.array_equal(trim[:, :, 2], full[:2, :, 4])


# ------------------------------------------------------------- big-integer re-derivation ----

@pytest.fixture(scope="module")
def tiny():
    o = OracleCKKS(4, [24, 24, 24, 26], 2.0 ** 10).keygen()
    o.gen_galois_keys([1, 3])
    # roots found independently of the oracle (smallest of all primitive 2N-th roots)
    t = TinyCKKS(o.N, o.q, [primitive_2n_roots(q, o.N)[0] for q in o.q])
    return o, t


def _rand_ct(o, level, seed):
    lim = inputs.random_limbs(o.q[:level], o.N, seed, polys=2)
    return oracle.Ct(np.ascontiguousarray(lim), level, 1.0)


def test_tiny_tensor_relin_rescale(tiny):
    """P4/P5: tensor product, relinearization and rescale equal the big-integer definitions."""
    o, t = tiny
    lvl = 3
    a, b = _rand_ct(o, lvl, 1), _rand_ct(o, lvl, 2)
    idx = list(range(lvl))
    Q = math.prod(o.q[:lvl])
    A = [t.to_int(a.data[p], idx) for p in range(2)]
    B = [t.to_int(b.data[p], idx) for p in range(2)]
    d3, _, _ = o.tensor(a, b)
    from tiny_ckks import negacyclic_mul
    d0 = negacyclic_mul(A[0], B[0], Q)
    d1 = [(x + y) % Q for x, y in zip(negacyclic_mul(A[0], B[1], Q), negacyclic_mul(A[1], B[0], Q))]
    d2 = negacyclic_mul(A[1], B[1], Q)
    for p, ref in enumerate((d0, d1, d2)):
        assert t.to_int(d3[p], idx) == ref
    rel = o.relinearize(d3, lvl, 1.0)
    k0, k1 = t.keyswitch(d2, lvl, o.rlk.data, o.rlk.level)
    assert t.to_int(rel.data[0], idx) == [(x + y) % Q for x, y in zip(d0, k0)]
    assert t.to_int(rel.data[1], idx) == [(x + y) % Q for x, y in zip(d1, k1)]
    rs = o.rescale(rel)
    for p in range(2):
        assert t.to_int(rs.data[p], idx[:-1]) == t.rescale(t.to_int(rel.data[p], idx), lvl)


def test_tiny_merged_relin_rescale(tiny):
    """A25: relinearization and rescale taken as one rounding equal round((P d + u) / (P q_last)) mod
    Q_{level-1} in big integers, u the key-switch inner product over Q P before any division."""
    o, t = tiny
    lvl = 3
    a, b = _rand_ct(o, lvl, 5), _rand_ct(o, lvl, 6)
    d3, _, _ = o.tensor(a, b)
    idx = list(range(lvl))
    Q = math.prod(o.q[:lvl])
    P, ql = t.P, o.q[lvl - 1]
    d = [t.to_int(d3[p], idx) for p in range(3)]
    u = t.keyswitch_u(d[2], lvl, o.rlk.data, o.rlk.level)
    got = o.relinearize_rescale(d3, lvl, 1.0)
    assert got.level == lvl - 1
    for p in range(2):
        ref = [t.round_div((P * x + y) % (Q * P), P * ql) % (Q // ql) for x, y in zip(d[p], u[p])]
        assert t.to_int(got.data[p], idx[:-1]) == ref


def test_tiny_rotation(tiny):
    """P5: rotation = coefficient automorphism, then key switch, in big integers."""
    o, t = tiny
    lvl = 2
    a = _rand_ct(o, lvl, 5)
    idx = list(range(lvl))
    Q = math.prod(o.q[:lvl])
    for step in (1, 3):
        g = o.galois_elt(step)
        A = [t.automorphism(t.to_int(a.data[p], idx), g, Q) for p in range(2)]
        k0, k1 = t.keyswitch(A[1], lvl, o.galois[step].data, o.galois[step].level)
        r = o.rotate(a, step)
        assert t.to_int(r.data[0], idx) == [(x + y) % Q for x, y in zip(A[0], k0)]
        assert t.to_int(r.data[1], idx) == k1


def test_tiny_three_component_ciphertext(tiny):
    """An unrelinearized product (c0, c1, c2): decryption c0 + c1 s + c2 s^2, the rescale of every
    component, mul_plain and the mixed-size sum, each against the big-integer definitions."""
    o, t = tiny
    from tiny_ckks import negacyclic_mul
    lvl = 3
    idx = list(range(lvl))
    Q = math.prod(o.q[:lvl])
    c3 = oracle.Ct(np.ascontiguousarray(inputs.random_limbs(o.q[:lvl], o.N, 31, polys=3)), lvl, 1.0)
    C = [t.to_int(c3.data[p], idx) for p in range(3)]
    S = t.to_int(o.s[:lvl], idx)
    S2 = negacyclic_mul(S, S, Q)
    c1s, c2s2 = negacyclic_mul(C[1], S, Q), negacyclic_mul(C[2], S2, Q)
    want = [(a + b + c) % Q for a, b, c in zip(C[0], c1s, c2s2)]
    assert t.to_int(o.decrypt(c3).data, idx) == want
    rs = o.rescale(c3)
    assert rs.data.shape[0] == 3
    for p in range(3):
        assert t.to_int(rs.data[p], idx[:-1]) == t.rescale(C[p], lvl)
    pt = oracle.Pt(np.ascontiguousarray(inputs.random_limbs(o.q[:lvl], o.N, 32, polys=1)[0]), lvl, 1.0)
    Pt_ = t.to_int(pt.data, idx)
    mp = o.mul_plain(c3, pt)
    for p in range(3):
        assert t.to_int(mp.data[p], idx) == negacyclic_mul(C[p], Pt_, Q)
    ap = o.add_plain(c3, pt)
    assert t.to_int(ap.data[0], idx) == [(a + b) % Q for a, b in zip(C[0], Pt_)]
    assert np.array_equal(ap.data[1:], c3.data[1:])
    c2 = _rand_ct(o, lvl, 33)
    D = [t.to_int(c2.data[p], idx) for p in range(2)]
    sm = o.sub(c2, c3)  # a missing third component is zero
    assert sm.data.shape[0] == 3
    for p in range(3):
        other = D[p] if p < 2 else [0] * o.N
        assert t.to_int(sm.data[p], idx) == [(a - b) % Q for a, b in zip(other, C[p])]


def test_three_component_product():
    """The product without relinearization: its decryption is the product of the operands'
    decryptions, limb by limb in NTT form (exactly: (a0 + a1 s)(b0 + b1 s) = d0 + d1 s + d2 s^2);
    relinearizing it gives the relinearized product bit for bit; rescaled before relinearization it
    still decrypts to x y. (The rescale's rounding error in c2 is multiplied by s^2 at decryption, so
    the chain's primes match the scale here, 40-bit primes at 2^40, as a user of this order would
    choose them.)"""
    o = OracleCKKS(12, [60, 40, 40, 60], 2.0 ** 40).keygen()
    x, y = inputs.uniform_slots(o.slots, 41), inputs.uniform_slots(o.slots, 42)
    a, b = o.encrypt_values(x, 43), o.encrypt_values(y, 44)
    d3 = o.mul(a, b, relin=False, rescale=False)
    assert d3.data.shape == (3, o.L, o.N) and d3.scale == a.scale * b.scale
    ma, mb, m3 = o.decrypt(a).data, o.decrypt(b).data, o.decrypt(d3).data
    for l in range(o.L):
        q = o.q[l]
        want = [int(u) * int(v) % q for u, v in zip(ma[l], mb[l])]
        assert np.array_equal(m3[l], np.array(want, dtype=np.uint64)), l
    rel = o.relinearize_ct(d3)
    assert np.array_equal(rel.data, o.mul(a, b, relin=True, rescale=False).data)
    tol = 1e-3  # the products' noise at scale 2^30, as for the relinearized product
    assert np.max(np.abs(o.decrypt_values(d3) - x * y)) < tol
    r3 = o.mul(a, b, relin=False, rescale=True)
    assert r3.data.shape == (3, o.L - 1, o.N)
    assert np.max(np.abs(o.decrypt_values(r3) - x * y)) < tol
    assert np.max(np.abs(o.decrypt_values(o.relinearize_ct(r3)) - x * y)) < tol


# --------------------------------------------------------------------- exact invariants ----

def test_automorphism_ntt_equals_coefficient_map(c1):
    """P7: the NTT-domain permutation equals the coefficient map a(X) -> a(X^g)."""
    L = oracle.lib()
    q = c1.q[0]
    a = inputs.random_limbs([q], c1.N, 9)[0, 0].copy()
    fa = a.copy()
    L.orc_ntt_limb(c1._ctx, oracle.ckks.P(fa), 0)
    for step in (1, 5, 2047):
        g = c1.galois_elt(step)
        ca = np.zeros_like(a)
        L.orc_automorphism_coeff(c1._ctx, oracle.ckks.P(a), q, g, oracle.ckks.P(ca))
        L.orc_ntt_limb(c1._ctx, oracle.ckks.P(ca), 0)
        na = np.zeros_like(fa)
        L.orc_automorphism_ntt(c1._ctx, oracle.ckks.P(fa), 1, g, oracle.ckks.P(na))
        assert np.array_equal(ca, na)


def test_automorphism_composition_and_rotation(c1):
    """P7: tau_a(tau_b(x)) = tau_(ab)(x) exactly, and tau_(5^k) rotates slots left by k."""
    L = oracle.lib()
    z = inputs.uniform_slots(c1.slots, 4)
    pt = c1.encode(z, level=1)
    ga, gb = c1.galois_elt(2), c1.galois_elt(5)
    t1 = np.zeros_like(pt.data)
    t2 = np.zeros_like(pt.data)
    L.orc_automorphism_ntt(c1._ctx, oracle.ckks.P(pt.data), 1, gb, oracle.ckks.P(t1))
    L.orc_automorphism_ntt(c1._ctx, oracle.ckks.P(t1), 1, ga, oracle.ckks.P(t2))
    t3 = np.zeros_like(pt.data)
    L.orc_automorphism_ntt(c1._ctx, oracle.ckks.P(pt.data), 1, ga * gb % (2 * c1.N), oracle.ckks.P(t3))
    assert np.array_equal(t2, t3)
    assert ga * gb % (2 * c1.N) == c1.galois_elt(7)
    dec = c1.decode(oracle.Pt(t1, 1, pt.scale))
    assert np.max(np.abs(dec - np.roll(z, -5))) < 1e-6


def test_hoisted_equals_plain_rotation(c1):
    """P9: rotating from hoisted (balanced) digits is bit-identical to the plain rotation."""
    ct = c1.encrypt_values(inputs.uniform_slots(c1.slots, 1), seed=11)
    outs = c1.rotate_hoisted(ct, [1, 2, 100])
    for st, h in zip([1, 2, 100], outs):
        assert np.array_equal(h.data, c1.rotate(ct, st).data)


def test_keyswitch_noise_bound(c1):
    """P10: decrypt(KS_{s'->s}(x)) - x*s' has infinity norm at most
    level*N*21*max(q_j)/(2P) + (N + 1)/2 (digits |D_j| <= q_j/2, |e| <= 21, ModDown rounding <= 1/2,
    s ternary)."""
    lvl = 3
    x = inputs.random_limbs(c1.q[:lvl], c1.N, 12)[0]
    ks = c1.keyswitch(x, lvl, c1.rlk)
    s2 = np.array([[int(v) * int(v) % c1.q[l] for v in c1.s[l]] for l in range(lvl)], dtype=np.uint64)
    dec = c1.decrypt(oracle.Ct(np.ascontiguousarray(ks), lvl, 1.0)).data
    diff = np.array([[(int(dec[l, i]) - int(x[l, i]) * int(s2[l, i])) % c1.q[l] for i in range(c1.N)]
                     for l in range(lvl)], dtype=np.uint64)
    err = c1.crt_compose(c1.intt_limbs(diff, lvl), lvl)
    bound = lvl * c1.N * 21 * max(c1.q[:lvl]) / (2 * c1.Pspecial) + (c1.N + 1) / 2
    assert max(abs(e) for e in err) <= bound
    assert max(abs(e) for e in err) > 0


# ------------------------------------------------------------- decrypt(op(Enc x)) ~ op(x) ----

def test_ops_against_fp64(c1):
    """P11 on C1's chain (scale 2^30): every element-wise op decrypts to the FP64 result."""
    x = inputs.uniform_slots(c1.slots, 1)
    y = inputs.uniform_slots(c1.slots, 2)
    cx, cy = c1.encrypt_values(x, seed=21), c1.encrypt_values(y, seed=22)
    tol = 2e-4  # fresh-encryption noise: ~sqrt(N) * 300 / 2^30 per slot
    dec = lambda ct: c1.decrypt_values(ct)
    assert np.max(np.abs(dec(c1.add(cx, cy)) - (x + y))) < tol
    assert np.max(np.abs(dec(c1.sub(cx, cy)) - (x - y))) < tol
    assert np.max(np.abs(dec(c1.negate(cx)) + x)) < tol
    assert np.max(np.abs(dec(c1.add_plain(cx, c1.encode(y))) - (x + y))) < tol
    assert np.max(np.abs(dec(c1.sub_plain(cx, c1.encode(y))) - (x - y))) < tol
    assert np.max(np.abs(dec(c1.rescale(c1.mul_plain(cx, c1.encode(y)))) - x * y)) < 1e-3
    m = c1.mul(cx, cy)
    assert m.level == 2
    assert np.max(np.abs(dec(m) - x * y)) < 1e-3
    assert np.max(np.abs(dec(c1.square(cx)) - x * x)) < 1e-3
    assert np.max(np.abs(dec(c1.rotate(cx, 1)) - np.roll(x, -1))) < tol
    assert np.max(np.abs(dec(c1.rotate(c1.rotate(cx, 1), 5)) - np.roll(x, -6))) < tol  # P8 (composition)
    assert np.max(np.abs(dec(c1.mod_switch(cx, 1)) - x)) < tol


def test_sum_dot():
    """sum / dot / dot_plain (§3.1) on a chain whose rescale keeps the scale at 2^40 (with C1's
    36-bit primes the scale drops to 2^24 after one rescale, and summing N/2 slots multiplies the
    per-slot noise by about sqrt(N/2))."""
    o = OracleCKKS(12, [55, 40, 40, 56], 2.0 ** 40).keygen()
    o.gen_galois_keys(o.sum_steps())
    n = 300
    x = np.zeros(o.slots)
    y = np.zeros(o.slots)
    x[:n] = inputs.uniform_slots(n, 5)
    y[:n] = inputs.uniform_slots(n, 6)
    cx, cy = o.encrypt_values(x, 31), o.encrypt_values(y, 32)
    s = o.decrypt_values(o.sum(cx, n))
    assert np.max(np.abs(s - x.sum())) < 1e-6
    d = o.decrypt_values(o.dot(cx, cy, n))
    assert np.max(np.abs(d - x @ y)) < 1e-6
    dp = o.decrypt_values(o.dot_plain(cx, y[:n], n))
    assert np.max(np.abs(dp - x @ y)) < 1e-6


def test_vecmat_identity_permutation_and_random():
    """P14 and P11: vector x plain matrix with identity, permutation and random matrices."""
    o = OracleCKKS(12, [36, 36, 36, 37], 2.0 ** 30).keygen()
    n, m = 16, 8
    o.gen_galois_keys(o.vecmat_steps(n))
    v = np.zeros(o.slots)
    v[:n] = inputs.uniform_slots(n, 7)
    ct = o.encrypt_values(v, 41)
    perm = np.random.default_rng(0).permutation(n)
    Mp = np.zeros((n, m))
    for s in range(m):
        Mp[perm[s], s] = 1.0
    Mr = inputs.random_matrix(n, m, 8, 0.5)
    for M in (np.eye(n)[:, :m], Mp, Mr):
        out = o.decrypt_values(o.vecmat(ct, o.encode_matrix(M, ct.level), n, m))
        # C1's chain: the result scale after the rescale is 2^60 / q_2 ~ 2^24
        assert np.max(np.abs(out[:m] - v[:n] @ M)) < 1e-3
        assert np.max(np.abs(out[m:])) < 1e-3


def test_im2col_layout_and_delta_conv():
    """§3.2 geometry pins (28x28, 7x7, stride 3 -> 64 windows x 49 taps = 3136 slots) and P14: a
    delta kernel reproduces the selected pixel of every window."""
    img = inputs.mnist_like_image(3)
    v, W = OracleCKKS.im2col(img, 7, 7, 3, 4096)
    assert W == 64 and (28 - 7) // 3 + 1 == 8
    assert np.all(v[49 * 64:] == 0)
    assert v[10 * 64 + 9] == img[3 * 1 + 10 // 7][3 * 1 + 10 % 7]
    o = OracleCKKS(13, [40, 30, 30, 41], 2.0 ** 30).keygen()
    o.gen_galois_keys(o.conv_steps(49, W))
    ct = o.encrypt_values(v, 51)
    ker = np.zeros(49)
    ker[24] = 1.0  # centre tap
    out = o.decrypt_values(o.conv2d_im2col(ct, ker, W))
    ref = np.array([img[3 * (w // 8) + 3][3 * (w % 8) + 3] for w in range(64)])
    assert np.max(np.abs(out[:64] - ref)) < 1e-3  # noise of the 64 summed blocks
    ker2 = inputs.cnn_weights(4)["conv_w"][0]
    out2 = o.decrypt_values(o.conv2d_im2col(ct, ker2, W))
    ref2 = np.array([np.sum(img[3 * (w // 8):3 * (w // 8) + 7, 3 * (w % 8):3 * (w % 8) + 7] * ker2.reshape(7, 7))
                     for w in range(64)])
    assert np.max(np.abs(out2[:64] - ref2)) < 1e-3


# ------------------------------------------------------------ double-hoisted vector x matrix ----

def _vecmat_dh_raw(o, ct, digits, diags_ext, rows):
    """orc_vecmat_dh before the rescale (steps 1-3)."""
    keys = [o._key(k) for k in range(1, rows)]
    arrs = [np.ascontiguousarray(k.data) for k in keys]
    ptrs = (oracle.ckks._u64p * len(arrs))(*[a.ctypes.data_as(oracle.ckks._u64p) for a in arrs])
    lv = np.array([k.level for k in keys], dtype=np.uint32)
    ge = np.array([o.galois_elt(k) for k in range(1, rows)], dtype=np.uint32)
    out = np.zeros((2, ct.level, o.N), dtype=np.uint64)
    P = lambda a: a.ctypes.data_as({np.dtype(np.uint64): oracle.ckks._u64p, np.dtype(np.uint32): oracle.ckks._u32p}[a.dtype])
    oracle.lib().orc_vecmat_dh(o._ctx, P(np.ascontiguousarray(ct.data)), P(np.ascontiguousarray(digits)), ct.level,
                               rows, P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
    return out


def test_vecmat_dh_equals_bigint_definition(tiny):
    """The double-hoisted product against its big-integer definition on a tiny ring:
    out_0 = c0 d_0 + sum_k tau_k(c0) d_k + round(U_0 / P),  out_1 = c1 d_0 + round(U_1 / P),
    U_b = sum_k u_b(tau_k(c1), gk_k) d_k over Q P, with u_b the key-switch inner product before the
    division by P (TinyCKKS.keyswitch_u, pinned by the relinearization test above)."""
    o, t = tiny
    rows, lvl = 4, 3
    o.gen_galois_keys([1, 2, 3])
    ct = _rand_ct(o, lvl, 31)
    idx, idx_ext = list(range(lvl)), t.mods(lvl, with_p=True)
    Q = math.prod(o.q[:lvl])
    QP = Q * o.q[-1]
    rng = np.random.default_rng(5)
    d_int = [[int(x) for x in rng.integers(-200, 201, size=o.N)] for _ in range(rows)]
    diags_ext = np.array([t.from_int(d, idx_ext) for d in d_int], dtype=np.uint64)
    got = _vecmat_dh_raw(o, ct, o.modup(ct), diags_ext, rows)
    from tiny_ckks import negacyclic_mul
    C = [t.to_int(ct.data[p], idx) for p in range(2)]
    A0 = negacyclic_mul(C[0], [x % Q for x in d_int[0]], Q)
    A1 = negacyclic_mul(C[1], [x % Q for x in d_int[0]], Q)
    U = [[0] * o.N, [0] * o.N]
    for k in range(1, rows):
        g = o.galois_elt(k)
        c0g = t.automorphism(C[0], g, Q)
        c1g = t.automorphism(C[1], g, Q)
        A0 = [(a + b) % Q for a, b in zip(A0, negacyclic_mul(c0g, [x % Q for x in d_int[k]], Q))]
        u = t.keyswitch_u(c1g, lvl, o.galois[k].data, o.galois[k].level)
        for b in range(2):
            U[b] = [(a + x) % QP for a, x in zip(U[b], negacyclic_mul(u[b], [x % QP for x in d_int[k]], QP))]
    ref0 = [(a + t.round_div(x, o.q[-1])) % Q for a, x in zip(A0, U[0])]
    ref1 = [(a + t.round_div(x, o.q[-1])) % Q for a, x in zip(A1, U[1])]
    assert t.to_int(got[0], idx) == ref0
    assert t.to_int(got[1], idx) == ref1


def test_encode_ext_limb_is_the_same_integer_polynomial(c1):
    """The P limb of an extended encoding is the NTT mod P of the integer coefficients the data limbs
    carry (recovered by the pinned CRT composition)."""
    o = c1
    z = inputs.uniform_slots(o.slots, 3)
    ext = o.encode_ext(z, 2)
    base = o.encode(z, level=2)
    assert np.array_equal(ext[:2], base.data)
    coef = o.crt_compose(o.intt_limbs(base.data, 2), 2)
    Pq = o.q[-1]
    ref = oracle.ntt(np.array([int(c) % Pq for c in coef], dtype=np.uint64), Pq, oracle.min_psi(Pq, o.log_n))
    assert np.array_equal(ext[2], ref)


def test_vecmat_dh_decrypts_to_product_and_tracks_single_hoisting():
    """decrypt(vecmat_dh(Enc(v))) = v M within the noise bound, and within a much smaller distance of
    the single-hoisted product (the two differ only in where the division by P is rounded)."""
    o = OracleCKKS(12, [55, 40, 40, 56], 2.0 ** 40).keygen()
    n, m = 16, 8
    o.gen_galois_keys(o.vecmat_steps(n))
    v = np.zeros(o.slots)
    v[:n] = inputs.uniform_slots(n, 7)
    ct = o.encrypt_values(v, 41)
    M = inputs.random_matrix(n, m, 8, 0.5)
    dh = o.decrypt_values(o.vecmat_dh(ct, o.encode_matrix_ext(M, ct.level), n, m))
    sh = o.decrypt_values(o.vecmat(ct, o.encode_matrix(M, ct.level), n, m))
    assert np.max(np.abs(dh[:m] - v[:n] @ M)) < 1e-6
    assert np.max(np.abs(dh[m:])) < 1e-6
    assert np.max(np.abs(dh - sh)) < 1e-7


@pytest.mark.parametrize("n,m", [(16, 4), (64, 10), (256, 64)])
def test_vecmat_rect_decrypts_to_product(n, m):
    """Rectangular (hybrid) diagonals: rect_width(m) hoisted rotations plus log2(n / rect_width(m))
    rotate-and-adds; slots s < m decrypt to v M, with one ModDown per rotation or once after the sum,
    and the two readings agree closely."""
    o = OracleCKKS(12, [55, 40, 40, 56], 2.0 ** 40).keygen()
    o.gen_galois_keys(o.vecmat_rect_steps(n, m))
    v = np.zeros(o.slots)
    v[:n] = inputs.uniform_slots(n, 17)
    ct = o.encrypt_values(v, 43)
    M = inputs.random_matrix(n, m, 9, 0.5)
    ref = v[:n] @ M
    a = o.decrypt_values(o.vecmat_rect(ct, n, m, diags=o.encode_matrix_rect(M, ct.level)))
    b = o.decrypt_values(o.vecmat_rect(ct, n, m, diags_ext=o.encode_matrix_rect_ext(M, ct.level)))
    assert np.max(np.abs(a[:m] - ref)) < 1e-6
    assert np.max(np.abs(b[:m] - ref)) < 1e-6
    assert np.max(np.abs(a[:m] - b[:m])) < 1e-7
    assert len(o.vecmat_rect_steps(n, m)) < len(o.vecmat_steps(n))


def test_cnn_rect_schedule_matches_fp64():
    """The CNN with both fully connected layers by rectangular diagonals (FC2 consuming FC1's output
    as it comes, replicated with period 64) decrypts to the FP64 network as the square schedule does,
    with far fewer Galois keys."""
    o = OracleCKKS(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26).keygen()
    sq, rc = oracle.cnn_galois_steps(o), oracle.cnn_galois_steps(o, rect=True)
    assert len(rc) < len(sq) // 2
    for st, lv in rc.items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(4))
    enc = oracle.cnn_encode(o, w, rect=True)
    img = inputs.mnist_like_image(3)
    v, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, 77)
    plain = oracle.cnn_plain(img, w)
    for dh in (False, True):
        logits = o.decrypt_values(oracle.cnn_forward(o, ct, w, enc, double_hoist=dh), 10)
        assert np.max(np.abs(logits - plain)) < 5e-3


def test_rotsum_and_hoisted_conv():
    """A hoisted rotation sum (one ModDown) decrypts to the plain sum of rotations and agrees with the
    chain of single rotations within the key-switch noise; the baby-step giant-step convolution sums the
    same 64 tap positions as the rotate-and-add chain."""
    o = OracleCKKS(12, [55, 40, 40, 56], 2.0 ** 40).keygen()
    steps = [3, 17, 100, 1000]
    o.gen_galois_keys(steps)
    z = inputs.uniform_slots(o.slots, 21)
    ct = o.encrypt_values(z, 50)
    got = o.decrypt_values(o.rotsum_dh(ct, steps))
    ref = z + sum(np.roll(z, -s) for s in steps)
    assert np.max(np.abs(got - ref)) < 1e-6
    chain = ct
    for s in steps:
        chain = o.add(chain, o.rotate(ct, s))
    assert np.max(np.abs(o.decrypt_values(chain) - got)) < 1e-7
    baby, giant = OracleCKKS.conv_bsgs_steps(49, 64)
    assert baby == [64 * b for b in range(1, 8)] and giant == [512 * g for g in range(1, 8)]
    sums = sorted(b + g for b in [0] + baby for g in [0] + giant)
    assert sums == [64 * t for t in range(64)]


def test_cnn_hoisted_conv_schedule_matches_fp64():
    """The CNN with the hoisted baby-step giant-step convolution sums and rectangular FC layers decrypts to
    the FP64 network."""
    o = OracleCKKS(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26).keygen()
    steps = oracle.cnn_galois_steps(o, rect=True, conv_hoist=True)
    for st, lv in steps.items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(4))
    enc = oracle.cnn_encode(o, w, rect=True, conv_hoist=True)
    img = inputs.mnist_like_image(3)
    v, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, 77)
    logits = o.decrypt_values(oracle.cnn_forward(o, ct, w, enc, double_hoist=True), 10)
    assert np.max(np.abs(logits - oracle.cnn_plain(img, w))) < 5e-3


def test_dh_sum_with_diagonals_and_shared_conv():
    """The double-hoisted sum with arbitrary steps and diagonals decrypts to sum_k rot(z, s_k) * d_k; the
    shared-baby-step convolution (kernel multiplied after the input's rotations) decrypts to the same
    tap sums as the hoisted one and as the FP64 convolution."""
    o = OracleCKKS(13, [55, 40, 40, 40, 56], 2.0 ** 40).keygen()
    baby, giant = OracleCKKS.conv_bsgs_steps(49, 64)
    o.gen_galois_keys(baby + giant + [5, 300])
    z = inputs.uniform_slots(o.slots, 31)
    ct = o.encrypt_values(z, 60)
    steps = [5, 300]
    ds = [inputs.uniform_slots(o.slots, 40 + k) for k in range(3)]
    ext = np.stack([o.encode_ext(d, ct.level) for d in ds])
    got = o.decrypt_values(o.rescale(o.dh_sum(ct, steps, ext)))
    ref = ds[0] * z + sum(np.roll(z, -s) * d for s, d in zip(steps, ds[1:]))
    assert np.max(np.abs(got - ref)) < 1e-6
    # the convolution: slot w of the result holds sum_t K[t] x[64 t + w]
    img = inputs.mnist_like_image(5)
    x, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    kern = np.random.default_rng(8).normal(0.0, 0.1, 49)
    ks = o.kernel_slots(kern, 64)
    cx = o.encrypt_values(x, 61)
    shared = o.conv2d_im2col_shared(cx, o.conv_baby_diagonals_ext(ks, 49, 64, cx.level), 49, 64)
    hoisted = o.conv2d_im2col_hoisted(cx, o.encode(ks, level=cx.level), 49, 64)
    assert shared.level == hoisted.level and shared.scale == hoisted.scale
    a, b = o.decrypt_values(shared, 64), o.decrypt_values(hoisted, 64)
    conv = np.array([sum(kern[t] * x[64 * t + w] for t in range(49)) for w in range(64)])
    assert np.max(np.abs(a - conv)) < 1e-6 and np.max(np.abs(a - b)) < 1e-6


def test_cnn_shared_conv_schedule_matches_fp64():
    """The CNN with the shared-baby-step convolution, rectangular FC layers and double hoisting decrypts
    to the FP64 network."""
    o = OracleCKKS(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26).keygen()
    steps = oracle.cnn_galois_steps(o, rect=True, conv_hoist=True, conv_shared=True)
    for st, lv in steps.items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(4))
    enc = oracle.cnn_encode(o, w, rect=True, conv_hoist=True, conv_shared=True)
    img = inputs.mnist_like_image(3)
    v, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, 77)
    logits = o.decrypt_values(oracle.cnn_forward(o, ct, w, enc, double_hoist=True), 10)
    assert np.max(np.abs(logits - oracle.cnn_plain(img, w))) < 5e-3


@pytest.mark.parametrize("shared", [True, False])
def test_cnn_pack_first_schedule_matches_fp64(shared):
    """The CNN with the channels packed after the baby-step sums and one giant-step sum per request
    (the packed vector repeats every 8 windows-blocks, so FC1 replicates with one rotation) decrypts to
    the FP64 network, with the shared or the per-kernel baby steps."""
    o = OracleCKKS(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26).keygen()
    steps = oracle.cnn_galois_steps(o, rect=True, conv_hoist=True, conv_shared=shared, pack_first=True)
    assert steps[512] == o.L - 2 and steps[o.slots - 256] == o.L - 3
    for st, lv in steps.items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(4))
    enc = oracle.cnn_encode(o, w, rect=True, conv_hoist=True, conv_shared=shared, pack_first=True)
    img = inputs.mnist_like_image(3)
    v, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, 77)
    logits = o.decrypt_values(oracle.cnn_forward(o, ct, w, enc, double_hoist=True), 10)
    assert np.max(np.abs(logits - oracle.cnn_plain(img, w))) < 5e-3


def _coeff_ints(o, data, level):
    """Balanced integer coefficients of each component [2][level][N] (exact CRT)."""
    Q = 1
    for q in o.primes[:level]:
        Q *= q
    out = []
    for b in range(2):
        c = o.crt_compose(o.intt_limbs(np.ascontiguousarray(data[b]), level), level)
        out.append(np.array([x - Q if x > Q // 2 else x for x in c], dtype=object))
    return out


@pytest.mark.parametrize("bits", [[36, 36, 36, 37], [31, 26, 26, 26, 31]])
def test_merged_moddown_rescale_within_one_of_separate(bits):
    """One rounding of (P d + U) / (P q_last) against ModDown then rescale, round((d + round(U/P)) / q):
    the two differ by at most 1 in any integer coefficient, for relinearization and for a double-hoisted
    sum, and decrypt alike."""
    o = OracleCKKS(12, bits, 2.0 ** 30 if bits[1] == 36 else 2.0 ** 26).keygen()
    o.gen_galois_keys([3, 700])
    L = o.L
    x, y = inputs.uniform_slots(o.slots, 41), inputs.uniform_slots(o.slots, 42)
    a, b = o.encrypt_values(x, 1), o.encrypt_values(y, 2)
    sep, mer = o.mul(a, b), o.mul(a, b, merged=True)
    assert mer.level == sep.level == L - 1 and mer.scale == sep.scale
    for u, v in zip(_coeff_ints(o, sep.data, L - 1), _coeff_ints(o, mer.data, L - 1)):
        assert max(abs(int(t)) for t in (u - v)) <= 1
    assert np.max(np.abs(o.decrypt_values(mer) - x * y)) < 1e-3
    ds = np.stack([o.encode_ext(inputs.uniform_slots(o.slots, 50 + k), L) for k in range(3)])
    sep = o.rescale(o.dh_sum(a, [3, 700], ds))
    mer = o.dh_sum(a, [3, 700], ds, merged=True)
    assert mer.level == sep.level and mer.scale == sep.scale
    for u, v in zip(_coeff_ints(o, sep.data, L - 1), _coeff_ints(o, mer.data, L - 1)):
        assert max(abs(int(t)) for t in (u - v)) <= 1


def test_cnn_merged_rescale_schedule_matches_fp64():
    """The bench's network (shared baby steps, packed channels, rectangular FC, double hoisting) with every
    ModDown that precedes a rescale merged into it decrypts to the FP64 network."""
    o = OracleCKKS(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26).keygen()
    for st, lv in oracle.cnn_galois_steps(o, rect=True, conv_hoist=True, conv_shared=True, pack_first=True).items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(4))
    enc = oracle.cnn_encode(o, w, rect=True, conv_hoist=True, conv_shared=True, pack_first=True)
    img = inputs.mnist_like_image(3)
    v, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, 77)
    logits = o.decrypt_values(oracle.cnn_forward(o, ct, w, enc, double_hoist=True, merged=True), 10)
    assert np.max(np.abs(logits - oracle.cnn_plain(img, w))) < 5e-3


@pytest.mark.parametrize("merged", [True, False])
def test_cnn_folded_masks_match_the_pack_and_fp64(merged):
    """Masks folded into the shared baby-step diagonals (reading A27): one diagonal-method sum over
    sum_k mask_k * d_kb, then a modulus switch, gives the packed vector the per-kernel sums, masks and
    pack give (same level, same slot values up to rounding noise), and the whole network decrypts to the
    FP64 network."""
    o = OracleCKKS(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26).keygen()
    for st, lv in oracle.cnn_galois_steps(o, rect=True, conv_hoist=True, conv_shared=True, pack_first=True).items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(4))
    enc = oracle.cnn_encode(o, w, rect=True, conv_hoist=True, conv_shared=True, pack_first=True)
    encf = oracle.cnn_encode(o, w, rect=True, conv_hoist=True, conv_shared=True, pack_first=True, fold=True)
    with pytest.raises(ValueError):
        oracle.cnn_encode(o, w, rect=True, conv_hoist=True, conv_shared=True, fold=True)
    img = inputs.mnist_like_image(5)
    v, _ = OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, 78)
    baby, _ = o.conv_bsgs_steps(enc.taps, enc.windows)
    zs = [o.dh_sum(ct, baby, enc.conv_baby_ext[k], merged=True) if merged
          else o.rescale(o.dh_sum(ct, baby, enc.conv_baby_ext[k])) for k in range(4)]
    packed = oracle.ckks._pack(o, zs, enc.masks, merged)
    folded = (o.dh_sum(ct, baby, encf.conv_baby_fold_ext, merged=True) if merged
              else o.rescale(o.dh_sum(ct, baby, encf.conv_baby_fold_ext)))
    folded = o.mod_switch(folded, folded.level - 1)
    assert folded.level == packed.level == o.L - 2
    a, b = o.decrypt_values(folded), o.decrypt_values(packed)
    assert np.max(np.abs(a - b)) < 1e-3 * max(1.0, float(np.max(np.abs(b))))
    assert np.max(np.abs(b)) > 0.1  # the comparison is not between two empty vectors
    logits = o.decrypt_values(oracle.cnn_forward(o, ct, w, encf, double_hoist=True, merged=merged), 10)
    assert np.max(np.abs(logits - oracle.cnn_plain(img, w))) < 5e-3
