"""GPU (through the C ABI) versus the CPU oracle, bit-exact on identical inputs.

Configurations: C1's chain (N=4096, [36,36,36|37], 2^30), C2's chain (N=8192, [31,26x6|31], 2^26,
an odd stage count), C4's chain (N=16384, [60,40,40|60], 2^40, the largest single-pass N), and a tiny
N=32 chain (one warp, ragged thread/element ratio).
"""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import Pair, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHAINS = {
    "C1": (12, [36, 36, 36, 37], 2.0 ** 30),
    "C2": (13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26),
    "C4": (14, [60, 40, 40, 60], 2.0 ** 40),
    "tiny": (5, [30, 30, 31], 2.0 ** 20),
}


@pytest.fixture(scope="module", params=sorted(CHAINS))
def pair(request):
    log_n, bits, scale = CHAINS[request.param]
    n = 1 << (log_n - 1)
    steps = sorted({1, 2, 3, 5, n - 1, n // 2} | {1 << m for m in range(log_n - 1)})
    return Pair(log_n, bits, scale, galois=steps)


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_ntt_parity(pair):
    o, g = pair.o, pair.g
    lv = o.L + 1
    x = inputs.random_limbs(o.primes, o.N, 101, polys=2)
    d = _dev(x)
    g.ntt_inplace(d.data_ptr(), 2, lv, inverse=False)
    g.synchronize()
    got = d.cpu().numpy().view(np.uint64).reshape(x.shape)
    for p in range(2):
        for l in range(lv):
            ref = oracle.ntt(x[p, l], o.primes[l], oracle.min_psi(o.primes[l], o.log_n))
            assert np.array_equal(got[p, l], ref), (p, l)
    g.ntt_inplace(d.data_ptr(), 2, lv, inverse=True)
    g.synchronize()
    back = d.cpu().numpy().view(np.uint64).reshape(x.shape)
    assert np.array_equal(back, x)


def test_keys_parity(pair):
    o, g = pair.o, pair.g
    assert np.array_equal(g.export_key(tk.KEY_SECRET), o.s)
    assert np.array_equal(g.export_key(tk.KEY_PUBLIC), o.pk)
    assert np.array_equal(g.export_key(tk.KEY_RELIN), o.rlk.data)
    for st in pair.steps[:3]:
        assert np.array_equal(g.export_key(tk.KEY_GALOIS, st), o.galois[st % o.slots].data), st


def test_trimmed_galois_key_parity():
    p = Pair(12, [36, 36, 36, 37], 2.0 ** 30)
    p.add_galois([7], key_level=2)
    assert np.array_equal(p.g.export_key(tk.KEY_GALOIS, 7), p.o.galois[7].data)


def test_encrypt_decrypt_parity(pair):
    o = pair.o
    z = inputs.uniform_slots(o.slots, 1)
    pt = o.encode(z)
    for level in (o.L, 1):
        ptl = oracle.Pt(np.ascontiguousarray(pt.data[:level]), level, pt.scale)
        ref = o.encrypt(ptl, seed=77)
        got = pair.g.encrypt(pair.import_pt(ptl), 77)
        assert_ct_equal(got, ref, f"encrypt level {level}")
        dec = pair.g.decrypt(got).export()
        assert np.array_equal(dec, o.decrypt(ref).data)


def test_elementwise_parity(pair):
    o, g = pair.o, pair.g
    x, y = inputs.uniform_slots(o.slots, 1), inputs.uniform_slots(o.slots, 2)
    cx, cy = o.encrypt_values(x, 11), o.encrypt_values(y, 12)
    py = o.encode(y)
    gx, gy, gp = pair.import_ct(cx), pair.import_ct(cy), pair.import_pt(py)
    assert_ct_equal(gx.add(gy), o.add(cx, cy), "add")
    assert_ct_equal(gx.sub(gy), o.sub(cx, cy), "sub")
    assert_ct_equal(gx.negate(), o.negate(cx), "negate")
    assert_ct_equal(gx.add_plain(gp), o.add_plain(cx, py), "add_plain")
    assert_ct_equal(gx.sub_plain(gp), o.sub_plain(cx, py), "sub_plain")
    assert_ct_equal(gx.mul_plain(gp), o.mul_plain(cx, py), "mul_plain")
    lo = o.mod_switch(cx, 1)
    assert_ct_equal(pair.import_ct(cx).mod_switch_(1), lo, "mod_switch")


def test_mul_relin_rescale_parity(pair):
    o = pair.o
    x, y = inputs.uniform_slots(o.slots, 3), inputs.uniform_slots(o.slots, 4)
    cx, cy = o.encrypt_values(x, 21), o.encrypt_values(y, 22)
    gx, gy = pair.import_ct(cx), pair.import_ct(cy)
    ref = o.mul(cx, cy)  # tensor, relinearize, rescale
    assert_ct_equal(gx.mul(gy), ref, "mul")
    assert_ct_equal(gx.square(), o.square(cx), "square")
    d3, lv, sc = o.tensor(cx, cy)
    rel = o.relinearize(d3, lv, sc)
    assert_ct_equal(pair.import_ct(rel).rescale_(), o.rescale(rel), "rescale")
    if o.L >= 3:  # a lower level, with the same (full-level) relinearization key
        c2x, c2y = o.mod_switch(cx, 2), o.mod_switch(cy, 2)
        assert_ct_equal(pair.import_ct(c2x).mul(pair.import_ct(c2y)), o.mul(c2x, c2y), "mul level 2")


def test_mul_merged_rescale_parity(pair):
    """TCKS_MERGED_RESCALE: the relinearization's ModDown and the rescale as one rounding, bit-exact
    against the oracle's merged multiply, at the top level and one level down."""
    o, g = pair.o, pair.g
    x, y = inputs.uniform_slots(o.slots, 5), inputs.uniform_slots(o.slots, 6)
    cx, cy = o.encrypt_values(x, 23), o.encrypt_values(y, 24)
    g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_MERGED_RESCALE)
    try:
        assert_ct_equal(pair.import_ct(cx).mul(pair.import_ct(cy)), o.mul(cx, cy, merged=True), "merged mul")
        if o.L >= 3:
            c2x, c2y = o.mod_switch(cx, 2), o.mod_switch(cy, 2)
            assert_ct_equal(pair.import_ct(c2x).mul(pair.import_ct(c2y)), o.mul(c2x, c2y, merged=True),
                            "merged mul level 2")
    finally:
        g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE)


def test_mul_relin_only_parity():
    log_n, bits, scale = CHAINS["C1"]
    p = Pair(log_n, bits, scale, flags=tk.TCKS_AUTO_RELIN)
    o = p.o
    cx = o.encrypt_values(inputs.uniform_slots(o.slots, 5), 31)
    cy = o.encrypt_values(inputs.uniform_slots(o.slots, 6), 32)
    d3, lv, sc = o.tensor(cx, cy)
    assert_ct_equal(p.import_ct(cx).mul(p.import_ct(cy)), o.relinearize(d3, lv, sc), "relin only")


def test_rotation_parity(pair):
    o = pair.o
    x = inputs.uniform_slots(o.slots, 7)
    cx = o.encrypt_values(x, 41)
    gx = pair.import_ct(cx)
    steps = pair.steps
    for st in steps:
        assert_ct_equal(gx.rotate(st), o.rotate(cx, st), f"rotate {st}")
    hs = gx.rotate_hoisted(steps + [0])
    for st, h in zip(steps + [0], hs):
        assert_ct_equal(h, o.rotate(cx, st), f"hoisted {st}")
    # at a lower level, with keys of the full level
    c1 = o.mod_switch(cx, 1)
    assert_ct_equal(pair.import_ct(c1).rotate(1), o.rotate(c1, 1), "rotate level 1")


def test_encode_decode_parity(pair):
    """Encode: identical integer coefficients except where the oracle's pre-rounding value lies
    within the FP64 error bound of a .5 tie; decode within 1e-9 of the oracle's slots."""
    o, g = pair.o, pair.g
    scale = o.scale
    for seed, n in ((1, o.slots), (2, max(1, o.slots // 3)), (3, 1)):
        z = inputs.uniform_slots(n, seed)
        ref_pt, pre = o.encode(z, want_pre=True)
        gpt = g.encode(z)
        assert gpt.info() == (o.L, scale)
        got = gpt.export()
        # coefficient domain through the oracle's own transform
        got_c = np.array(o.crt_compose(o.intt_limbs(got, o.L), o.L), dtype=object)
        ref_c = np.array(o.crt_compose(o.intt_limbs(ref_pt.data, o.L), o.L), dtype=object)
        diff = np.nonzero(got_c != ref_c)[0]
        # FP64 error bound of the size-N/2 FFT: ~ log2(N) * 2^-53 * scale * (2/N) * sum|z|
        bound = 4 * o.log_n * 2.0 ** -53 * scale * (2.0 / o.N) * np.sum(np.abs(z)) + 1e-9
        for i in diff:
            frac = abs(pre[i] - np.floor(pre[i]) - 0.5)
            assert abs(int(got_c[i]) - int(ref_c[i])) == 1 and frac <= bound, (i, pre[i])
        dec_g = g.decode(pair.import_pt(ref_pt))
        dec_o = o.decode(ref_pt)
        assert np.max(np.abs(dec_g - dec_o)) < 1e-9
    assert g.encode(np.zeros(0)).export().any() == False  # empty input encodes the zero polynomial


def test_decode_at_every_level(pair):
    o, g = pair.o, pair.g
    z = inputs.uniform_slots(o.slots, 9)
    pt = o.encode(z)
    for lv in range(1, o.L + 1):
        ptl = oracle.Pt(np.ascontiguousarray(pt.data[:lv]), lv, pt.scale)
        assert np.max(np.abs(g.decode(pair.import_pt(ptl)) - o.decode(ptl))) < 1e-9


def test_errors(pair):
    o, g = pair.o, pair.g
    cx = pair.import_ct(o.encrypt_values(inputs.uniform_slots(o.slots, 1), 1))
    low = pair.import_ct(o.mod_switch(o.encrypt_values(inputs.uniform_slots(o.slots, 1), 1), 1))
    with pytest.raises(tk.TcksError) as e:
        cx.add(low)
    assert e.value.name == "LEVEL_MISMATCH"
    with pytest.raises(tk.TcksError) as e:
        low.rescale_()
    assert e.value.name == "LEVEL_EXHAUSTED"
    with pytest.raises(tk.TcksError) as e:
        cx.rotate(o.slots // 2 + 7 if o.slots > 16 else 6)
    assert e.value.name == "NO_GALOIS_KEY"
    sq = cx.mul_plain(g.encode(np.ones(4)))
    with pytest.raises(tk.TcksError) as e:
        cx.add(sq)
    assert e.value.name in ("SCALE_MISMATCH",)
    with pytest.raises(tk.TcksError) as e:
        g.encode(np.full(4, 1e30))
    assert e.value.name == "VALUE_OVERFLOW"


def test_autotune_keeps_results(tmp_path):
    """The autotuner only moves the launch shape: results stay bit-exact, and its choice is cached."""
    p = Pair(13, [31, 26, 26, 26, 31], 2.0 ** 26, galois=[1])
    o = p.o
    cx = o.encrypt_values(inputs.uniform_slots(o.slots, 1), 3)
    cache = str(tmp_path / "tune.json")
    t = p.g.autotune(cache)
    assert t % 32 == 0 and 32 <= t <= 1024
    assert p.g.autotune(cache) == t  # read back from the cache
    assert_ct_equal(p.import_ct(cx).mul(p.import_ct(cx)), o.mul(cx, cx), "mul after tuning")
    assert_ct_equal(p.import_ct(cx).rotate(1), o.rotate(cx, 1), "rotate after tuning")
    import json
    assert any(k.endswith("|13|32") for k in json.load(open(cache)))
