"""Hybrid key switching on the GPU (digits of alpha data primes, K special primes; reading A26) versus
the oracle, bit for bit on identical keys and ciphertexts: the keys, relinearization, rotation (plain,
hoisted, at lower levels where the last digit is partial), batched jobs, 64-bit and 32-bit words,
one-CTA and clustered transforms, and the primitive sweep's largest shape (N = 2^16, 32 data primes
in 4 digits of 8, 8 special primes)."""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import Pair, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHAINS = {
    # name: (log_n, bits (data, then special), scale, n_special, alpha)
    "a2k2": (12, [50, 40, 40, 40, 40, 60, 60], 2.0 ** 40, 2, 2),
    "a3k3": (13, [50, 50, 50, 50, 50, 60, 60, 60], 2.0 ** 40, 3, 3),
    "a1k2": (12, [60, 40, 40, 60, 60], 2.0 ** 40, 2, 1),
    "narrow": (13, [30, 30, 30, 30, 30, 31, 31], 2.0 ** 25, 2, 2),
    "a2k2_n15": (15, [50, 45, 45, 45, 60, 60], 2.0 ** 40, 2, 2),
}


@pytest.fixture(scope="module", params=sorted(CHAINS))
def pair(request):
    log_n, bits, scale, k, a = CHAINS[request.param]
    return Pair(log_n, bits, scale, flags=tk.TCKS_AUTO_RELIN, galois=[1, 5], n_special=k, alpha=a)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def test_hybrid_keys(pair):
    o, g = pair.o, pair.g
    assert g.L == o.L and g.primes == o.primes
    assert np.array_equal(g.export_key(tk.KEY_SECRET), o.s)
    assert np.array_equal(g.export_key(tk.KEY_PUBLIC), o.pk)
    assert np.array_equal(g.export_key(tk.KEY_RELIN), o.rlk.data)
    assert np.array_equal(g.export_key(tk.KEY_GALOIS, 5), o.galois[5].data)


def test_hybrid_relinearize_and_rotate(pair):
    o, g = pair.o, pair.g
    x, y = inputs.uniform_slots(o.slots, 1), inputs.uniform_slots(o.slots, 2)
    cx, cy = o.encrypt_values(x, 3), o.encrypt_values(y, 4)
    gx, gy = pair.import_ct(cx), pair.import_ct(cy)
    assert_ct_equal(gx.mul(gy), o.mul(cx, cy, rescale=False), "relinearized product")
    for lv in sorted({o.L, o.L - 1, 2, 1}):
        c = o.mod_switch(cx, lv)
        gc = pair.import_ct(c)
        for st in (1, 5):
            assert_ct_equal(gc.rotate(st), o.rotate(c, st), f"rotate {st} at level {lv}")
        hs = gc.rotate_hoisted([1, 5, 0])
        for st, h in zip((1, 5, 0), hs):
            assert_ct_equal(h, o.rotate(c, st), f"hoisted {st} at level {lv}")
        if lv >= 2:
            d = o.mod_switch(cy, lv)
            assert_ct_equal(gc.mul(pair.import_ct(d)), o.mul(c, d, rescale=False), f"product at level {lv}")
    if o.log_n <= 14:  # the GPU's decoder covers N <= 2^14
        dec = g.decrypt_values(gx.mul(gy).rescale_().rotate(1))
        assert np.max(np.abs(dec - np.roll(x * y, -1))) < 0.05


def test_hybrid_batched_jobs(pair):
    o, g = pair.o, pair.g
    lv = o.L
    d3 = np.stack([inputs.random_limbs(o.primes[:lv], o.N, 60 + i, polys=3) for i in range(3)])
    c2 = np.stack([inputs.random_limbs(o.primes[:lv], o.N, 70 + i, polys=2) for i in range(3)])
    di, do = _dev(d3), torch.empty((3, 2, lv, o.N), dtype=torch.int64, device="cuda")
    ri, ro = _dev(c2), torch.empty((3, 2, lv, o.N), dtype=torch.int64, device="cuda")
    tk.batch_run([(g, tk.JOB_RELIN, 0, 3, lv, di.data_ptr(), do.data_ptr()),
                  (g, tk.JOB_ROTATE, 5, 3, lv, ri.data_ptr(), ro.data_ptr())])
    g.synchronize()
    got_r = do.cpu().numpy().view(np.uint64).reshape(3, 2, lv, o.N)
    got_t = ro.cpu().numpy().view(np.uint64).reshape(3, 2, lv, o.N)
    for i in range(3):
        assert np.array_equal(got_r[i], o.relinearize(d3[i], lv, 1.0).data), i
        assert np.array_equal(got_t[i], o.rotate(oracle.Ct(np.ascontiguousarray(c2[i]), lv, 1.0), 5).data), i


def test_hybrid_refuses_fused_schedules(pair):
    o, g = pair.o, pair.g
    if o.log_n > 14:
        pytest.skip("the GPU's encoder covers N <= 2^14")
    ct = g.encrypt_values(inputs.uniform_slots(4, 1), 1)
    M = g.matrix_encode(np.ones((4, 2)), level=g.L)
    with pytest.raises(tk.TcksError) as e:
        ct.vecmat_plain(M)
    assert e.value.name == "UNSUPPORTED"
    with pytest.raises(tk.TcksError) as e:
        ct.rotate_sum_hoisted([1])
    assert e.value.name == "UNSUPPORTED"


def test_hybrid_bad_params_refused():
    chain = oracle.gen_primes(12, [50, 50, 50, 40])
    with pytest.raises(tk.TcksError) as e:  # one 40-bit special prime below two 50-bit digit primes
        tk.Params(12, primes=chain, scale=2.0 ** 40, n_special=1, alpha=2)
    assert e.value.name == "BAD_PARAMS"


def test_hybrid_full_sweep_shape():
    """N = 2^16, the sweep's 32 data primes (50-59 bits) in digits of 8, 8 special 60-bit primes: 4
    ciphertexts relinearized and rotated in one batch, every one equal to the oracle's."""
    bits = [59 - (i % 10) for i in range(32)] + [60] * 8
    o = oracle.OracleCKKS(16, bits, 2.0 ** 50, key_seed=0x7E5EA1, n_special=8, alpha=8).keygen()
    o.gen_galois_keys([1])
    g = tk.Context(tk.Params(16, primes=o.primes, scale=2.0 ** 50, n_special=8, alpha=8), seed=0x7E5EA1,
                   flags=tk.TCKS_AUTO_RELIN)
    g.gen_galois_keys([1])
    assert np.array_equal(g.export_key(tk.KEY_GALOIS, 1), o.galois[1].data)
    lv, count = 32, 4
    d3 = np.stack([inputs.random_limbs(o.primes[:lv], o.N, 90 + i, polys=3) for i in range(count)])
    c2 = np.stack([inputs.random_limbs(o.primes[:lv], o.N, 95 + i, polys=2) for i in range(count)])
    di, do = _dev(d3), torch.empty((count, 2, lv, o.N), dtype=torch.int64, device="cuda")
    ri, ro = _dev(c2), torch.empty((count, 2, lv, o.N), dtype=torch.int64, device="cuda")
    tk.batch_run([(g, tk.JOB_RELIN, 0, count, lv, di.data_ptr(), do.data_ptr()),
                  (g, tk.JOB_ROTATE, 1, count, lv, ri.data_ptr(), ro.data_ptr())])
    g.synchronize()
    got_r = do.cpu().numpy().view(np.uint64).reshape(count, 2, lv, o.N)
    got_t = ro.cpu().numpy().view(np.uint64).reshape(count, 2, lv, o.N)
    for i in range(count):
        assert np.array_equal(got_r[i], o.relinearize(d3[i], lv, 1.0).data), i
        assert np.array_equal(got_t[i], o.rotate(oracle.Ct(np.ascontiguousarray(c2[i]), lv, 1.0), 1).data), i
