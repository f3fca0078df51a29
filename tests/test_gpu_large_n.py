"""N = 2^15 and 2^16 (the top of the C3 sweep): limbs split over a 2- or 4-CTA thread-block cluster.
NTT, keys, relinearization and rotation bit-exact against the oracle on uniform random limbs."""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import Pair, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=[15, 16])
def big(request):
    log_n = request.param
    return Pair(log_n, [59, 58, 57, 56, 60], 2.0 ** 50, flags=tk.TCKS_AUTO_RELIN, galois=[1, 3], key_level=None)


def test_ntt_large(big):
    o, g = big.o, big.g
    lv = o.L + 1
    x = inputs.random_limbs(o.primes, o.N, 7, polys=1)
    d = torch.from_numpy(x.view(np.int64).copy()).cuda()
    g.ntt_inplace(d.data_ptr(), 1, lv, inverse=False)
    g.synchronize()
    got = d.cpu().numpy().view(np.uint64).reshape(x.shape)
    for l in range(lv):
        assert np.array_equal(got[0, l], oracle.ntt(x[0, l], o.primes[l], oracle.min_psi(o.primes[l], o.log_n))), l
    g.ntt_inplace(d.data_ptr(), 1, lv, inverse=True)
    g.synchronize()
    assert np.array_equal(d.cpu().numpy().view(np.uint64).reshape(x.shape), x)


def test_keys_large(big):
    o, g = big.o, big.g
    assert np.array_equal(g.export_key(tk.KEY_SECRET), o.s)
    assert np.array_equal(g.export_key(tk.KEY_RELIN), o.rlk.data)
    assert np.array_equal(g.export_key(tk.KEY_GALOIS, 3), o.galois[3].data)


def test_relin_rotate_large(big):
    o = big.o
    lv = o.L
    a = oracle.Ct(np.ascontiguousarray(inputs.random_limbs(o.primes[:lv], o.N, 11, polys=2)), lv, 1.0)
    b = oracle.Ct(np.ascontiguousarray(inputs.random_limbs(o.primes[:lv], o.N, 12, polys=2)), lv, 1.0)
    d3, _, sc = o.tensor(a, b)
    ref = o.relinearize(d3, lv, sc)
    assert_ct_equal(big.import_ct(a).mul(big.import_ct(b)), ref, "relinearize")
    for st in (1, 3):
        assert_ct_equal(big.import_ct(a).rotate(st), o.rotate(a, st), f"rotate {st}")
