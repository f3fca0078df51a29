"""The allocation-free rescale, for callers that must not allocate device memory while they run (for
example a serving loop that reserves its whole device budget up front and admits work against it).

It must give the same limbs as the ordinary rescale, on two calls in a row (the second call reuses
the static scratch the first one left behind). The buffers here come from PyTorch, so the library
call under test is the only thing that touches the library's own memory, and it touches none.
"""
import numpy as np
import pytest

import paper_2104_03152_gb300 as tk
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("log_n,bits,level", [(13, [31, 26, 26, 26, 26, 26, 26, 31], 7), (14, [60, 40, 40, 60], 3),
                                              (12, [36, 36, 36, 37], 2)])
def test_rescale_noalloc_matches_rescale_twice(log_n, bits, level):
    ctx = tk.Context(tk.Params(log_n, bits, 2.0 ** 30), seed=inputs.SEED_KEYS)
    n = 1 << log_n
    for call in range(2):
        limbs = inputs.random_limbs(ctx.primes[:level], n, 500 + call, polys=2)
        ref = ctx.ct_import(limbs, 1.0).rescale_().export()  # the existing entry point
        d_in = torch.from_numpy(limbs.view(np.int64).copy()).cuda()
        d_out = torch.full((2 * (level - 1) * n,), -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        ctx.rescale_noalloc(d_in.data_ptr(), level, d_out.data_ptr())
        ctx.synchronize()
        got = d_out.cpu().numpy().view(np.uint64).reshape(2, level - 1, n)
        assert np.array_equal(got, ref), f"call {call}"


def test_rescale_noalloc_after_a_smaller_ordinary_rescale():
    """The shared-memory limit the first call needs (a 2^14 limb of 64-bit words, 128 KB) must survive an
    ordinary rescale at N = 2^13 of the same kernels, which needs only 64 KB."""
    big = tk.Context(tk.Params(14, [60, 40, 40, 60], 2.0 ** 40), seed=inputs.SEED_KEYS)
    small = tk.Context(tk.Params(13, [50, 40, 40, 50], 2.0 ** 40), seed=inputs.SEED_KEYS)
    n, level = 1 << 14, 3

    def noalloc_once(seed):
        limbs = inputs.random_limbs(big.primes[:level], n, seed, polys=2)
        ref = big.ct_import(limbs, 1.0).rescale_().export()
        d_in = torch.from_numpy(limbs.view(np.int64).copy()).cuda()
        d_out = torch.full((2 * (level - 1) * n,), -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        big.rescale_noalloc(d_in.data_ptr(), level, d_out.data_ptr())
        big.synchronize()
        assert np.array_equal(d_out.cpu().numpy().view(np.uint64).reshape(2, level - 1, n), ref), seed

    noalloc_once(600)
    limbs = inputs.random_limbs(small.primes[:3], 1 << 13, 601, polys=2)
    small.ct_import(limbs, 1.0).rescale_().export()  # the ordinary path at N = 2^13, 64-bit words
    noalloc_once(602)


def test_rescale_noalloc_rejects_bad_level():
    small = tk.Context(tk.Params(12, [36, 36, 37], 2.0 ** 30), seed=inputs.SEED_KEYS)
    buf = torch.zeros(2 * 2 * (1 << 12), dtype=torch.int64, device="cuda")
    with pytest.raises(tk.TcksError) as e:
        small.rescale_noalloc(buf.data_ptr(), 1, buf.data_ptr())
    assert e.value.name == "LEVEL_EXHAUSTED"
    with pytest.raises(tk.TcksError) as e:
        small.rescale_noalloc(buf.data_ptr(), 3, buf.data_ptr())
    assert e.value.name == "INVALID_ARG"
