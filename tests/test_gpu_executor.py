"""The persistent executor: NTT / INTT jobs posted to a resident kernel through a host-mapped queue give
the single calls' results, and a kernel left without work writes TIMEOUT to its status word after its
idle limit (a bounded wait on the GPU's global timer) and stops; later posts report that status."""
import time

import numpy as np
import pytest

import paper_2104_03152_gb300 as tk
from gpu_common import SEED
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TIMEOUT = -10  # TCKS_ERR_TIMEOUT


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("log_n,bits", [(13, [50, 40, 40, 60]), (12, [30, 30, 30, 31])], ids=["64-bit", "32-bit"])
def test_executor_jobs_equal_single_calls(log_n, bits):
    g = tk.Context(tk.Params(log_n, bits, 2.0 ** 30), seed=SEED)
    # Every buffer and every single-call result exists before the executor starts: while it is resident,
    # a device-wide synchronize (or anything that implies one) would wait for it.
    jobs = []
    for k, (op, polys, level) in enumerate(((tk.EXEC_NTT, 3, 3), (tk.EXEC_INTT, 2, 2), (tk.EXEC_NTT, 5, 3))):
        x = inputs.random_limbs(g.primes[:level], g.N, 900 + k, polys=polys)
        d_in, d_out, single = _dev(x), torch.zeros((polys, level, g.N), dtype=torch.int64, device="cuda"), _dev(x)
        g.ntt_inplace(single.data_ptr(), polys, level, inverse=(op == tk.EXEC_INTT))
        jobs.append((op, polys, level, d_in, d_out, single))
    g.synchronize()
    torch.cuda.current_stream().synchronize()
    ex = tk.Executor(g, capacity=64, idle_timeout_ns=5_000_000_000)
    try:
        tickets = [ex.post(op, d_in.data_ptr(), d_out.data_ptr(), polys, level)
                   for op, polys, level, d_in, d_out, _ in jobs]
        for (op, polys, level, _, d_out, single), ticket in zip(jobs, tickets):
            ex.wait(ticket, 10_000_000_000)
            got = d_out.cpu().numpy().view(np.uint64)
            assert np.array_equal(got, single.cpu().numpy().view(np.uint64)), (op, polys, level)
        assert ex.close() == 0
    finally:
        del ex


def test_executor_ring_wraps():
    """A ring of 8 slots takes 12 posts of 6 tasks: every slot is reused while other tasks may still run,
    and each ticket completes only once all tasks up to it have."""
    g = tk.Context(tk.Params(13, [50, 40, 40, 60], 2.0 ** 30), seed=SEED)
    polys, level, posts = 2, 3, 12
    x = inputs.random_limbs(g.primes[:level], g.N, 77, polys=polys * posts)
    d_in = _dev(x)
    d_out = torch.zeros_like(d_in)
    single = _dev(x)
    g.ntt_inplace(single.data_ptr(), polys * posts, level, inverse=False)
    g.synchronize()
    torch.cuda.current_stream().synchronize()
    ex = tk.Executor(g, capacity=8, idle_timeout_ns=5_000_000_000)
    try:
        stride = polys * level * g.N * 8
        tickets = [ex.post(tk.EXEC_NTT, d_in.data_ptr() + k * stride, d_out.data_ptr() + k * stride, polys, level)
                   for k in range(posts)]
        assert tickets == [(k + 1) * polys * level for k in range(posts)]
        ex.wait(tickets[-1], 10_000_000_000)
        with pytest.raises(tk.TcksError):
            ex.wait(tickets[-1] + 1, 0)  # beyond the last posted task
        assert np.array_equal(d_out.cpu().numpy().view(np.uint64), single.cpu().numpy().view(np.uint64))
        assert ex.close() == 0
    finally:
        del ex


def test_executor_idle_limit_writes_timeout():
    g = tk.Context(tk.Params(12, [50, 40, 60], 2.0 ** 30), seed=SEED)
    x = torch.zeros((1, 2, g.N), dtype=torch.int64, device="cuda")
    torch.cuda.current_stream().synchronize()
    ex = tk.Executor(g, capacity=16, idle_timeout_ns=20_000_000)  # 20 ms
    time.sleep(0.5)  # nothing posted: every CTA's wait runs out
    with pytest.raises(tk.TcksError) as e:
        ex.post(tk.EXEC_NTT, x.data_ptr(), x.data_ptr(), 1, 2)
    assert e.value.name == "TIMEOUT"
    assert ex.close() == TIMEOUT
    g.synchronize()  # the context is still usable
    y = g.encrypt_values(inputs.uniform_slots(4, 1), 1)
    assert np.max(np.abs(g.decrypt_values(y, 4) - inputs.uniform_slots(4, 1))) < 1e-3
