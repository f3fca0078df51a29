"""Batched launches over a descriptor table: NTT / INTT / relinearize / rotate jobs of mixed N and
level in one batch, bit-identical to the single calls and to the oracle, eager and replayed from a
CUDA graph. The chain is the primitive sweep's: primes == 1 (mod 2^17), data prime i of 59 - (i mod 10)
bits, P the largest 60-bit one, shared by every N <= 2^16."""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import SEED
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L_SMALL, L_LARGE = 32, 8  # data primes of the N = 2^13 and N = 2^15 contexts


def _chain():
    return oracle.gen_primes(16, [59 - (i % 10) for i in range(L_SMALL)] + [60])


def _pair(log_n, n_data, steps):
    full = _chain()
    primes = full[:n_data] + [full[-1]]
    o = oracle.OracleCKKS(log_n, None, 2.0 ** 50, key_seed=SEED, primes=primes).keygen()
    g = tk.Context(tk.Params(log_n, primes=primes, scale=2.0 ** 50), seed=SEED, flags=tk.TCKS_AUTO_RELIN)
    assert g.primes == primes
    o.gen_galois_keys(steps)
    g.gen_galois_keys(steps)
    return o, g


@pytest.fixture(scope="module")
def ctxs():
    return {13: _pair(13, L_SMALL, [1]), 15: _pair(15, L_LARGE, [1])}


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _host(d, shape):
    return d.cpu().numpy().view(np.uint64).reshape(shape)


def _ntt_jobs(ctxs):
    """(context, op, count, level, seed, in_place) for a mix of N, levels and directions."""
    (o13, g13), (o15, g15) = ctxs[13], ctxs[15]
    return [
        (o13, g13, tk.JOB_NTT, 3, 4, 11, True),
        (o13, g13, tk.JOB_NTT, 1, 33, 12, False),  # every prime including P
        (o15, g15, tk.JOB_NTT, 2, 8, 13, True),
        (o13, g13, tk.JOB_INTT, 2, 16, 14, False),
        (o13, g13, tk.JOB_NTT, 0, 4, 15, True),  # an empty entry
        (o15, g15, tk.JOB_INTT, 1, 5, 16, True),
    ]


def test_mixed_ntt_batch_matches_single_calls_and_oracle(ctxs):
    specs = _ntt_jobs(ctxs)
    jobs, bufs = [], []
    for o, g, op, count, level, seed, in_place in specs:
        x = inputs.random_limbs(o.primes[:level], o.N, seed, polys=max(count, 1))[:count]
        d_in = _dev(x)
        d_out = d_in if in_place else torch.empty_like(d_in)
        bufs.append((x, d_in, d_out))
        jobs.append((g, op, 0, count, level, d_in.data_ptr(), d_out.data_ptr()))
    tk.batch_run(jobs)
    ctxs[13][1].synchronize()
    for (o, g, op, count, level, seed, in_place), (x, d_in, d_out) in zip(specs, bufs):
        if count == 0:
            continue
        got = _host(d_out, x.shape)
        single = _dev(x)
        g.ntt_inplace(single.data_ptr(), count, level, inverse=(op == tk.JOB_INTT))
        g.synchronize()
        assert np.array_equal(got, _host(single, x.shape)), (o.log_n, level)
        for p, l in {(0, 0), (count - 1, level - 1)}:
            q = o.primes[l]
            f = oracle.intt if op == tk.JOB_INTT else oracle.ntt
            assert np.array_equal(got[p, l], f(x[p, l], q, oracle.min_psi(q, o.log_n))), (o.log_n, level, p, l)


def _ks_specs(ctxs):
    """(N, op, count, level, seed) for relinearize / rotate jobs of mixed N and level."""
    return [(13, tk.JOB_RELIN, 3, 4, 21), (13, tk.JOB_RELIN, 2, 16, 22), (15, tk.JOB_RELIN, 2, 8, 23),
            (13, tk.JOB_ROTATE, 2, 32, 24), (15, tk.JOB_ROTATE, 1, 4, 25)]


def _ks_batch(ctxs, contexts=None):
    """The relinearize / rotate batch of _ks_specs; `contexts` (N -> GPU context) replaces the fixture's
    GPU contexts, with the same inputs."""
    jobs, bufs = [], []
    for log_n, op, count, level, seed in _ks_specs(ctxs):
        o, g = ctxs[log_n]
        g = contexts[log_n] if contexts else g
        polys = 3 if op == tk.JOB_RELIN else 2
        x = np.stack([inputs.random_limbs(o.primes[:level], o.N, seed * 100 + i, polys=polys) for i in range(count)])
        d_in = _dev(x)
        d_out = torch.empty((count, 2, level, o.N), dtype=torch.int64, device="cuda")
        bufs.append((x, d_in, d_out))
        jobs.append((g, op, 1, count, level, d_in.data_ptr(), d_out.data_ptr()))
    return jobs, bufs


def _ks_reference(o, op, x, level):
    if op == tk.JOB_RELIN:
        return o.relinearize(x, level, 1.0).data
    return o.rotate(oracle.Ct(np.ascontiguousarray(x), level, 1.0), 1).data


def test_mixed_keyswitch_batch_matches_oracle(ctxs):
    jobs, bufs = _ks_batch(ctxs)
    tk.batch_run(jobs)
    ctxs[13][1].synchronize()
    for (log_n, op, count, level, seed), (x, d_in, d_out) in zip(_ks_specs(ctxs), bufs):
        o = ctxs[log_n][0]
        got = _host(d_out, (count, 2, level, o.N))
        for i in range(count):
            assert np.array_equal(got[i], _ks_reference(o, op, x[i], level)), (log_n, op, level, i)


def test_batch_graph_replay_is_bit_identical(ctxs):
    jobs, bufs = _ks_batch(ctxs)
    tk.batch_run(jobs)
    ctxs[13][1].synchronize()
    eager = [_host(d_out, tuple(d_out.shape)).copy() for _, _, d_out in bufs]
    for _, _, d_out in bufs:
        d_out.zero_()
    graph = tk.BatchGraph(jobs)
    assert graph.launches > 0
    for _ in range(2):
        for _, _, d_out in bufs:
            d_out.zero_()
        torch.cuda.synchronize()
        before = tk.launch_count()
        graph.run()
        ctxs[13][1].synchronize()
        assert tk.launch_count() - before == graph.launches
        for ref, (_, _, d_out) in zip(eager, bufs):
            assert np.array_equal(_host(d_out, ref.shape), ref)


def test_batch_graph_with_caller_allocator(ctxs):
    """Contexts whose memory comes from PyTorch's caching allocator (callbacks that cannot run inside a
    capture): the graph takes its scratch from one block of that allocator, sized by an uncaptured
    pass, and replays to the same bits as the fixture's pool-allocator contexts run eagerly."""
    jobs, bufs = _ks_batch(ctxs)
    tk.batch_run(jobs)
    ctxs[13][1].synchronize()
    eager = [_host(d_out, tuple(d_out.shape)).copy() for _, _, d_out in bufs]
    mine = {}
    for log_n, n_data in ((13, L_SMALL), (15, L_LARGE)):
        primes = ctxs[log_n][0].primes
        g = tk.Context(tk.Params(log_n, primes=primes, scale=2.0 ** 50), seed=SEED, flags=tk.TCKS_AUTO_RELIN,
                       allocator="torch")
        g.gen_galois_keys([1])
        mine[log_n] = g
    jobs, bufs = _ks_batch(ctxs, mine)
    graph = tk.BatchGraph(jobs)
    for _ in range(2):
        for _, _, d_out in bufs:
            d_out.zero_()
        torch.cuda.synchronize()
        graph.run()
        mine[13].synchronize()
        for ref, (_, _, d_out) in zip(eager, bufs):
            assert np.array_equal(_host(d_out, ref.shape), ref)
    del graph


def test_batch_validation_launches_nothing(ctxs):
    o, g = ctxs[13]
    d = torch.zeros((2, 2, 4, o.N), dtype=torch.int64, device="cuda")
    e = torch.zeros_like(d)
    good = (g, tk.JOB_ROTATE, 1, 2, 4, d.data_ptr(), e.data_ptr())
    cases = {
        "INVALID_ARG": [good, (g, 7, 0, 1, 4, d.data_ptr(), e.data_ptr())],
        "NO_GALOIS_KEY": [good, (g, tk.JOB_ROTATE, 5, 1, 4, d.data_ptr(), e.data_ptr())],
    }
    cases_level = [good, (g, tk.JOB_RELIN, 0, 1, L_SMALL + 1, d.data_ptr(), e.data_ptr())]
    torch.cuda.synchronize()
    before = tk.launch_count()
    for name, jobs in cases.items():
        with pytest.raises(tk.TcksError) as err:
            tk.batch_run(jobs)
        assert err.value.name == name
    with pytest.raises(tk.TcksError) as err:
        tk.batch_run(cases_level)
    assert err.value.name == "INVALID_ARG"
    with pytest.raises(tk.TcksError) as err:
        tk.batch_run([(g, tk.JOB_ROTATE, 1, 1, 4, d.data_ptr(), d.data_ptr())])
    assert err.value.name == "INVALID_ARG"
    assert tk.launch_count() == before


def test_profiler_counts_butterflies_and_calibration(ctxs):
    o, g = ctxs[13]
    x = _dev(inputs.random_limbs(o.primes[:8], o.N, 31, polys=4))
    tk.profile_start()
    tk.batch_run([(g, tk.JOB_NTT, 0, 4, 8, x.data_ptr(), x.data_ptr())])
    g.synchronize()
    tk.profile_stop()
    prof = tk.profile_read(with_ops=True)
    launches, ms, by, ops = prof["ntt_fwd"]
    assert launches == 1 and by == 16 * o.N * 32 and ops == 32 * (o.N // 2) * o.log_n
    assert tk.calibrate_butterflies(64) > 1e10 and tk.calibrate_butterflies(32) > 1e10
    assert tk.calibrate_macs(64) > 1e10 and tk.calibrate_macs(32) > tk.calibrate_macs(64)


def test_batch_submit_wait_and_timeout(ctxs):
    """tcks_batch_submit queues a job table and returns a handle; tcks_batch_wait reports TIMEOUT while
    the work cannot have finished (the context's stream is held by a bounded GPU sleep of about a
    second queued before it), then OK, with the results of the single calls."""
    if not hasattr(torch.cuda, "_sleep"):
        pytest.skip("torch.cuda._sleep is not available")
    o, _ = ctxs[13]
    st = torch.cuda.Stream()
    g = tk.Context(tk.Params(13, primes=o.primes, scale=2.0 ** 50), seed=SEED, flags=tk.TCKS_AUTO_RELIN,
                   stream=st.cuda_stream)
    x = inputs.random_limbs(o.primes[:8], o.N, 41, polys=4)
    d = _dev(x)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        torch.cuda._sleep(2_000_000_000)  # ~1 s at 2 GHz, ends by itself
    b = tk.Batch([(g, tk.JOB_NTT, 0, 4, 8, d.data_ptr(), d.data_ptr())])
    with pytest.raises(tk.TcksError) as e:
        b.wait(1_000_000)
    assert e.value.name == "TIMEOUT"
    b.wait(60_000_000_000)
    b.wait(0)  # completed work polls as done
    single = _dev(x)
    g.ntt_inplace(single.data_ptr(), 4, 8, inverse=False)
    g.synchronize()
    assert np.array_equal(_host(d, x.shape), _host(single, x.shape))
    del b
    with pytest.raises(tk.TcksError) as e:  # validation fails before anything is queued
        tk.Batch([(g, 7, 0, 1, 8, d.data_ptr(), d.data_ptr())])
    assert e.value.name == "INVALID_ARG"


def test_ntt_jobs_of_four_ring_sizes_in_one_launch_pair(ctxs):
    """NTT and INTT jobs of contexts with N = 2^13, 2^14, 2^15 and 2^16 go out as one columns launch and one
    slices launch per direction (4 launches for the whole table), bit-identical to the single calls."""
    o13 = ctxs[13][0]
    gs = {13: ctxs[13][1], 15: ctxs[15][1]}
    for ln in (14, 16):
        gs[ln] = tk.Context(tk.Params(ln, primes=o13.primes[:5] + [o13.primes[-1]], scale=2.0 ** 50), seed=SEED,
                            flags=tk.TCKS_AUTO_RELIN)
    jobs, bufs = [], []
    for k, (ln, g) in enumerate(sorted(gs.items())):
        n = 1 << ln
        for op, level, count in ((tk.JOB_NTT, 3, 2), (tk.JOB_INTT, 2, 3)):
            x = inputs.random_limbs(g.primes[:level], n, 200 + 10 * k + op, polys=count)
            d_in = _dev(x)
            d_out = torch.empty_like(d_in)
            bufs.append((g, op, count, level, x, d_out))
            jobs.append((g, op, 0, count, level, d_in.data_ptr(), d_out.data_ptr()))
    torch.cuda.synchronize()
    before = tk.launch_count()
    tk.batch_run(jobs)
    for g in gs.values():
        g.synchronize()
    assert tk.launch_count() - before == 4
    for g, op, count, level, x, d_out in bufs:
        single = _dev(x)
        g.ntt_inplace(single.data_ptr(), count, level, inverse=(op == tk.JOB_INTT))
        g.synchronize()
        assert np.array_equal(_host(d_out, x.shape), _host(single, x.shape)), (g.N, op)
