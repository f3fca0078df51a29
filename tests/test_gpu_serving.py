"""The serving loop: continuous batching at stage granularity, HBM-budget admission, and failures
injected on the host (a shrunk budget, an allocator that refuses). Every served result must equal the
single-request result bit for bit, alone or in any mix."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import SEED
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu

BITS = [31, 26, 26, 26, 26, 26, 26, 31]


@pytest.fixture(scope="module")
def cnn():
    ctx = tk.Context(tk.Params(13, BITS, 2.0 ** 26), seed=SEED)
    w = inputs.cnn_weights(4)
    model = tk.CNN(ctx, w["conv_w"], w["conv_b"], w["fc1_w"], w["fc1_b"], w["fc2_w"], w["fc2_b"], windows=64)
    model.gen_keys()
    reqs = []
    for i in range(8):
        v, _ = tk.im2col_encode(inputs.mnist_like_image(300 + i), 7, 7, 3, ctx.slots)
        reqs.append(ctx.encrypt_values(v, 900 + i))
    singles = [model.forward(c).export() for c in reqs]
    return ctx, model, reqs, singles


@pytest.fixture(scope="module")
def vm():
    ctx = tk.Context(tk.Params(12, [55, 40, 40, 56], 2.0 ** 40), seed=SEED)
    n, m = 16, 8
    M = inputs.random_matrix(n, m, 8, 0.5)
    ctx.gen_galois_keys([ctx.slots - n * (1 << i) for i in range(7)] + list(range(1, n)))
    mat = ctx.matrix_encode(M, level=3)
    reqs = []
    for i in range(3):
        v = np.zeros(ctx.slots)
        v[:n] = inputs.uniform_slots(n, 40 + i)
        reqs.append(ctx.encrypt_values(v, 700 + i))
    singles = [c.vecmat_plain(mat).export() for c in reqs]
    return ctx, mat, reqs, singles


BENCH_CNN_FLAGS = (tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_RECT_DIAG | tk.TCKS_CONV_HOIST
                   | tk.TCKS_CONV_SHARED | tk.TCKS_CONV_PACK | tk.TCKS_CONV_FOLD | tk.TCKS_MERGED_RESCALE
                   | tk.TCKS_DOUBLE_HOIST)


@pytest.fixture(scope="module")
def bench_lanes():
    """The lanes in the layout the benchmark serves: the CNN with rectangular FC layers, shared baby
    steps with the pack masks folded into their diagonals, ModDown and rescale merged and double hoisting; the
    vector x matrix product in rectangular form, double hoisted."""
    ctx = tk.Context(tk.Params(13, BITS, 2.0 ** 26), seed=SEED, flags=BENCH_CNN_FLAGS)
    w = inputs.cnn_weights(4)
    model = tk.CNN(ctx, w["conv_w"], w["conv_b"], w["fc1_w"], w["fc1_b"], w["fc2_w"], w["fc2_b"], windows=64)
    model.gen_keys()
    reqs = []
    for i in range(8):
        v, _ = tk.im2col_encode(inputs.mnist_like_image(320 + i), 7, 7, 3, ctx.slots)
        reqs.append(ctx.encrypt_values(v, 920 + i))
    singles = [model.forward(c).export() for c in reqs]
    vctx = tk.Context(tk.Params(12, [55, 40, 40, 56], 2.0 ** 40), seed=SEED,
                      flags=tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | tk.TCKS_DOUBLE_HOIST)
    n, m = 64, 10
    o = oracle.OracleCKKS(12, [55, 40, 40, 56], 2.0 ** 40)
    vctx.gen_galois_keys(o.vecmat_rect_steps(n, m))
    mat = vctx.matrix_encode_rect(inputs.random_matrix(n, m, 8, 0.5), level=3)
    vreqs = []
    for i in range(3):
        v = np.zeros(vctx.slots)
        v[:n] = inputs.uniform_slots(n, 60 + i)
        vreqs.append(vctx.encrypt_values(v, 760 + i))
    vsingles = [c.vecmat_plain(mat).export() for c in vreqs]
    return (ctx, model, reqs, singles), (vctx, mat, vreqs, vsingles)


def _mix_is_bit_identical(cnn, vm):
    ctx, model, reqs, singles = cnn
    vctx, mat, vreqs, vsingles = vm
    srv = tk.Server(hbm_budget_bytes=200 << 30, max_in_flight=64, max_batch=4)
    lane = srv.add_cnn(model)
    vlane = srv.add_vecmat(mat)
    ids = {}
    for i in range(5):
        ids[srv.submit(lane, reqs[i])] = ("cnn", i)
    ids[srv.submit(vlane, vreqs[0])] = ("vm", 0)
    srv.step()  # 4 CNN requests start (max_batch) and, on its own lane, the vector-matrix request
    st = srv.stats()
    assert st["queued"] == 0 and st["in_flight"] == 6
    for i in range(5, 8):  # arrive while the first requests are mid-pipeline
        ids[srv.submit(lane, reqs[i])] = ("cnn", i)
    for i in (1, 2):
        ids[srv.submit(vlane, vreqs[i])] = ("vm", i)
    done = {}
    for _ in range(400):
        srv.step()
        for rid in srv.poll():
            kind, i = ids[rid]
            done[rid] = srv.take(rid, ctx if kind == "cnn" else vctx).export()
        if len(done) == len(ids):
            break
    assert len(done) == len(ids)
    for rid, out in done.items():
        kind, i = ids[rid]
        ref = singles[i] if kind == "cnn" else vsingles[i]
        assert np.array_equal(out, ref), (kind, i)


def test_continuous_batching_mix_is_bit_identical(cnn, vm):
    _mix_is_bit_identical(cnn, vm)


def test_continuous_batching_mix_bench_layout(bench_lanes):
    """The same alone-versus-mix identity for the layout the benchmark's served trace uses."""
    _mix_is_bit_identical(*bench_lanes)


def test_budget_admission(cnn):
    ctx, model, reqs, singles = cnn
    probe = tk.Server(hbm_budget_bytes=1 << 60, max_in_flight=64, max_batch=64)
    lane = probe.add_cnn(model)
    resident = probe.stats()["bytes_resident"]
    per_req = (2 * 7 * ctx.N * 8) * 65
    tight = tk.Server(hbm_budget_bytes=resident + per_req - 1, max_in_flight=64, max_batch=64)
    tl = tight.add_cnn(model)
    with pytest.raises(tk.TcksError) as e:
        tight.submit(tl, reqs[0])
    assert e.value.name == "BUDGET_EXCEEDED"
    two = tk.Server(hbm_budget_bytes=resident + 2 * per_req, max_in_flight=64, max_batch=64)
    l2 = two.add_cnn(model)
    ids = [two.submit(l2, reqs[i]) for i in range(5)]
    two.step()
    st = two.stats()
    assert st["in_flight"] == 2 and st["queued"] == 3
    got = {}
    for _ in range(400):
        two.step()
        assert two.stats()["in_flight"] <= 2
        for rid in two.poll():
            got[rid] = two.take(rid, ctx).export()
        if len(got) == 5:
            break
    for k, rid in enumerate(ids):
        assert np.array_equal(got[rid], singles[k])
    with pytest.raises(tk.TcksError) as e:
        two.take(12345, ctx)
    assert e.value.name == "NOT_READY"


def test_allocator_failure_is_reported():
    """An allocator that starts refusing (injected on the host) turns into OUT_OF_MEMORY, and the
    context keeps working once allocations succeed again."""
    torch = pytest.importorskip("torch")
    state = {"n": 0, "limit": 10 ** 9}

    @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    def alloc(nbytes, stream, user):
        state["n"] += 1
        if state["n"] > state["limit"]:
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)

    @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    def free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = tk._Allocator(alloc, free, None)
    tk._CALLBACKS_IN_USE.append((a, alloc, free))  # the context frees through them after this test
    params = tk.Params(12, [36, 36, 36, 37], 2.0 ** 30)
    h = ctypes.c_void_p()
    tk.check(tk.lib().tcks_context_create(params.h, SEED, 3, ctypes.cast(ctypes.pointer(a), ctypes.c_void_p), None,
                                          ctypes.byref(h)))
    ctx = tk.Context.__new__(tk.Context)
    ctx.h, ctx.params, ctx.N, ctx.slots, ctx.primes, ctx.L = h, params, params.N, params.N // 2, params.primes, 3
    ctx._alloc_keep = (a, alloc, free)
    x = ctx.encrypt_values(inputs.uniform_slots(ctx.slots, 1), 5)
    state["limit"] = state["n"]  # every further allocation fails
    with pytest.raises(tk.TcksError) as e:
        x.mul(x)
    assert e.value.name == "OUT_OF_MEMORY"
    state["limit"] = 10 ** 9
    y = x.mul(x)
    assert np.max(np.abs(ctx.decrypt_values(y) - inputs.uniform_slots(ctx.slots, 1) ** 2)) < 1e-3
    del x, y, ctx  # the context (and its stream) go before any later test runs
    torch.cuda.synchronize()
