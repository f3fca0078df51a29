"""Checks run against the debug build of the library (TCKS_DEBUG_CHECKS=1 selects it; the build's
index and bounds checks on descriptor tables and the kernels' device range checks are compiled in).
Run as a script in its own process, since a process loads one build; prints one JSON line of results
that tests/test_gpu_debug_build.py asserts on. Needs a GPU."""
import json
import os
import sys

os.environ["TCKS_DEBUG_CHECKS"] = "1"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2104_03152_gb300 import build as tkbuild  # noqa: E402

tkbuild.build(debug=True)
import paper_2104_03152_gb300 as tk  # noqa: E402
from paper_2104_03152_gb300 import inputs  # noqa: E402

SEED = 20210406


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host(d):
    return d.cpu().numpy().view(np.uint64)


def selftest(log_n, polys, level, understate):
    """The descriptor declares `understate` limbs fewer than the grid covers: the kernels must skip
    those limbs (left as they were), transform the others exactly as the single call does, and set
    the limb-range bit of the error word."""
    g = tk.Context(tk.Params(log_n, [50, 40, 40, 60], 2.0 ** 30), seed=SEED)
    x = inputs.random_limbs(g.primes[:level], g.N, 300 + log_n, polys=polys)
    d, ref = dev(x), dev(x)
    g.ntt_inplace(ref.data_ptr(), polys, level, inverse=False)
    g.synchronize()
    word = tk.debug_selftest(g, d.data_ptr(), polys, level, understate)
    got, want = host(d).reshape(polys * level, g.N), host(ref).reshape(polys * level, g.N)
    kept = polys * level - understate
    return {"word": word, "transformed_equal": bool(np.array_equal(got[:kept], want[:kept])),
            "skipped_unchanged": bool(np.array_equal(got[kept:], x.reshape(polys * level, g.N)[kept:]))}


def overlap_refused():
    """Two NTT jobs of one batch whose outputs overlap: the debug build refuses the list before any
    launch."""
    g = tk.Context(tk.Params(13, [50, 40, 60], 2.0 ** 30), seed=SEED)
    d = torch.zeros((4, 2, g.N), dtype=torch.int64, device="cuda")
    torch.cuda.current_stream().synchronize()
    half = 2 * 2 * g.N * 8
    jobs = [(g, tk.JOB_NTT, 0, 2, 2, d.data_ptr(), d.data_ptr()),
            (g, tk.JOB_NTT, 0, 2, 2, d.data_ptr() + half // 2, d.data_ptr() + half // 2)]
    before = tk.launch_count()
    try:
        tk.batch_run(jobs)
        return {"refused": None, "launches": tk.launch_count() - before}
    except tk.TcksError as e:
        return {"refused": e.name, "launches": tk.launch_count() - before}


def clean_batch():
    """A mixed NTT / INTT / relinearize / rotate batch over two ring sizes: every check passes and
    the results equal the single calls."""
    out = {}
    ctxs = {}
    for log_n in (13, 14):
        g = tk.Context(tk.Params(log_n, [50, 40, 40, 60], 2.0 ** 30), seed=SEED, flags=tk.TCKS_AUTO_RELIN)
        g.gen_galois_keys([1])
        ctxs[log_n] = g
    jobs, checks = [], []
    for log_n, g in ctxs.items():
        x = inputs.random_limbs(g.primes[:3], g.N, 40 + log_n, polys=3)
        d_in, d_out = dev(x), torch.zeros((3, 3, g.N), dtype=torch.int64, device="cuda")
        jobs.append((g, tk.JOB_NTT, 0, 3, 3, d_in.data_ptr(), d_out.data_ptr()))
        checks.append(("ntt", g, x, d_in, d_out, 3, 3))
        r = inputs.random_limbs(g.primes[:3], g.N, 50 + log_n, polys=2)
        r_in, r_out = dev(r), torch.zeros((1, 2, 3, g.N), dtype=torch.int64, device="cuda")
        jobs.append((g, tk.JOB_ROTATE, 1, 1, 3, r_in.data_ptr(), r_out.data_ptr()))
        checks.append(("rotate", g, r, r_in, r_out, 1, 3))
    torch.cuda.current_stream().synchronize()
    tk.batch_run(jobs)
    for kind, g, x, d_in, d_out, count, level in checks:
        g.synchronize()
        if kind == "ntt":
            ref = dev(x)
            g.ntt_inplace(ref.data_ptr(), count, level, inverse=False)
            g.synchronize()
            out[f"ntt_{g.N}"] = bool(np.array_equal(host(d_out), host(ref)))
        else:
            ct = g.ct_import(x.reshape(2, level, g.N), 1.0)
            out[f"rotate_{g.N}"] = bool(np.array_equal(host(d_out).reshape(2, level, g.N), ct.rotate(1).export()))
    return out


if __name__ == "__main__":
    res = {"debug_checks": tk.debug_checks(),
           "selftest_n13": selftest(13, 3, 3, 2),
           "selftest_n14": selftest(14, 2, 4, 3),
           "overlap": overlap_refused(),
           "clean": clean_batch()}
    print(json.dumps(res))
