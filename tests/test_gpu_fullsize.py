"""Bit-exact oracle parity at the full sizes the benchmark reports, in the launch configurations that only
those sizes reach.

* The 4096 x 256 vector x plain matrix product (§3.1's diagonal method) in its rectangular form at
  N = 16384, primes [60, 40, 40 | 60], scale 2^40: 64-bit words, 255 hoisted rotations and 4
  rotate-and-adds, 260 Galois keys. Nine vectors in one batch take the per-rotation schedule past its
  512 MB bound on the P-limb scratch (two blocks of rotations); the double-hoisted schedule runs its
  64-bit-word accumulation. Both schedules run on the oracle's own diagonals (imported), and the first
  and last vector of the batch must equal the oracle's product bit for bit.
* Relinearization and rotation at N = 2^16 with 32 data primes of 50-59 bits (the top of the primitive
  sweep): eight ciphertexts in one job need 4.5 GB of key-switch scratch, so the job runs as two
  sub-batches under the 4 GB bound; every ciphertext must equal the oracle's.
"""
import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from gpu_common import SEED, assert_ct_equal
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROWS, COLS, VECS = 4096, 256, 9


@pytest.fixture(scope="module")
def c4():
    bits, scale = [60, 40, 40, 60], 2.0 ** 40
    o = oracle.OracleCKKS(14, bits, scale, key_seed=SEED).keygen()
    g = tk.Context(tk.Params(14, bits, scale), seed=SEED, flags=tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE)
    steps = o.vecmat_rect_steps(ROWS, COLS)
    assert len(steps) == 1 + 255 + 4
    o.gen_galois_keys(steps)
    g.gen_galois_keys(steps)
    for st in (steps[0], 1, 255, 2048):
        assert np.array_equal(g.export_key(tk.KEY_GALOIS, st), o.galois[st].data), st
    M = np.random.default_rng(7).normal(0.0, 0.05, size=(ROWS, COLS))
    vs = np.random.default_rng(6).normal(0.0, 1.0, size=(VECS, ROWS))
    cts = []
    for i in range(VECS):
        z = np.zeros(o.slots)
        z[:ROWS] = vs[i]
        cts.append(o.encrypt_values(z, 800 + i))
    level = cts[0].level
    ext = o.encode_matrix_rect_ext(M, level)  # [256][level + 1][N], the oracle's own encodings
    mat = g.matrix_import_rect(ext, ROWS, COLS, o.scale)
    return o, g, M, vs, cts, ext, mat


@pytest.mark.parametrize("double_hoist", [False, True], ids=["moddown-per-rotation", "double-hoisted"])
def test_c4_rect_full_size_matches_oracle(c4, double_hoist):
    o, g, M, vs, cts, ext, mat = c4
    flags = tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | (tk.TCKS_DOUBLE_HOIST if double_hoist else 0)
    g.set_flags(flags)
    try:
        outs = mat.vecmat_batch([g.ct_import(c.data, c.scale) for c in cts])
        level = cts[0].level
        diags = None if double_hoist else [oracle.Pt(np.ascontiguousarray(e[:level]), level, o.scale) for e in ext]
        for i in (0, VECS - 1):
            if double_hoist:
                ref = o.vecmat_rect(cts[i], ROWS, COLS, diags_ext=ext)
            else:
                ref = o.vecmat_rect(cts[i], ROWS, COLS, diags=diags)
            assert_ct_equal(outs[i], ref, f"vector {i}")
            assert np.max(np.abs(g.decrypt_values(outs[i])[:COLS] - vs[i] @ M)) < 1e-3
    finally:
        g.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE)


@pytest.fixture(scope="module")
def c3():
    chain = oracle.gen_primes(16, [59 - (i % 10) for i in range(32)] + [60])
    o = oracle.OracleCKKS(16, None, 2.0 ** 50, key_seed=SEED, primes=chain).keygen()
    g = tk.Context(tk.Params(16, primes=chain, scale=2.0 ** 50), seed=SEED, flags=tk.TCKS_AUTO_RELIN)
    o.gen_galois_keys([1])
    g.gen_galois_keys([1])
    return o, g


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("op", ["relinearize", "rotate"])
def test_c3_keyswitch_full_size_matches_oracle(c3, op):
    o, g = c3
    lv, count = 32, 8
    polys = 3 if op == "relinearize" else 2
    x = np.stack([inputs.random_limbs(o.primes[:lv], o.N, 4000 + 10 * polys + i, polys=polys) for i in range(count)])
    d_in = _dev(x)
    d_out = torch.empty((count, 2, lv, o.N), dtype=torch.int64, device="cuda")
    job = tk.JOB_RELIN if op == "relinearize" else tk.JOB_ROTATE
    tk.batch_run([(g, job, 1, count, lv, d_in.data_ptr(), d_out.data_ptr())])
    g.synchronize()
    got = d_out.cpu().numpy().view(np.uint64).reshape(count, 2, lv, o.N)
    del d_in, d_out
    torch.cuda.empty_cache()
    for i in range(count):
        if op == "relinearize":
            ref = o.relinearize(x[i], lv, 1.0).data
        else:
            ref = o.rotate(oracle.Ct(np.ascontiguousarray(x[i]), lv, 1.0), 1).data
        if not np.array_equal(got[i], ref):
            bad = np.argwhere(got[i] != ref)
            raise AssertionError(f"{op} ciphertext {i}: {len(bad)} words differ, first at {bad[0].tolist()}")
