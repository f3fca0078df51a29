"""The rotation-heavy vector x plain matrix workload at full size (the diagonal method of §3.1):
N = 16384, primes [60, 40, 40 | 60], scale 2^40, 4096-dim N(0, 1) vectors times a 4096 x 256
N(0, 0.05) matrix encoded as 4096 diagonals at level 3, 4095 Galois keys, 64 vectors per batch.

At this size the oracle would need the 12.9 GB key set on the host, so the checks are properties
that hold at any size (bit-exact oracle parity of the same schedule runs at smaller sizes in
test_gpu_composite.py): sampled batched results equal the single-vector call bit for bit, and every
result decrypts to v M within 1e-3 of the FP64 product."""
import numpy as np
import pytest

import paper_2104_03152_gb300 as tk
from gpu_common import SEED

pytestmark = pytest.mark.gpu

ROWS, COLS, BATCH = 4096, 256, 64


@pytest.fixture(scope="module")
def c4():
    ctx = tk.Context(tk.Params(14, [60, 40, 40, 60], 2.0 ** 40), seed=SEED, flags=tk.TCKS_AUTO_RELIN)
    steps = [ctx.slots - ROWS] + list(range(1, ROWS))
    ctx.gen_galois_keys(steps)
    M = np.random.default_rng(7).normal(0.0, 0.05, size=(ROWS, COLS))
    mat = ctx.matrix_encode(M, level=3)
    vs = np.random.default_rng(6).normal(0.0, 1.0, size=(BATCH, ROWS))
    cts = []
    for i in range(BATCH):
        z = np.zeros(ctx.slots)
        z[:ROWS] = vs[i]
        cts.append(ctx.encrypt_values(z, 600 + i))
    return ctx, M, mat, vs, cts


def test_c4_batch_matches_single_and_fp64(c4):
    ctx, M, mat, vs, cts = c4
    outs = mat.vecmat_batch(cts)
    for i in (0, 17, BATCH - 1):
        single = cts[i].vecmat_plain(mat)
        assert np.array_equal(outs[i].export(), single.export()), i
    err = 0.0
    for i in range(BATCH):
        y = ctx.decrypt_values(outs[i])
        err = max(err, float(np.max(np.abs(y[:COLS] - vs[i] @ M))))
    assert err < 1e-3, err


def test_c4_batch_rejects_mixed_levels(c4):
    ctx, M, mat, vs, cts = c4
    low = ctx.ct_import(cts[1].export(), cts[1].info()[1])
    low.mod_switch_(2)
    with pytest.raises(tk.TcksError) as e:
        mat.vecmat_batch([cts[0], low])
    assert e.value.name == "LEVEL_MISMATCH"


def test_c4_double_hoisted(c4):
    """The same workload with the ModDown once after the rotation sum: batch equals single, and the
    result decrypts to v M as accurately."""
    ctx, M, mat, vs, cts = c4
    ctx.set_flags(tk.TCKS_AUTO_RELIN | tk.TCKS_DOUBLE_HOIST)
    try:
        outs = mat.vecmat_batch(cts)
        for i in (0, BATCH - 1):
            assert np.array_equal(outs[i].export(), cts[i].vecmat_plain(mat).export()), i
        err = max(float(np.max(np.abs(ctx.decrypt_values(outs[i])[:COLS] - vs[i] @ M))) for i in range(0, BATCH, 7))
        assert err < 1e-3, err
    finally:
        ctx.set_flags(tk.TCKS_AUTO_RELIN)


def test_c4_rectangular_double_hoisted():
    """The rectangular form at full size: 255 hoisted rotations + 4 rotate-and-adds (260 Galois keys
    instead of 4096); batch equals single and slots < 256 decrypt to v M."""
    ctx = tk.Context(tk.Params(14, [60, 40, 40, 60], 2.0 ** 40), seed=SEED,
                     flags=tk.TCKS_AUTO_RELIN | tk.TCKS_DOUBLE_HOIST)
    steps = [ctx.slots - ROWS] + list(range(1, COLS)) + [COLS << j for j in range(4)]
    ctx.gen_galois_keys(steps)
    M = np.random.default_rng(7).normal(0.0, 0.05, size=(ROWS, COLS))
    mat = ctx.matrix_encode_rect(M, level=3)
    vs = np.random.default_rng(6).normal(0.0, 1.0, size=(8, ROWS))
    cts = []
    for i in range(8):
        z = np.zeros(ctx.slots)
        z[:ROWS] = vs[i]
        cts.append(ctx.encrypt_values(z, 800 + i))
    outs = mat.vecmat_batch(cts)
    assert np.array_equal(outs[3].export(), cts[3].vecmat_plain(mat).export())
    err = max(float(np.max(np.abs(ctx.decrypt_values(outs[i])[:COLS] - vs[i] @ M))) for i in range(8))
    assert err < 1e-3, err
