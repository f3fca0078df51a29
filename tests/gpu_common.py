"""Helpers shared by the GPU parity tests: paired oracle / GPU contexts on the same chain and seed."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2104_03152_gb300 as tk

SEED = 0x7E5EA1


class Pair:
    """An oracle context and a GPU context with the same chain, scale and key seed."""

    def __init__(self, log_n, bits, scale, flags=tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE, galois=(), key_level=None):
        self.o = oracle.OracleCKKS(log_n, bits, scale, key_seed=SEED).keygen()
        self.params = tk.Params(log_n, bits, scale)
        assert self.params.primes == self.o.primes
        self.g = tk.Context(self.params, seed=SEED, flags=flags)
        self.steps = []
        if galois:
            self.add_galois(galois, key_level)

    def add_galois(self, steps, key_level=None):
        steps = list(steps)
        self.o.gen_galois_keys(steps, key_level)
        self.g.gen_galois_keys(steps, key_level or 0)
        self.steps += steps

    def import_ct(self, ct: oracle.Ct) -> tk.Ciphertext:
        return self.g.ct_import(ct.data, ct.scale)

    def import_pt(self, pt: oracle.Pt) -> tk.Plaintext:
        return self.g.pt_import(pt.data, pt.scale)


def assert_ct_equal(gpu_ct: tk.Ciphertext, ref: oracle.Ct, what: str = ""):
    level, scale = gpu_ct.info()
    assert level == ref.level, f"{what}: level {level} != {ref.level}"
    assert scale == ref.scale, f"{what}: scale {scale!r} != {ref.scale!r}"
    got = gpu_ct.export()
    if not np.array_equal(got, ref.data):
        bad = np.argwhere(got != ref.data)
        raise AssertionError(f"{what}: {len(bad)} of {got.size} words differ, first at {bad[0].tolist()}")
