"""Helpers shared by the GPU parity tests: paired oracle / GPU contexts on the same chain and seed."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2104_03152_gb300 as tk

SEED = 0x7E5EA1


class Pair:
    """An oracle context and a GPU context with the same chain, scale and key seed."""

    def __init__(self, log_n, bits, scale, flags=tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE, galois=(), key_level=None,
                 primes=None, n_special=1, alpha=1):
        self.o = oracle.OracleCKKS(log_n, bits, scale, key_seed=SEED, primes=primes, n_special=n_special,
                                   alpha=alpha).keygen()
        self.params = tk.Params(log_n, bits, scale, primes=self.o.primes if (primes or n_special > 1 or alpha > 1)
                                else None, n_special=n_special, alpha=alpha)
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


U53 = 2.0 ** -53


def encode_tie_bound(o: oracle.OracleCKKS, z: np.ndarray, scale: float) -> float:
    """Worst-case FP64 error of a coefficient scale*m_i before rounding, the oracle's and the GPU's
    together, up to a term 3u|scale*m_i| added per coefficient. The oracle sums n = len(z) products
    z_j cos(theta) directly: cos and the product cost two roundings, the running sum n - 1, so its
    error is at most (n + 3) u (2/N) scale sum|z| (the factor 2/N is exact, the scale one more
    relative rounding). The GPU's special FFT passes each input through log2(N/2) butterfly stages and
    a twiddle pre- and post-multiplication, each stage at most a complex product and an addition
    (about 4u, plus the twiddle's own error), bounded here by 8 log2(N) u (2/N) scale sum|z|."""
    z = np.asarray(z, dtype=np.float64)
    return U53 * (2.0 / o.N) * float(scale) * float(np.sum(np.abs(z))) * (len(z) + 3 + 8 * o.log_n)


def assert_encoding_agrees(o: oracle.OracleCKKS, got: np.ndarray, z, scale: float, level: int,
                           what: str = "") -> int:
    """A plaintext the GPU encoded, [level][N] or over the extended basis [level+1][N] (P last), NTT
    form, against the oracle's own encoding of the same slot values z at `scale` (reading A9): the
    same integer coefficients, except that a coefficient may differ by exactly one where the
    oracle's value before rounding lies within the FP64 error bound of a .5 tie. Every limb (P's
    included) must carry that same integer. Returns the number of near-tie coefficients."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    got = np.ascontiguousarray(got, dtype=np.uint64)
    ext = got.shape[0] == level + 1
    if ext:
        ref, pre = o.encode_ext(z, level, scale, want_pre=True)
    else:
        ref_pt, pre = o.encode(z, scale=scale, level=level, want_pre=True)
        ref = ref_pt.data
    assert got.shape == ref.shape, f"{what}: shape {got.shape} != {ref.shape}"
    if np.array_equal(got, ref):
        return 0
    idx = list(range(level)) + ([o.L] if ext else [])
    gc, rc = o.intt_rows(got, idx), o.intt_rows(ref, idx)
    cols = np.nonzero((gc != rc).any(axis=0))[0]
    q = np.array([o.q[i] for i in idx], dtype=np.uint64)[:, None]
    d = (gc[:, cols] + q - rc[:, cols]) % q  # got - ref in every limb
    up, down = np.all(d == 1, axis=0), np.all(d == q - 1, axis=0)
    assert np.all(up | down), f"{what}: {int(np.sum(~(up | down)))} coefficients differ by more than one"
    p = pre[cols]
    frac = np.abs(p - np.floor(p) - 0.5)
    bound = encode_tie_bound(o, z, scale) + 3 * U53 * np.abs(p)
    far = frac > bound
    assert not far.any(), (f"{what}: {int(far.sum())} of {len(cols)} differing coefficients are not near a .5 tie "
                           f"(first: index {int(cols[far][0])}, value {p[far][0]!r}, bound {bound[far][0]:.3e})")
    return len(cols)
