"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no CKKS arithmetic: it only draws numbers (numpy's default_rng) in the shapes of the
paper's workloads (§5: a 28x28 MNIST-sized image in [0, 1], conv 4x7x7 stride 3, FC 256->64, FC
64->10) and of the primitive sweeps. The MNIST set and trained weights are not available, so seeded
uniform images and N(0, 0.1) weights stand in for them.
"""
from __future__ import annotations

import numpy as np

SEED_KEYS = 0x7E5EA1


def uniform_slots(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def normal_slots(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).normal(0.0, sigma, size=n)


def mnist_like_image(seed: int = 3, h: int = 28, w: int = 28) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(h, w))


def cnn_weights(seed: int = 4, kernels: int = 4, taps: int = 49, hidden: int = 64, windows: int = 64,
                classes: int = 10, sigma: float = 0.1) -> dict:
    """conv [kernels][taps], conv bias [kernels], fc1 [hidden][kernels*windows], fc1 bias, fc2
    [classes][hidden], fc2 bias; all N(0, sigma)."""
    r = np.random.default_rng(seed)
    return {
        "conv_w": r.normal(0, sigma, size=(kernels, taps)),
        "conv_b": r.normal(0, sigma, size=kernels),
        "fc1_w": r.normal(0, sigma, size=(hidden, kernels * windows)),
        "fc1_b": r.normal(0, sigma, size=hidden),
        "fc2_w": r.normal(0, sigma, size=(classes, hidden)),
        "fc2_b": r.normal(0, sigma, size=classes),
    }


def random_limbs(primes, n: int, seed: int, polys: int = 1) -> np.ndarray:
    """[polys][len(primes)][n] uniform residues, limb l uniform in [0, primes[l])."""
    r = np.random.default_rng(seed)
    out = np.empty((polys, len(primes), n), dtype=np.uint64)
    for p in range(polys):
        for l, q in enumerate(primes):
            out[p, l] = r.integers(0, int(q), size=n, dtype=np.uint64)
    return out


def random_matrix(rows: int, cols: int, seed: int, sigma: float) -> np.ndarray:
    return np.random.default_rng(seed).normal(0.0, sigma, size=(rows, cols))
