"""Independent big-integer re-derivation of CKKS for tiny N (test infrastructure).

No RNS, no fast transforms: polynomials are lists of Python integers modulo Q (or Q*P), products
are schoolbook negacyclic (X^N = -1), the NTT form is converted with the O(N^2) evaluation formula,
and every rounding division is the exact rational rule round(u / d) = floor((2u + d) / (2d)).
Used to pin the C++ oracle's RNS arithmetic (tensor product, relinearization, rescale, rotation).
"""
from __future__ import annotations

import math


def brv(x: int, bits: int) -> int:
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def primitive_2n_roots(q: int, n: int) -> list[int]:
    """All x with x^n == -1 mod q (the primitive 2n-th roots), found from one root by odd powers."""
    m = 2 * n
    assert (q - 1) % m == 0
    for x in range(2, q):
        c = pow(x, (q - 1) // m, q)
        if pow(c, n, q) == q - 1:
            return sorted(pow(c, k, q) for k in range(1, m, 2))
    raise ValueError("no root")


def negacyclic_mul(a: list[int], b: list[int], mod: int) -> list[int]:
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return [x % mod for x in out]


def ntt_eval(a: list[int], q: int, psi: int) -> list[int]:
    """out_j = a(psi^(2 brv(j) + 1)) mod q."""
    n = len(a)
    bits = n.bit_length() - 1
    out = []
    for j in range(n):
        w = pow(psi, 2 * brv(j, bits) + 1, q)
        acc, x = 0, 1
        for c in a:
            acc = (acc + c * x) % q
            x = x * w % q
        out.append(acc)
    return out


def ntt_interp(v: list[int], q: int, psi: int) -> list[int]:
    """Inverse of ntt_eval: a_i = N^-1 sum_j v_j psi^-(2 brv(j) + 1) i."""
    n = len(v)
    bits = n.bit_length() - 1
    ninv = pow(n, -1, q)
    ipsi = pow(psi, -1, q)
    out = []
    for i in range(n):
        acc = 0
        for j in range(n):
            acc += v[j] * pow(ipsi, (2 * brv(j, bits) + 1) * i, q)
        out.append(acc * ninv % q)
    return out


class TinyCKKS:
    """Big-integer view of RNS objects over a chain `primes` (data primes, then P)."""

    def __init__(self, n: int, primes: list[int], psis: list[int]):
        self.n = n
        self.primes = list(primes)
        self.L = len(primes) - 1
        self.P = primes[-1]
        self.psis = list(psis)

    def mods(self, level: int, with_p: bool = False) -> list[int]:
        idx = list(range(level)) + ([self.L] if with_p else [])
        return idx

    def to_int(self, limbs, idx: list[int]) -> list[int]:
        """NTT-form residues (one row per chain index in idx) -> coefficients mod prod(q_idx)."""
        qs = [self.primes[i] for i in idx]
        Q = math.prod(qs)
        coeff_rows = [ntt_interp([int(x) for x in limbs[r]], self.primes[i], self.psis[i]) for r, i in enumerate(idx)]
        out = []
        for k in range(self.n):
            x = 0
            for r, qi in enumerate(qs):
                Qi = Q // qi
                x += coeff_rows[r][k] * pow(Qi % qi, -1, qi) * Qi
            out.append(x % Q)
        return out

    def from_int(self, coeffs: list[int], idx: list[int]) -> list[list[int]]:
        return [ntt_eval([c % self.primes[i] for c in coeffs], self.primes[i], self.psis[i]) for i in idx]

    @staticmethod
    def round_div(u: int, d: int) -> int:
        return (2 * u + d) // (2 * d)

    @staticmethod
    def bal(x: int, q: int) -> int:
        x %= q
        return x if x <= (q - 1) // 2 else x - q

    def automorphism(self, a: list[int], g: int, mod: int) -> list[int]:
        n = self.n
        out = [0] * n
        for i, c in enumerate(a):
            e = i * g % (2 * n)
            if e < n:
                out[e] = c % mod
            else:
                out[e - n] = (-c) % mod
        return out

    def keyswitch_u(self, x: list[int], level: int, key, key_level: int) -> list[list[int]]:
        """u_b = sum_j bal_{q_j}(x) * ksk_j over Q_level * P (before the division by P)."""
        Q = math.prod(self.primes[:level])
        QP = Q * self.P
        key_rows = list(range(level)) + [key_level]
        idx = self.mods(level, with_p=True)
        u = [[0] * self.n, [0] * self.n]
        for j in range(level):
            qj = self.primes[j]
            d = [self.bal(c, qj) for c in x]
            for b in range(2):
                k = self.to_int([key[j][b][r] for r in key_rows], idx)
                prod = negacyclic_mul([c % QP for c in d], k, QP)
                u[b] = [(s + t) % QP for s, t in zip(u[b], prod)]
        return u

    def keyswitch(self, x: list[int], level: int, key, key_level: int) -> tuple[list[int], list[int]]:
        """x: coefficients mod Q_level. key: [K][2][K+1][N] NTT-form limbs.
        u = sum_j bal_{q_j}(x) * ksk_j over Q_level * P, out = round(u / P) mod Q_level."""
        Q = math.prod(self.primes[:level])
        u = self.keyswitch_u(x, level, key, key_level)
        return tuple([self.round_div(c, self.P) % Q for c in u[b]] for b in range(2))

    def rescale(self, c: list[int], level: int) -> list[int]:
        Q = math.prod(self.primes[:level])
        ql = self.primes[level - 1]
        return [self.round_div(v % Q, ql) % (Q // ql) for v in c]
