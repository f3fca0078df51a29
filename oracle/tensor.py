"""Oracle of TenSEAL's CKKSTensor (§2.3): an N-dimensional tensor of reals encrypted as a tensor of
ciphertexts, with optionally the first axis batched into the slots. Written plainly as loops over the
per-ciphertext oracle operations of ckks.py, in the order the tensor operations define them.

TEST INFRASTRUCTURE ONLY: imported by tests/; never by the GPU library.

Layout (the reading shared with the GPU tensor): the ciphertexts are the elements of the grid (the
shape without the batched axis) in C order; ciphertext i is encrypted with seed + i. Batched: it holds
the B values along axis 0 in slots [0, B). Not batched: it holds its one value in slot 0.
"""
from __future__ import annotations

import math

import numpy as np

from .ckks import Ct, OracleCKKS


class OracleTensor:
    def __init__(self, o: OracleCKKS, cts: list, grid: tuple, batch: bool, B: int, clean: bool = True):
        self.o, self.cts, self.grid, self.batch, self.B, self.clean = o, cts, tuple(grid), batch, B, clean

    # ------------------------------------------------------------------------------ creation ----
    @classmethod
    def encrypt(cls, o: OracleCKKS, values, batch: bool = False, seed: int = 0) -> "OracleTensor":
        v = np.asarray(values, dtype=np.float64)
        if batch:
            B, grid = v.shape[0], v.shape[1:]
            cols = v.reshape(B, -1).T  # [count][B]
        else:
            B, grid = 1, v.shape
            cols = v.reshape(-1, 1)
        cts = [o.encrypt(o.encode(cols[i], level=o.L), seed + i) for i in range(cols.shape[0])]
        return cls(o, cts, grid, batch, B)

    @property
    def shape(self):
        return ((self.B,) if self.batch else ()) + self.grid

    @property
    def level(self):
        return self.cts[0].level

    def _like(self, cts, grid=None, clean=None):
        return OracleTensor(self.o, cts, self.grid if grid is None else grid, self.batch, self.B,
                            self.clean if clean is None else clean)

    def decrypt(self) -> np.ndarray:
        vals = np.stack([self.o.decrypt_values(c, self.B) for c in self.cts])  # [count][B]
        if self.batch:
            return vals.T.reshape(self.shape)
        return vals[:, 0].reshape(self.grid)

    # ----------------------------------------------------------------------- re-arrangement ----
    def gather(self, idx, grid) -> "OracleTensor":
        return self._like([self.cts[i] for i in np.asarray(idx).reshape(-1)], grid)

    def broadcast_to(self, grid) -> "OracleTensor":
        grid = tuple(grid)
        if grid == self.grid:
            return self
        idx = np.broadcast_to(np.arange(len(self.cts)).reshape(self.grid), grid)
        return self.gather(idx, grid)

    def reshape(self, grid) -> "OracleTensor":
        return self._like(list(self.cts), tuple(grid))

    def transpose(self, axes=None) -> "OracleTensor":
        idx = np.arange(len(self.cts)).reshape(self.grid).transpose(axes)
        return self.gather(idx, idx.shape)

    def mod_switch(self, level: int) -> "OracleTensor":
        return self._like([self.o.mod_switch(c, level) for c in self.cts])

    # --------------------------------------------------------------------- element-wise ops ----
    def _pair(self, other: "OracleTensor"):
        if self.batch != other.batch or self.B != other.B:
            raise ValueError("tensors batched differently")
        grid = np.broadcast_shapes(self.grid, other.grid)
        a, b = self.broadcast_to(grid), other.broadcast_to(grid)
        lvl = min(a.level, b.level)
        return a.mod_switch(lvl), b.mod_switch(lvl), grid

    def add(self, other):
        if isinstance(other, OracleTensor):
            a, b, grid = self._pair(other)
            return a._like([self.o.add(x, y) for x, y in zip(a.cts, b.cts)], grid, a.clean and b.clean)
        return self._plain_op("add", other)

    def sub(self, other):
        if isinstance(other, OracleTensor):
            a, b, grid = self._pair(other)
            return a._like([self.o.sub(x, y) for x, y in zip(a.cts, b.cts)], grid, a.clean and b.clean)
        return self._plain_op("sub", other)

    def mul(self, other):
        if isinstance(other, OracleTensor):
            a, b, grid = self._pair(other)
            return a._like([self.o.mul(x, y) for x, y in zip(a.cts, b.cts)], grid, a.clean or b.clean)
        return self._plain_op("mul", other)

    def negate(self):
        return self._like([self.o.negate(c) for c in self.cts])

    def square(self):
        return self.mul(self)

    def power(self, k: int):
        return self._like([self.o.power(c, k) for c in self.cts])

    def polyval(self, coeffs):
        clean = self.clean and float(coeffs[0]) == 0.0
        return self._like([self.o.polyval(c, coeffs) for c in self.cts], clean=clean)

    def _plain_rows(self, plain):
        """The plain operand broadcast to the tensor's shape, as one row of slot values per ciphertext."""
        p = np.broadcast_to(np.asarray(plain, dtype=np.float64), self.shape)
        if self.batch:
            return p.reshape(self.B, -1).T
        return p.reshape(-1, 1)

    def _plain_is_scalar_per_ct(self, plain) -> bool:
        """True when the plain operand cannot vary inside a ciphertext: the tensor is not batched, or
        the operand has no batched axis of its own (fewer dimensions, or size 1 there)."""
        p = np.asarray(plain)
        if not self.batch:
            return True
        return p.ndim < len(self.shape) or p.shape[0] == 1

    def _plain_op(self, op, plain):
        o, rows = self.o, self._plain_rows(plain)
        if op == "mul" and self._plain_is_scalar_per_ct(plain):
            # the constant polynomial of each ciphertext's value at the context scale, then rescale
            out = [o.rescale(o.mul_plain(c, o.const_pt(rows[i][0], o.scale, c.level))) for i, c in enumerate(self.cts)]
            return self._like(out)
        out = []
        for i, c in enumerate(self.cts):
            if op == "mul":
                out.append(o.rescale(o.mul_plain(c, o.encode(rows[i], level=c.level))))
            else:
                pt = o.encode(rows[i], scale=c.scale, level=c.level)
                out.append(o.add_plain(c, pt) if op == "add" else o.sub_plain(c, pt))
        return self._like(out)

    # ----------------------------------------------------------------------------- reductions ----
    def sum(self, axis=None):
        if axis is None:
            t = self
            for _ in range(len(self.grid)):
                t = t.sum(-1)
            return t.sum(0) if t.batch else t
        nd = len(self.shape)
        ax = axis % nd
        if self.batch and ax == 0:
            B = self.B
            if not self.clean and B & (B - 1):
                raise ValueError("slots beyond the batch are not zero: sum over the batched axis needs B a power of two")
            out = []
            for c in self.cts:
                s = 1
                while s < B:
                    c = self.o.add(c, self.o.rotate(c, s))
                    s <<= 1
                out.append(c)
            return OracleTensor(self.o, out, self.grid, False, 1, True)
        g = ax - (1 if self.batch else 0)
        idx = np.moveaxis(np.arange(len(self.cts)).reshape(self.grid), g, -1)
        grid = idx.shape[:-1]
        out = []
        for row in idx.reshape(-1, idx.shape[-1]):
            acc = self.cts[row[0]]
            for i in row[1:]:
                acc = self.o.add(acc, self.cts[i])
            out.append(acc)
        return self._like(out, grid)

    def dot(self, other: "OracleTensor"):
        """1-D grids: sum of the products; 2-D grids: the matrix product."""
        if len(self.grid) == 1:
            return self.mul(other).sum(-1)
        m, k = self.grid
        k2, p = other.grid
        if k != k2:
            raise ValueError("inner dimensions differ")
        a = self.reshape((m, 1, k)).broadcast_to((m, p, k))
        b = other.transpose().reshape((1, p, k)).broadcast_to((m, p, k))
        return a.mul(b).sum(-1)

    def mm_plain(self, M):
        """grid (..., k) times a plain (k, p) matrix: out[..., j] = sum_t x[..., t] M[t, j], each product
        with the constant polynomial of M[t, j] at the context scale, one rescale per output."""
        M = np.asarray(M, dtype=np.float64)
        k, p = M.shape
        if self.grid[-1] != k:
            raise ValueError("inner dimensions differ")
        o = self.o
        rows = len(self.cts) // k
        out = []
        for r in range(rows):
            for j in range(p):
                acc = None
                for t in range(k):
                    c = self.cts[r * k + t]
                    term = o.mul_plain(c, o.const_pt(M[t, j], o.scale, c.level))
                    acc = term if acc is None else o.add(acc, term)
                out.append(o.rescale(acc))
        return self._like(out, self.grid[:-1] + (p,))
