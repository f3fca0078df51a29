"""CKKSTensor (§2.3): an N-dimensional tensor of reals encrypted as a tensor of ciphertexts, with
optionally the first axis batched into the slots, on the GPU.

The ciphertexts are the elements of the grid (the shape without the batched axis) in C order, all in
one device array (tcks_cta); ciphertext i is encrypted with seed + i. Batched, it holds the B values
along axis 0 in slots [0, B); not batched, its one value in slot 0. This module is host bookkeeping
only (shapes, broadcasting, axes, index tables): every operation is one call into the C ABI, which
runs it as batched launches over the whole array.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import (TCKS_CTA_ADD, TCKS_CTA_MUL, TCKS_CTA_SUB, Ciphertext, Context, _p, _vp, check, lib)


class CKKSTensor:
    def __init__(self, ctx: Context, h, grid, batch: bool, B: int, clean: bool = True):
        self.ctx, self.h, self.grid, self.batch, self.B, self.clean = ctx, h, tuple(grid), batch, B, clean

    def __del__(self):
        if getattr(self, "h", None):
            lib().tcks_cta_free(self.h)
            self.h = None

    # ------------------------------------------------------------------------------ creation ----
    @classmethod
    def encrypt(cls, ctx: Context, values, batch: bool = False, seed: int = 0) -> "CKKSTensor":
        v = np.asarray(values, dtype=np.float64)
        if batch:
            B, grid = v.shape[0], v.shape[1:]
            if B > ctx.slots:
                raise ValueError("the batched axis exceeds the slot count")
            rows = np.ascontiguousarray(v.reshape(B, -1).T)
        else:
            B, grid = 1, v.shape
            rows = np.ascontiguousarray(v.reshape(-1, 1))
        h = _vp()
        check(lib().tcks_cta_encrypt(ctx.h, _p(rows), rows.shape[0], rows.shape[1], 0, seed, ctypes.byref(h)))
        return cls(ctx, h, grid, batch, B)

    @classmethod
    def from_limbs(cls, ctx: Context, limbs: np.ndarray, scale: float, grid, batch: bool, B: int) -> "CKKSTensor":
        """An encrypted tensor from host limbs [count][2][level][N] (for example another implementation's)."""
        limbs = np.ascontiguousarray(limbs, dtype=np.uint64)
        h = _vp()
        check(lib().tcks_cta_import(ctx.h, _p(limbs), limbs.shape[0], limbs.shape[2], scale, ctypes.byref(h)))
        return cls(ctx, h, grid, batch, B)

    def info(self):
        n, lv, sc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
        check(lib().tcks_cta_info(self.h, ctypes.byref(n), ctypes.byref(lv), ctypes.byref(sc)))
        return n.value, lv.value, sc.value

    @property
    def count(self) -> int:
        return self.info()[0]

    @property
    def level(self) -> int:
        return self.info()[1]

    @property
    def scale(self) -> float:
        return self.info()[2]

    @property
    def shape(self):
        return ((self.B,) if self.batch else ()) + self.grid

    def export(self) -> np.ndarray:
        n, lv, _ = self.info()
        out = np.empty((n, 2, lv, self.ctx.params.N), dtype=np.uint64)
        check(lib().tcks_cta_export(self.h, _p(out), out.size))
        return out

    def ciphertext(self, i: int) -> Ciphertext:
        h = _vp()
        check(lib().tcks_cta_get(self.h, i, ctypes.byref(h)))
        return Ciphertext(self.ctx, h)

    def decrypt(self) -> np.ndarray:
        vals = np.empty((self.count, self.B), dtype=np.float64)
        check(lib().tcks_cta_decrypt(self.h, _p(vals), self.B))
        if self.batch:
            return vals.T.reshape(self.shape)
        return vals[:, 0].reshape(self.grid)

    def _new(self, fn, *args, grid=None, batch=None, B=None, clean=None) -> "CKKSTensor":
        h = _vp()
        check(fn(*args, ctypes.byref(h)))
        return CKKSTensor(self.ctx, h, self.grid if grid is None else grid, self.batch if batch is None else batch,
                          self.B if B is None else B, self.clean if clean is None else clean)

    # ----------------------------------------------------------------------- re-arrangement ----
    def _combine(self, idx, w, mode: int, grid, clean=None) -> "CKKSTensor":
        idx = np.ascontiguousarray(idx, dtype=np.uint32)
        w = np.ascontiguousarray(np.broadcast_to(np.asarray(w, dtype=np.float64), idx.shape))
        outs, terms = (idx.shape[0], idx.shape[1]) if idx.ndim == 2 else (idx.size, 1)
        return self._new(lib().tcks_cta_combine, self.h, _p(idx), _p(w), outs, terms, mode, grid=grid, clean=clean)

    def gather(self, idx, grid) -> "CKKSTensor":
        return self._combine(np.asarray(idx).reshape(-1), 1.0, 0, tuple(grid))

    def broadcast_to(self, grid) -> "CKKSTensor":
        grid = tuple(grid)
        if grid == self.grid:
            return self
        return self.gather(np.broadcast_to(np.arange(self.count).reshape(self.grid), grid), grid)

    def reshape(self, grid) -> "CKKSTensor":
        """A new grid shape (the batched axis, if any, stays in the slots); shares nothing with self."""
        grid = tuple(grid)
        if int(np.prod(grid)) != self.count:
            raise ValueError("cannot reshape")
        return self.gather(np.arange(self.count), grid)

    def transpose(self, axes=None) -> "CKKSTensor":
        idx = np.arange(self.count).reshape(self.grid).transpose(axes)
        return self.gather(idx, idx.shape)

    def mod_switch(self, level: int) -> "CKKSTensor":
        t = self.gather(np.arange(self.count), self.grid)
        check(lib().tcks_cta_mod_switch(t.h, level))
        return t

    # --------------------------------------------------------------------- element-wise ops ----
    def _pair(self, other: "CKKSTensor"):
        if self.batch != other.batch or self.B != other.B:
            raise ValueError("tensors batched differently")
        grid = np.broadcast_shapes(self.grid, other.grid)
        a, b = self.broadcast_to(grid), other.broadcast_to(grid)
        la, lb = a.level, b.level
        if la > lb:
            a = a.mod_switch(lb)
        elif lb > la:
            b = b.mod_switch(la)
        return a, b, grid

    def _binary(self, op: int, other: "CKKSTensor", clean: bool) -> "CKKSTensor":
        a, b, grid = self._pair(other)
        return self._new(lib().tcks_cta_binary, op, a.h, b.h, grid=grid, clean=clean)

    def add(self, other):
        if isinstance(other, CKKSTensor):
            return self._binary(TCKS_CTA_ADD, other, self.clean and other.clean)
        return self._plain_op(TCKS_CTA_ADD, other)

    def sub(self, other):
        if isinstance(other, CKKSTensor):
            return self._binary(TCKS_CTA_SUB, other, self.clean and other.clean)
        return self._plain_op(TCKS_CTA_SUB, other)

    def mul(self, other):
        if isinstance(other, CKKSTensor):
            return self._binary(TCKS_CTA_MUL, other, self.clean or other.clean)
        return self._plain_op(TCKS_CTA_MUL, other)

    __add__, __sub__, __mul__ = add, sub, mul

    def __neg__(self):
        return self.negate()

    def negate(self):
        return self._new(lib().tcks_cta_negate, self.h)

    def square(self):
        return self.mul(self)

    def power(self, k: int):
        return self._new(lib().tcks_cta_power, self.h, k)

    def polyval(self, coeffs):
        a = np.ascontiguousarray(coeffs, dtype=np.float64)
        clean = self.clean and (a.size == 0 or a[0] == 0.0)
        return self._new(lib().tcks_cta_polyval, self.h, _p(a), a.size, clean=clean)

    def _plain_rows(self, plain):
        p = np.broadcast_to(np.asarray(plain, dtype=np.float64), self.shape)
        if self.batch:
            return np.ascontiguousarray(p.reshape(self.B, -1).T)
        return np.ascontiguousarray(p.reshape(-1, 1))

    def _plain_is_scalar_per_ct(self, plain) -> bool:
        p = np.asarray(plain)
        return (not self.batch) or p.ndim < len(self.shape) or p.shape[0] == 1

    def _plain_op(self, op: int, plain):
        rows = self._plain_rows(plain)
        if op == TCKS_CTA_MUL and self._plain_is_scalar_per_ct(plain):
            # each ciphertext times the constant polynomial of its value at the context scale
            return self._combine(np.arange(self.count), rows[:, 0], 1, self.grid)
        return self._new(lib().tcks_cta_plain, op, self.h, _p(rows), rows.shape[1])

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
            return self._new(lib().tcks_cta_sum_slots, self.h, B, batch=False, B=1, clean=True)
        g = ax - (1 if self.batch else 0)
        idx = np.moveaxis(np.arange(self.count).reshape(self.grid), g, -1)
        grid = idx.shape[:-1]
        return self._combine(idx.reshape(-1, idx.shape[-1]), 1.0, 0, grid)

    def dot(self, other: "CKKSTensor"):
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
        """grid (..., k) times a plain (k, p) matrix in one gathered combination and one rescale:
        out[..., j] = sum_t x[..., t] M[t, j], with the constant polynomial of M[t, j] at the scale."""
        M = np.asarray(M, dtype=np.float64)
        k, p = M.shape
        if self.grid[-1] != k:
            raise ValueError("inner dimensions differ")
        rows = self.count // k
        idx = (np.arange(rows)[:, None, None] * k + np.arange(k)[None, None, :]).repeat(p, axis=1)
        w = np.broadcast_to(M.T[None, :, :], (rows, p, k))
        return self._combine(idx.reshape(rows * p, k), w.reshape(rows * p, k), 1, self.grid[:-1] + (p,))
