"""Python layer of the CPU oracle: ctypes bindings to liboracle.so, the exact big-integer CRT step of
decoding, and the composite schedules (sum, dot, vector x plain matrix, im2col convolution, the
MNIST-shaped CNN) written in the order their definitions state.

TEST INFRASTRUCTURE ONLY: imported by tests/, the package smoke check and the benchmark's
CPU-baseline leg; never by the GPU library. Shares no code with it.

The paper (TenSEAL) describes the operations at the level of its tensor API (§2-§3, Table 3); the
RNS-CKKS definitions each function follows are stated in its docstring.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from .build import build

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_dblp = ctypes.POINTER(ctypes.c_double)
_lib = None


def lib():
    """Load (building first if needed) the oracle's shared library."""
    global _lib
    if _lib is not None:
        return _lib
    L = ctypes.CDLL(build())
    u64, u32, i64, vp, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    sig = {
        "orc_is_prime": (i32, [u64]),
        "orc_gen_primes": (i32, [u32, _u32p, u32, _u64p]),
        "orc_min_psi": (u64, [u64, u32]),
        "orc_bit_reverse": (u32, [u32, u32]),
        "orc_philox4x64": (None, [_u64p, _u64p, _u64p]),
        "orc_ntt_naive": (None, [_u64p, _u64p, u32, u64, u64]),
        "orc_ntt": (None, [_u64p, u32, u64, u64]),
        "orc_intt": (None, [_u64p, u32, u64, u64]),
        "orc_ctx_new": (vp, [u32, _u64p, u32]),
        "orc_ctx_free": (None, [vp]),
        "orc_ctx_psi": (u64, [vp, u32]),
        "orc_ntt_limb": (None, [vp, _u64p, u32]),
        "orc_intt_limb": (None, [vp, _u64p, u32]),
        "orc_galois_elt": (u32, [vp, i64]),
        "orc_automorphism_ntt": (None, [vp, _u64p, u32, u32, _u64p]),
        "orc_automorphism_coeff": (None, [vp, _u64p, u64, u32, _u64p]),
        "orc_keygen_secret": (None, [vp, u64, _u64p]),
        "orc_keygen_public": (None, [vp, u64, _u64p, _u64p]),
        "orc_keygen_switch": (None, [vp, u64, u64, _u64p, _u64p, u32, _u64p]),
        "orc_keygen_relin": (None, [vp, u64, _u64p, u32, _u64p]),
        "orc_keygen_galois": (None, [vp, u64, _u64p, u32, u32, _u64p]),
        "orc_encode": (i32, [vp, _dblp, u32, ctypes.c_double, u32, _dblp, _u64p]),
        "orc_decode_sum": (None, [vp, _dblp, ctypes.c_double, u32, _dblp]),
        "orc_encrypt": (None, [vp, _u64p, _u64p, u32, u64, _u64p]),
        "orc_decrypt": (None, [vp, _u64p, _u64p, u32, _u64p]),
        "orc_decrypt_sized": (None, [vp, _u64p, _u64p, u32, u32, _u64p]),
        "orc_sample_sym_a": (None, [vp, u32, u64, _u64p]),
        "orc_encrypt_symmetric": (None, [vp, _u64p, _u64p, u32, u64, u64, _u64p]),
        "orc_relinearize_rescale": (None, [vp, _u64p, u32, _u64p, u32, _u64p]),
        "orc_add": (None, [vp, _u64p, _u64p, u32, u32, _u64p]),
        "orc_sub": (None, [vp, _u64p, _u64p, u32, u32, _u64p]),
        "orc_negate": (None, [vp, _u64p, u32, u32, _u64p]),
        "orc_add_plain": (None, [vp, _u64p, _u64p, u32, _u64p]),
        "orc_sub_plain": (None, [vp, _u64p, _u64p, u32, _u64p]),
        "orc_mul_plain": (None, [vp, _u64p, _u64p, u32, _u64p]),
        "orc_tensor": (None, [vp, _u64p, _u64p, u32, _u64p]),
        "orc_rescale": (None, [vp, _u64p, u32, _u64p]),
        "orc_rescale_polys": (None, [vp, _u64p, u32, u32, _u64p]),
        "orc_mul_plain_polys": (None, [vp, _u64p, _u64p, u32, u32, _u64p]),
        "orc_modup": (None, [vp, _u64p, u32, _u64p]),
        "orc_encode_ext": (i32, [vp, _dblp, u32, ctypes.c_double, u32, _dblp, _u64p]),
        "orc_vecmat_dh": (None, [vp, _u64p, _u64p, u32, u32, _u64p, ctypes.POINTER(_u64p), _u32p, _u32p, _u64p]),
        "orc_vecmat_dh_rs": (None, [vp, _u64p, _u64p, u32, u32, _u64p, ctypes.POINTER(_u64p), _u32p, _u32p, _u64p]),
        "orc_keyswitch_digits": (None, [vp, _u64p, u32, _u64p, u32, u32, _u64p]),
        "orc_keyswitch": (None, [vp, _u64p, u32, _u64p, u32, _u64p]),
        "orc_relinearize": (None, [vp, _u64p, u32, _u64p, u32, _u64p]),
        "orc_rotate": (None, [vp, _u64p, u32, u32, _u64p, u32, _u64p]),
        "orc_rotate_from_digits": (None, [vp, _u64p, _u64p, u32, u32, _u64p, u32, _u64p]),
        "orc_ctx_new_hybrid": (vp, [u32, _u64p, u32, u32]),
        "orc_keygen_switch_hyb": (None, [vp, u64, u64, _u64p, _u64p, u32, u32, _u64p]),
        "orc_keygen_relin_hyb": (None, [vp, u64, _u64p, u32, u32, _u64p]),
        "orc_keygen_galois_hyb": (None, [vp, u64, _u64p, u32, u32, u32, _u64p]),
        "orc_modup_hyb": (None, [vp, _u64p, u32, u32, _u64p]),
        "orc_keyswitch_digits_hyb": (None, [vp, _u64p, u32, u32, _u64p, u32, u32, _u64p]),
        "orc_keyswitch_hyb": (None, [vp, _u64p, u32, u32, _u64p, u32, _u64p]),
        "orc_relinearize_hyb": (None, [vp, _u64p, u32, u32, _u64p, u32, _u64p]),
        "orc_rotate_hyb": (None, [vp, _u64p, u32, u32, u32, _u64p, u32, _u64p]),
        "orc_rotate_from_digits_hyb": (None, [vp, _u64p, _u64p, u32, u32, u32, _u64p, u32, _u64p]),
        "orc_max_threads": (i32, []),
        "orc_set_threads": (None, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def P(a: np.ndarray):
    """Pointer to a C-contiguous uint64 / uint32 / float64 numpy array."""
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    if a.dtype == np.uint64:
        return a.ctypes.data_as(_u64p)
    if a.dtype == np.uint32:
        return a.ctypes.data_as(_u32p)
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dblp)
    raise TypeError(a.dtype)


# ------------------------------------------------------------------------------ free functions --

def is_prime(n: int) -> bool:
    return bool(lib().orc_is_prime(n))


def gen_primes(log_n: int, bits) -> list[int]:
    b = np.ascontiguousarray(bits, dtype=np.uint32)
    out = np.zeros(len(bits), dtype=np.uint64)
    if lib().orc_gen_primes(log_n, P(b), len(bits), P(out)) != 0:
        raise ValueError(f"no NTT-friendly primes for bits={list(bits)} at N=2^{log_n}")
    return [int(x) for x in out]


def min_psi(q: int, log_n: int) -> int:
    return int(lib().orc_min_psi(q, log_n))


def philox4x64(ctr, key) -> list[int]:
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(P(c), P(k), P(o))
    return [int(x) for x in o]


def ntt_naive(a, q: int, psi: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().orc_ntt_naive(P(a), P(out), int(len(a)).bit_length() - 1, q, psi)
    return out


def ntt(a, q: int, psi: int) -> np.ndarray:
    a = np.array(a, dtype=np.uint64)
    lib().orc_ntt(P(a), int(len(a)).bit_length() - 1, q, psi)
    return a


def intt(a, q: int, psi: int) -> np.ndarray:
    a = np.array(a, dtype=np.uint64)
    lib().orc_intt(P(a), int(len(a)).bit_length() - 1, q, psi)
    return a


def power_products(ks) -> list[tuple[int, int, int]]:
    """The products (i, a, b), x^i = x^a x^b, of a minimum-depth circuit for x^k, k in ks (§3, power):
    x^(2m) = (x^m)^2, and for i not a power of two x^i = x^(2^m) x^(i - 2^m) with 2^m the largest power
    of two below i. Each x^i then has depth ceil(log2 i), the lower bound for a product of i factors.
    Listed in increasing i, so both operands of a product come before it."""
    need = set()

    def visit(i):
        if i == 1 or i in need:
            return
        need.add(i)
        m = 1 << (i.bit_length() - 1)
        if m == i:
            visit(i // 2)
        else:
            visit(m)
            visit(i - m)

    for k in ks:
        visit(int(k))
    out = []
    for i in sorted(need):
        m = 1 << (i.bit_length() - 1)
        out.append((i, i // 2, i // 2) if m == i else (i, m, i - m))
    return out


# ------------------------------------------------------------------------ ciphertext records --

@dataclass
class Ct:
    """A CKKSVector ciphertext: data [2][level][N] (NTT form), its level and its scale."""
    data: np.ndarray
    level: int
    scale: float


@dataclass
class Pt:
    """An encoded plaintext: data [level][N] (NTT form), its level and its scale."""
    data: np.ndarray
    level: int
    scale: float


@dataclass
class SwitchKey:
    """A switching key of level K: [K][2][K+1][N] (limb K is the special prime), or with hybrid key
    switching [ceil(K/alpha)][2][K+n_special][N] (limbs K.. are the special primes)."""
    data: np.ndarray
    level: int


class OracleCKKS:
    """RNS-CKKS over the chain q_0..q_{L-1} (data primes) and P (special prime).

    Mirrors the TenSEAL context of §2.1: it owns the secret, public, relinearization and Galois keys,
    and the context-wide default scale.
    """

    def __init__(self, log_n: int, bits, scale: float, key_seed: int = 0x7E5EA1, primes=None, n_special: int = 1,
                 alpha: int = 1):
        """n_special > 1 or alpha > 1: hybrid key switching (reading A26) with digits of `alpha` data
        primes and the last `n_special` primes of the chain as the special primes."""
        self.log_n = log_n
        self.N = 1 << log_n
        self.slots = self.N // 2
        self.primes = list(primes) if primes is not None else gen_primes(log_n, bits)
        self.q = self.primes
        self.K = int(n_special)
        self.alpha = int(alpha)
        self.hybrid = self.K > 1 or self.alpha > 1
        self.L = len(self.primes) - self.K
        self.Pspecial = self.primes[-1]
        self.scale = float(scale)
        self.key_seed = key_seed
        arr = np.array(self.primes, dtype=np.uint64)
        if self.hybrid:
            self._ctx = lib().orc_ctx_new_hybrid(log_n, P(arr), len(self.primes), self.K)
        else:
            self._ctx = lib().orc_ctx_new(log_n, P(arr), len(self.primes))
        if not self._ctx:
            raise ValueError("a prime of the chain has no primitive 2N-th root")
        self.s = None
        self.pk = None
        self.rlk = None
        self.galois = {}

    def __del__(self):
        if getattr(self, "_ctx", None):
            lib().orc_ctx_free(self._ctx)
            self._ctx = None

    # ------------------------------------------------------------------------------- keys ----
    def keygen(self, relin_level: int | None = None):
        """Secret, public and relinearization keys from the context seed (§2.1)."""
        N, L = self.N, self.L
        self.s = np.zeros((len(self.primes), N), dtype=np.uint64)
        lib().orc_keygen_secret(self._ctx, self.key_seed, P(self.s))
        self.pk = np.zeros((2, L, N), dtype=np.uint64)
        lib().orc_keygen_public(self._ctx, self.key_seed, P(self.s), P(self.pk))
        K = L if relin_level is None else relin_level
        rlk = np.zeros(self.switch_key_shape(K), dtype=np.uint64)
        if self.hybrid:
            lib().orc_keygen_relin_hyb(self._ctx, self.key_seed, P(self.s), self.alpha, K, P(rlk))
        else:
            lib().orc_keygen_relin(self._ctx, self.key_seed, P(self.s), K, P(rlk))
        self.rlk = SwitchKey(rlk, K)
        return self

    def digits(self, level: int) -> int:
        """Key-switching digits at `level`: one per data prime, or ceil(level / alpha) (hybrid)."""
        return -(-level // self.alpha)

    def switch_key_shape(self, key_level: int) -> tuple:
        return (self.digits(key_level), 2, key_level + self.K, self.N)

    def galois_elt(self, step: int) -> int:
        return int(lib().orc_galois_elt(self._ctx, step))

    def gen_galois_key(self, step: int, key_level: int | None = None) -> SwitchKey:
        """Galois key for a left rotation by `step` slots, trimmed to `key_level` (default L)."""
        K = self.L if key_level is None else key_level
        g = self.galois_elt(step)
        gk = np.zeros(self.switch_key_shape(K), dtype=np.uint64)
        if self.hybrid:
            lib().orc_keygen_galois_hyb(self._ctx, self.key_seed, P(self.s), g, self.alpha, K, P(gk))
        else:
            lib().orc_keygen_galois(self._ctx, self.key_seed, P(self.s), g, K, P(gk))
        self.galois[step % self.slots] = SwitchKey(gk, K)
        return self.galois[step % self.slots]

    def gen_galois_keys(self, steps, key_level: int | None = None):
        for st in steps:
            self.gen_galois_key(st, key_level)

    # -------------------------------------------------------------------- encode / decode ----
    def encode(self, z, scale: float | None = None, level: int | None = None, want_pre: bool = False):
        """Encode real slot values (O9); returns Pt (and the pre-rounding scale*m_i if asked)."""
        z = np.ascontiguousarray(z, dtype=np.float64)
        scale = self.scale if scale is None else float(scale)
        level = self.L if level is None else level
        pt = np.zeros((level, self.N), dtype=np.uint64)
        pre = np.zeros(self.N, dtype=np.float64)
        st = lib().orc_encode(self._ctx, P(z), len(z), scale, level, P(pre), P(pt))
        if st == -1:
            raise ValueError("encode: bad size or level")
        if st == -2:
            raise OverflowError("encode: |scale * m_i| >= 2^62")
        out = Pt(pt, level, scale)
        return (out, pre) if want_pre else out

    def intt_limbs(self, limbs: np.ndarray, level: int) -> np.ndarray:
        out = np.array(limbs, dtype=np.uint64, copy=True).reshape(level, self.N)
        for l in range(level):
            row = np.ascontiguousarray(out[l])
            lib().orc_intt_limb(self._ctx, P(row), l)
            out[l] = row
        return out

    def intt_rows(self, limbs: np.ndarray, chain_idx) -> np.ndarray:
        """Inverse NTT of rows [k][N], row r modulo the chain's prime chain_idx[r] (P is index L)."""
        out = np.array(limbs, dtype=np.uint64, copy=True).reshape(len(chain_idx), self.N)
        for r, l in enumerate(chain_idx):
            row = np.ascontiguousarray(out[r])
            lib().orc_intt_limb(self._ctx, P(row), l)
            out[r] = row
        return out

    def crt_compose(self, coeffs: np.ndarray, level: int) -> list[int]:
        """Exact CRT of coefficient-domain residues [level][N] to centred integers in (-Q/2, Q/2]."""
        qs = self.q[:level]
        Q = math.prod(qs)
        terms = []
        for l, ql in enumerate(qs):
            Ql = Q // ql
            terms.append((ql, pow(Ql % ql, -1, ql), Ql))
        rows = [[int(v) for v in coeffs[l]] for l in range(level)]
        out = []
        half = Q // 2
        for i in range(self.N):
            x = 0
            for l, (ql, inv, Ql) in enumerate(terms):
                x += (rows[l][i] * inv % ql) * Ql
            x %= Q
            if x > half:
                x -= Q
            out.append(x)
        return out

    def decode(self, pt: Pt, n: int | None = None) -> np.ndarray:
        """Decode (O10): INTT, exact CRT to centred integers, round to double, canonical embedding."""
        n = self.slots if n is None else n
        coeffs = self.intt_limbs(pt.data, pt.level)
        ints = self.crt_compose(coeffs, pt.level)
        p = np.array([float(x) for x in ints], dtype=np.float64)
        z = np.zeros(n, dtype=np.float64)
        lib().orc_decode_sum(self._ctx, P(p), pt.scale, n, P(z))
        return z

    # ------------------------------------------------------------------ encrypt / decrypt ----
    def encrypt(self, pt: Pt, seed: int) -> Ct:
        """Public-key encryption at the plaintext's level (O11)."""
        ct = np.zeros((2, pt.level, self.N), dtype=np.uint64)
        data = np.ascontiguousarray(pt.data)
        lib().orc_encrypt(self._ctx, P(self.pk), P(data), pt.level, seed, P(ct))
        return Ct(ct, pt.level, pt.scale)

    def encrypt_symmetric(self, pt: Pt, seed_a: int, seed_e: int) -> Ct:
        """Secret-key encryption (-a s + e + m, a): a uniform from the public seed seed_a, e from the
        private seed seed_e. The pair travels as c0 and seed_a (wire kind 1)."""
        ct = np.zeros((2, pt.level, self.N), dtype=np.uint64)
        lib().orc_encrypt_symmetric(self._ctx, P(self.s), P(np.ascontiguousarray(pt.data)), pt.level, seed_a, seed_e,
                                    P(ct))
        return Ct(ct, pt.level, pt.scale)

    def sample_sym_a(self, level: int, seed_a: int) -> np.ndarray:
        a = np.zeros((level, self.N), dtype=np.uint64)
        lib().orc_sample_sym_a(self._ctx, level, seed_a, P(a))
        return a

    def decrypt(self, ct: Ct) -> Pt:
        """m = c0 + c1 s (O11); a three-component ciphertext (an unrelinearized product) adds c2 s^2."""
        pt = np.zeros((ct.level, self.N), dtype=np.uint64)
        size = ct.data.shape[0]
        if size == 2:
            lib().orc_decrypt(self._ctx, P(self.s), P(np.ascontiguousarray(ct.data)), ct.level, P(pt))
        else:
            lib().orc_decrypt_sized(self._ctx, P(self.s), P(np.ascontiguousarray(ct.data)), ct.level, size, P(pt))
        return Pt(pt, ct.level, ct.scale)

    def encrypt_values(self, z, seed: int, level: int | None = None) -> Ct:
        return self.encrypt(self.encode(z, level=level), seed)

    def decrypt_values(self, ct: Ct, n: int | None = None) -> np.ndarray:
        return self.decode(self.decrypt(ct), n)

    # ------------------------------------------------------------------- element-wise ops ----
    @staticmethod
    def _check_pair(a: Ct, b: Ct):
        if a.level != b.level:
            raise ValueError("level mismatch")
        if a.scale != b.scale:
            raise ValueError("scale mismatch")

    def _same_size(self, a: Ct, b: Ct) -> tuple[np.ndarray, np.ndarray]:
        """Both operands' components, the shorter one padded with zero polynomials (a missing
        component of a ciphertext is the zero polynomial: m = sum_k c_k s^k)."""
        k = max(a.data.shape[0], b.data.shape[0])

        def pad(x):
            if x.shape[0] == k:
                return np.ascontiguousarray(x)
            return np.ascontiguousarray(np.concatenate([x, np.zeros((k - x.shape[0],) + x.shape[1:], np.uint64)]))
        return pad(a.data), pad(b.data)

    def add(self, a: Ct, b: Ct) -> Ct:
        self._check_pair(a, b)
        x, y = self._same_size(a, b)
        out = np.zeros_like(x)
        lib().orc_add(self._ctx, P(x), P(y), a.level, x.shape[0], P(out))
        return Ct(out, a.level, a.scale)

    def sub(self, a: Ct, b: Ct) -> Ct:
        self._check_pair(a, b)
        x, y = self._same_size(a, b)
        out = np.zeros_like(x)
        lib().orc_sub(self._ctx, P(x), P(y), a.level, x.shape[0], P(out))
        return Ct(out, a.level, a.scale)

    def negate(self, a: Ct) -> Ct:
        out = np.zeros_like(a.data)
        lib().orc_negate(self._ctx, P(np.ascontiguousarray(a.data)), a.level, a.data.shape[0], P(out))
        return Ct(out, a.level, a.scale)

    def _plain_for(self, ct: Ct, pt: Pt) -> np.ndarray:
        if pt.level < ct.level:
            raise ValueError("plaintext level below ciphertext level")
        return np.ascontiguousarray(pt.data[: ct.level])

    def add_plain(self, ct: Ct, pt: Pt) -> Ct:
        if pt.scale != ct.scale:
            raise ValueError("scale mismatch")
        out = np.array(ct.data, copy=True)  # a third component is unchanged
        lib().orc_add_plain(self._ctx, P(np.ascontiguousarray(ct.data[:2])), P(self._plain_for(ct, pt)), ct.level,
                            P(out[:2]))
        return Ct(out, ct.level, ct.scale)

    def sub_plain(self, ct: Ct, pt: Pt) -> Ct:
        if pt.scale != ct.scale:
            raise ValueError("scale mismatch")
        out = np.array(ct.data, copy=True)
        lib().orc_sub_plain(self._ctx, P(np.ascontiguousarray(ct.data[:2])), P(self._plain_for(ct, pt)), ct.level,
                            P(out[:2]))
        return Ct(out, ct.level, ct.scale)

    def mul_plain(self, ct: Ct, pt: Pt) -> Ct:
        out = np.zeros_like(ct.data)
        polys = ct.data.shape[0]
        if polys == 2:
            lib().orc_mul_plain(self._ctx, P(ct.data), P(self._plain_for(ct, pt)), ct.level, P(out))
        else:
            lib().orc_mul_plain_polys(self._ctx, P(np.ascontiguousarray(ct.data)), P(self._plain_for(ct, pt)), ct.level,
                                      polys, P(out))
        return Ct(out, ct.level, ct.scale * pt.scale)

    def tensor(self, a: Ct, b: Ct) -> tuple[np.ndarray, int, float]:
        """(d0, d1, d2) of O13 as [3][level][N], with scale a.scale * b.scale."""
        if a.level != b.level:
            raise ValueError("level mismatch")
        out = np.zeros((3, a.level, self.N), dtype=np.uint64)
        lib().orc_tensor(self._ctx, P(a.data), P(b.data), a.level, P(out))
        return out, a.level, a.scale * b.scale

    def relinearize(self, d3: np.ndarray, level: int, scale: float) -> Ct:
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        if self.hybrid:
            lib().orc_relinearize_hyb(self._ctx, P(np.ascontiguousarray(d3)), level, self.alpha, P(self.rlk.data),
                                      self.rlk.level, P(out))
        else:
            lib().orc_relinearize(self._ctx, P(np.ascontiguousarray(d3)), level, P(self.rlk.data), self.rlk.level,
                                  P(out))
        return Ct(out, level, scale)

    def relinearize_rescale(self, d3: np.ndarray, level: int, scale: float) -> Ct:
        """Relinearization and rescale with one rounding (reading A25): [2][level-1][N]."""
        if self.hybrid:
            raise NotImplementedError("the merged rounding is defined for one special prime and one-prime digits")
        out = np.zeros((2, level - 1, self.N), dtype=np.uint64)
        lib().orc_relinearize_rescale(self._ctx, P(np.ascontiguousarray(d3)), level, P(self.rlk.data), self.rlk.level,
                                      P(out))
        return Ct(out, level - 1, scale / float(self.q[level - 1]))

    def rescale(self, ct: Ct) -> Ct:
        """Divide by the last prime with rounding (O14)."""
        if ct.level < 2:
            raise ValueError("level exhausted")
        polys = ct.data.shape[0]
        out = np.zeros((polys, ct.level - 1, self.N), dtype=np.uint64)
        if polys == 2:
            lib().orc_rescale(self._ctx, P(np.ascontiguousarray(ct.data)), ct.level, P(out))
        else:  # every component of a three-component ciphertext on its own
            lib().orc_rescale_polys(self._ctx, P(np.ascontiguousarray(ct.data)), ct.level, polys, P(out))
        return Ct(out, ct.level - 1, ct.scale / float(self.q[ct.level - 1]))

    def mod_switch(self, ct: Ct, level: int) -> Ct:
        """Drop limbs level..ell-1; the scale is unchanged (O19)."""
        return Ct(np.ascontiguousarray(ct.data[:, :level]), level, ct.scale)

    def mul(self, a: Ct, b: Ct, relin: bool = True, rescale: bool = True, merged: bool = False) -> Ct:
        """enc x enc multiply with the context's auto relinearize / rescale policy (§2.1); merged: the
        relinearization's ModDown and the rescale as one rounding (A25)."""
        d3, level, scale = self.tensor(a, b)
        if not relin:  # the three-component product, rescaled component by component if asked
            ct = Ct(d3, level, scale)
            return self.rescale(ct) if rescale else ct
        if merged and rescale:
            if level < 2:
                raise ValueError("level exhausted")
            return self.relinearize_rescale(d3, level, scale)
        ct = self.relinearize(d3, level, scale)
        return self.rescale(ct) if rescale else ct

    def relinearize_ct(self, ct: Ct) -> Ct:
        """A three-component ciphertext relinearized to two (O17); a two-component one is returned as is."""
        if ct.data.shape[0] == 2:
            return ct
        return self.relinearize(ct.data, ct.level, ct.scale)

    def square(self, a: Ct) -> Ct:
        return self.mul(a, a)

    # ------------------------------------------------------------- power and polyval (§3) ----
    def const_pt(self, a: float, scale: float, level: int) -> Pt:
        """The plaintext of the real constant a at `scale`: the constant polynomial c = rint(a * scale)
        (round half to even of the FP64 product). A constant polynomial evaluates to c at every root, so
        its canonical embedding is c in every slot and its NTT is c mod q_j at every point."""
        v = float(a) * float(scale)
        if not abs(v) < 2.0 ** 62:
            raise OverflowError("|a * scale| >= 2^62")
        c = int(np.rint(v))
        data = np.empty((level, self.N), dtype=np.uint64)
        for j in range(level):
            data[j, :] = c % self.q[j]
        return Pt(data, level, float(scale))

    def power(self, ct: Ct, k: int) -> Ct:
        """x^k element-wise with the minimum multiplicative depth ceil(log2 k) (§3, power): the products
        of power_products, each operand pair brought to the lower of their levels by dropping limbs,
        then multiplied, relinearized and rescaled."""
        if k < 1:
            raise ValueError("k must be >= 1")
        return self._powers(ct, [k])[k]

    def _powers(self, ct: Ct, ks) -> dict:
        pw = {1: ct}
        for i, a, b in power_products(ks):
            A, B = pw[a], pw[b]
            lvl = min(A.level, B.level)
            if lvl < 2:
                raise ValueError("level exhausted")
            pw[i] = self.mul(self.mod_switch(A, lvl), self.mod_switch(B, lvl))
        return pw

    def polyval(self, ct: Ct, coeffs) -> Ct:
        """p(x) = sum_i a_i x^i element-wise (§3, polyval) with the minimum depth ceil(log2 d) + 1.

        The powers with a_i != 0 come from one minimum-depth power table (_powers). With l_min the lowest
        of their levels, every term is taken to level l_min (limbs dropped), multiplied by the constant
        a_i encoded at scale t_i = S q / s_i, where S is the context scale, q the prime q_{l_min - 1}
        that the final rescale divides by and s_i the term's scale, so that every product has the
        scale S q; the products are added, rescaled once, and the result, whose scale is S, gets a_0
        encoded at scale S added. Result level l_min - 1."""
        a = [float(c) for c in coeffs]
        while a and a[-1] == 0.0:
            a.pop()
        ks = [i for i in range(1, len(a)) if a[i] != 0.0]
        if not ks:
            raise ValueError("polyval needs a non-zero coefficient of degree >= 1")
        pw = self._powers(ct, ks)
        lt = min(pw[i].level for i in ks)
        if lt < 2:
            raise ValueError("level exhausted")
        S, q = self.scale, float(self.q[lt - 1])
        acc = None
        for i in ks:
            t = self.mod_switch(pw[i], lt)
            u = self.mul_plain(t, self.const_pt(a[i], S * q / t.scale, lt))
            u = Ct(u.data, lt, S * q)
            acc = u if acc is None else self.add(acc, u)
        res = self.rescale(acc)
        res = Ct(res.data, res.level, S)
        if a[0] != 0.0:
            res = self.add_plain(res, self.const_pt(a[0], S, res.level))
        return res

    # ----------------------------------------------------------------------------- rotate ----
    def _key(self, step: int) -> SwitchKey:
        k = step % self.slots
        if k not in self.galois:
            raise KeyError(f"no Galois key for step {step}")
        return self.galois[k]

    def rotate(self, ct: Ct, step: int) -> Ct:
        """Left rotation by `step` slots (O18): automorphism then key switch."""
        if step % self.slots == 0:
            return Ct(ct.data.copy(), ct.level, ct.scale)
        key = self._key(step)
        out = np.zeros_like(ct.data)
        if self.hybrid:
            lib().orc_rotate_hyb(self._ctx, P(np.ascontiguousarray(ct.data)), ct.level, self.alpha, self.galois_elt(step),
                                 P(key.data), key.level, P(out))
        else:
            lib().orc_rotate(self._ctx, P(ct.data), ct.level, self.galois_elt(step), P(key.data), key.level, P(out))
        return Ct(out, ct.level, ct.scale)

    def modup(self, ct: Ct) -> np.ndarray:
        """Digits of c1 for hoisted rotations: [level][level+1][N], or [ceil(level/alpha)][level+K][N]."""
        return self.modup_poly(np.ascontiguousarray(ct.data[1]), ct.level)

    def modup_poly(self, x: np.ndarray, level: int) -> np.ndarray:
        """ModUp (O16) of one NTT-form polynomial [level][N]."""
        d = np.zeros((self.digits(level), level + self.K, self.N), dtype=np.uint64)
        x = np.ascontiguousarray(x, dtype=np.uint64)
        if self.hybrid:
            lib().orc_modup_hyb(self._ctx, P(x), level, self.alpha, P(d))
        else:
            lib().orc_modup(self._ctx, P(x), level, P(d))
        return d

    def rotate_from_digits(self, ct: Ct, digits: np.ndarray, step: int) -> Ct:
        if step % self.slots == 0:
            return Ct(ct.data.copy(), ct.level, ct.scale)
        key = self._key(step)
        out = np.zeros_like(ct.data)
        if self.hybrid:
            lib().orc_rotate_from_digits_hyb(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), ct.level,
                                             self.alpha, self.galois_elt(step), P(key.data), key.level, P(out))
        else:
            lib().orc_rotate_from_digits(self._ctx, P(ct.data), P(digits), ct.level, self.galois_elt(step),
                                         P(key.data), key.level, P(out))
        return Ct(out, ct.level, ct.scale)

    def rotate_hoisted(self, ct: Ct, steps) -> list[Ct]:
        """Several rotations of one ciphertext sharing one ModUp of c1 (O18)."""
        digits = self.modup(ct)
        return [self.rotate_from_digits(ct, digits, s) for s in steps]

    def keyswitch(self, x: np.ndarray, level: int, key: SwitchKey) -> np.ndarray:
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        if self.hybrid:
            lib().orc_keyswitch_hyb(self._ctx, P(np.ascontiguousarray(x)), level, self.alpha, P(key.data), key.level,
                                    P(out))
        else:
            lib().orc_keyswitch(self._ctx, P(np.ascontiguousarray(x)), level, P(key.data), key.level, P(out))
        return out

    def keyswitch_digits(self, digits: np.ndarray, level: int, key: SwitchKey, g: int = 1) -> np.ndarray:
        """The inner product of (automorphed) digits with a key and the ModDown: [2][level][N]."""
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        if self.hybrid:
            lib().orc_keyswitch_digits_hyb(self._ctx, P(np.ascontiguousarray(digits)), level, self.alpha,
                                           P(key.data), key.level, g, P(out))
        else:
            lib().orc_keyswitch_digits(self._ctx, P(np.ascontiguousarray(digits)), level, P(key.data), key.level, g,
                                       P(out))
        return out

    # ---------------------------------------------------------------- composite schedules ----
    def sum_steps(self) -> list[int]:
        return [1 << m for m in range(self.log_n - 1)]

    def sum(self, ct: Ct, n: int) -> Ct:
        """Rotate-and-add over all N/2 slots (O20); slots >= n must be zero. Every slot ends up with
        the total."""
        if n > self.slots:
            raise ValueError("n exceeds the slot count")
        for m in range(self.log_n - 1):
            ct = self.add(ct, self.rotate(ct, 1 << m))
        return ct

    def dot(self, a: Ct, b: Ct, n: int) -> Ct:
        """enc . enc dot product (§3.1): sum(rescale(relin(a x b)), n)."""
        return self.sum(self.mul(a, b), n)

    def dot_plain(self, a: Ct, w, n: int) -> Ct:
        """enc . plain dot product (§3.1): sum(rescale(a * enc(w)), n)."""
        pt = self.encode(w, level=a.level)
        return self.sum(self.rescale(self.mul_plain(a, pt)), n)

    def replicate_steps(self, n: int, period: int | None = None) -> list[int]:
        """Left-rotation steps that replicate an n-vector over all N/2 slots (§3.1). With `period`, the
        input already repeats with that period (the vector in [0, n), zeros in [n, period)): only the
        steps that take the period down to n."""
        reps = (self.slots if period is None else period) // n
        return [self.slots - n * (1 << m) for m in range(int(math.log2(reps)))]

    def matrix_diagonals(self, M: np.ndarray) -> list[np.ndarray]:
        """Generalised diagonals d_k[s] = M[(s+k) mod n][s] for s < m, 0 elsewhere (O21)."""
        n, m = M.shape
        out = []
        for k in range(n):
            d = np.zeros(self.slots, dtype=np.float64)
            for s in range(m):
                d[s] = M[(s + k) % n][s]
            out.append(d)
        return out

    def encode_matrix(self, M: np.ndarray, level: int) -> list[Pt]:
        return [self.encode(d, level=level) for d in self.matrix_diagonals(np.asarray(M, dtype=np.float64))]

    def encode_ext(self, z, level: int, scale: float | None = None, want_pre: bool = False):
        """Encode (O9) over the extended basis: [level+1][N], limbs q_0..q_{level-1} then P (and the
        pre-rounding scale*m_i if asked)."""
        z = np.ascontiguousarray(z, dtype=np.float64)
        scale = self.scale if scale is None else float(scale)
        out = np.zeros((level + 1, self.N), dtype=np.uint64)
        pre = np.zeros(self.N, dtype=np.float64)
        st = lib().orc_encode_ext(self._ctx, P(z), len(z), scale, level, P(pre), P(out))
        if st:
            raise ValueError(f"encode_ext failed ({st})")
        return (out, pre) if want_pre else out

    @staticmethod
    def rect_width(m: int) -> int:
        """Diagonals of the rectangular form: the smallest power of two >= m."""
        return 1 << max(0, (m - 1).bit_length())

    def matrix_diagonals_rect(self, M: np.ndarray) -> list[np.ndarray]:
        """Rectangular (hybrid) diagonals of an n x m matrix, m' = rect_width(m) <= n of them:
        d_k[t] = M[(t' + k) mod n][t' mod m'] with t' = t mod n, zero where t' mod m' >= m (all N/2
        slots, period n)."""
        M = np.asarray(M, dtype=np.float64)
        n, m = M.shape
        mw = self.rect_width(m)
        if mw > n:
            raise ValueError("more outputs than inputs")
        t = np.arange(self.slots) % n
        cols = t % mw
        out = []
        for k in range(mw):
            d = np.zeros(self.slots)
            ok = cols < m
            d[ok] = M[(t[ok] + k) % n, cols[ok]]
            out.append(d)
        return out

    def encode_matrix_rect(self, M: np.ndarray, level: int) -> list[Pt]:
        return [self.encode(d, level=level) for d in self.matrix_diagonals_rect(M)]

    def encode_matrix_rect_ext(self, M: np.ndarray, level: int) -> np.ndarray:
        return np.stack([self.encode_ext(d, level) for d in self.matrix_diagonals_rect(M)])

    def vecmat_rect_steps(self, n: int, m: int) -> list[int]:
        mw = self.rect_width(m)
        chain = [mw << j for j in range(int(math.log2(n // mw)))]
        return (self.replicate_steps(n) if n < self.slots else []) + list(range(1, mw)) + chain

    def vecmat_rect(self, ct: Ct, n: int, m: int, diags: list[Pt] | None = None,
                    diags_ext: np.ndarray | None = None, replicate: bool = True, period: int | None = None,
                    merged: bool = False) -> Ct:
        """Vector x plain n x m matrix by the rectangular diagonal method: replicate, y' = sum over
        the m' = rect_width(m) diagonals of rot(ct, k) * d_k (hoisted; with one ModDown per rotation
        when `diags` is given, or once after the sum when `diags_ext` is), rescale, then
        log2(n / m') rotate-and-adds by m' 2^j. Slots s < m hold y_s = sum_i v_i M[i][s]; with the
        input replicated over all slots (period n) every slot s holds the entry s mod m' (zero where
        s mod m' >= m): the product comes out replicated with period m'. replicate=False: the input is
        already replicated with period n; `period`: the input repeats with that period (see
        replicate_steps)."""
        mw = self.rect_width(m)
        if diags_ext is not None:
            y = self._vecmat_dh_rows(ct, diags_ext, n, mw, replicate, period, merged)
        else:
            y = self._vecmat_rows(ct, diags, n, mw, replicate, period)
        for j in range(int(math.log2(n // mw))):
            y = self.add(y, self.rotate(y, mw << j))
        return y

    def _vecmat_rows(self, ct: Ct, diags: list[Pt], n: int, rows: int, replicate: bool = True,
                     period: int | None = None) -> Ct:
        """Replicate an n-vector, then sum_{k < rows} rot(ct, k) * d_k (hoisted), then rescale."""
        if replicate and n < self.slots:
            for st in self.replicate_steps(n, period):
                ct = self.add(ct, self.rotate(ct, st))
        digits = self.modup(ct)
        acc = None
        for k in range(rows):
            r = ct if k == 0 else self.rotate_from_digits(ct, digits, k)
            t = self.mul_plain(r, diags[k])
            acc = t if acc is None else self.add(acc, t)
        return self.rescale(acc)

    def _vecmat_dh_rows(self, ct: Ct, diags_ext: np.ndarray, n: int, rows: int, replicate: bool = True,
                        period: int | None = None, merged: bool = False) -> Ct:
        """The same with the ModDown once after the sum (orc_vecmat_dh over `rows` diagonals); merged:
        the ModDown and the rescale as one rounding (orc_vecmat_dh_rs, A25)."""
        level = ct.level
        if replicate and n < self.slots:
            for st in self.replicate_steps(n, period):
                ct = self.add(ct, self.rotate(ct, st))
        digits = self.modup(ct)
        keys = [self._key(k) for k in range(1, rows)]
        key_arrs = [np.ascontiguousarray(k.data) for k in keys]
        ptrs = (_u64p * max(1, len(keys)))(*[P(a) for a in key_arrs])
        lv = np.array([k.level for k in keys] or [0], dtype=np.uint32)
        ge = np.array([self.galois_elt(k) for k in range(1, rows)] or [1], dtype=np.uint32)
        if merged:
            out = np.zeros((2, level - 1, self.N), dtype=np.uint64)
            lib().orc_vecmat_dh_rs(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, rows,
                                   P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
            return Ct(out, level - 1, ct.scale * self.scale / float(self.q[level - 1]))
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        lib().orc_vecmat_dh(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, rows,
                            P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
        return self.rescale(Ct(out, level, ct.scale * self.scale))

    def dh_sum(self, ct: Ct, steps, diags_ext: np.ndarray, merged: bool = False) -> Ct:
        """sum_k rot(ct, s_k) * d_k with s_0 = 0 and s_k = steps[k - 1], the diagonals d_k given over
        the extended basis [len(steps) + 1][level + 1][N], with one ModUp before and one ModDown after
        the sum (orc_vecmat_dh). The scale is the ciphertext's times the diagonals' (no rescale)."""
        steps = list(steps)
        level = ct.level
        rows = len(steps) + 1
        if diags_ext.shape != (rows, level + 1, self.N):
            raise ValueError("diagonals do not match the steps and the level")
        digits = self.modup(ct)
        keys = [self._key(st) for st in steps]
        key_arrs = [np.ascontiguousarray(k.data) for k in keys]
        ptrs = (_u64p * max(1, len(keys)))(*[P(a) for a in key_arrs])
        lv = np.array([k.level for k in keys] or [0], dtype=np.uint32)
        ge = np.array([self.galois_elt(st) for st in steps] or [1], dtype=np.uint32)
        if merged:  # with the rescale, one rounding (A25)
            out = np.zeros((2, level - 1, self.N), dtype=np.uint64)
            lib().orc_vecmat_dh_rs(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, rows,
                                   P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
            return Ct(out, level - 1, ct.scale * self.scale / float(self.q[level - 1]))
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        lib().orc_vecmat_dh(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, rows,
                            P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
        return Ct(out, level, ct.scale * self.scale)

    def rotsum_dh(self, ct: Ct, steps) -> Ct:
        """ct + sum over `steps` of rot(ct, s), hoisted with one ModDown after the sum: orc_vecmat_dh
        with every diagonal the constant polynomial 1 (all ones in NTT form over the extended basis),
        rotation k taking steps[k - 1]. No rescale: the scale is unchanged."""
        steps = list(steps)
        level = ct.level
        rows = len(steps) + 1
        ones = np.ones((rows, level + 1, self.N), dtype=np.uint64)
        digits = self.modup(ct)
        keys = [self._key(st) for st in steps]
        key_arrs = [np.ascontiguousarray(k.data) for k in keys]
        ptrs = (_u64p * max(1, len(keys)))(*[P(a) for a in key_arrs])
        lv = np.array([k.level for k in keys] or [0], dtype=np.uint32)
        ge = np.array([self.galois_elt(st) for st in steps] or [1], dtype=np.uint32)
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        lib().orc_vecmat_dh(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, rows, P(ones), ptrs, P(lv),
                            P(ge), P(out))
        return Ct(out, level, ct.scale)

    @staticmethod
    def conv_bsgs_steps(taps: int, windows: int) -> tuple[list[int], list[int]]:
        """Baby and giant steps of the hoisted convolution sum: the 2^ceil(log2 taps) tap positions
        t = b + B g (b < B, g < G) with B = 2^floor(e/2), G = 2^ceil(e/2)."""
        e = (taps - 1).bit_length()
        nb, ng = 1 << (e // 2), 1 << (e - e // 2)
        return [windows * b for b in range(1, nb)], [windows * nb * g for g in range(1, ng)]

    def conv2d_im2col_hoisted(self, ct: Ct, kernel_pt: Pt, taps: int, windows: int) -> Ct:
        """The im2col convolution with its rotate-and-add chain replaced by two hoisted rotation sums
        (baby steps, then giant steps), each with one ModDown: rescale(ct * kernel), then
        x1 = sum_{b < B} rot(x, windows b), x2 = sum_{g < G} rot(x1, windows B g); the same sum over
        all 2^ceil(log2 taps) taps as the chain."""
        x = self.rescale(self.mul_plain(ct, kernel_pt))
        baby, giant = self.conv_bsgs_steps(taps, windows)
        return self.rotsum_dh(self.rotsum_dh(x, baby), giant)

    def conv_baby_diagonals_ext(self, kernel_slots: np.ndarray, taps: int, windows: int, level: int) -> np.ndarray:
        """The baby-step diagonals of the shared convolution sum: the kernel's slot vector rotated left
        by each baby step (0 first), over the extended basis at `level`: [B][level+1][N]."""
        baby, _ = self.conv_bsgs_steps(taps, windows)
        return np.stack([self.encode_ext(np.roll(kernel_slots, -s), level) for s in [0] + baby])

    def conv2d_im2col_shared(self, ct: Ct, baby_ext: np.ndarray, taps: int, windows: int) -> Ct:
        """The hoisted convolution sum with the kernel multiplied after the baby-step rotations:
        x1 = sum_{b < B} rot(ct * K, windows b) = sum_b rot(ct, windows b) * rot(K, windows b), a
        diagonal-method sum over the input's own rotations (one ModUp of ct, shared by every kernel of
        the layer, one ModDown per kernel), rescaled; then the giant steps as before,
        sum_{g < G} rot(x1, windows B g)."""
        baby, giant = self.conv_bsgs_steps(taps, windows)
        x1 = self.rescale(self.dh_sum(ct, baby, baby_ext))
        return self.rotsum_dh(x1, giant)

    def encode_matrix_ext(self, M: np.ndarray, level: int) -> np.ndarray:
        """The diagonals over the extended basis: [n][level+1][N]."""
        return np.stack([self.encode_ext(d, level) for d in self.matrix_diagonals(np.asarray(M, dtype=np.float64))])

    def vecmat_steps(self, n: int) -> list[int]:
        steps = self.replicate_steps(n) if n < self.slots else []
        return steps + list(range(1, n))

    def vecmat(self, ct: Ct, diags: list[Pt], n: int, m: int, period: int | None = None) -> Ct:
        """Encrypted vector (slots [0, n), zeros elsewhere) times a plain n x m matrix given as
        pre-encoded diagonals (§3.1, the diagonal method with left rotations only and a replicated
        input): replicate, then y = sum_k rot(ct, k) * d_k with hoisted rotations, then rescale."""
        if len(diags) != n or m > n:
            raise ValueError("bad matrix shape")
        if n < self.slots:
            for st in self.replicate_steps(n, period):
                ct = self.add(ct, self.rotate(ct, st))
        digits = self.modup(ct)
        acc = None
        for k in range(n):
            r = ct if k == 0 else self.rotate_from_digits(ct, digits, k)
            t = self.mul_plain(r, diags[k])
            acc = t if acc is None else self.add(acc, t)
        return self.rescale(acc)

    def vecmat_dh(self, ct: Ct, diags_ext: np.ndarray, n: int, m: int, scale: float | None = None,
                  period: int | None = None, merged: bool = False) -> Ct:
        """The same product with the ModDown taken once after the sum over rotations (double
        hoisting): replicate, ModUp(c1) once, then orc_vecmat_dh (steps 1-3 there), then rescale.
        diags_ext [n][level+1][N] at the ciphertext's level; `scale` is the diagonals' scale."""
        level = ct.level
        if diags_ext.shape != (n, level + 1, self.N) or m > n:
            raise ValueError("bad matrix shape")
        if n < self.slots:
            for st in self.replicate_steps(n, period):
                ct = self.add(ct, self.rotate(ct, st))
        digits = self.modup(ct)
        keys = [self._key(k) for k in range(1, n)]
        key_arrs = [np.ascontiguousarray(k.data) for k in keys]
        ptrs = (_u64p * max(1, len(keys)))(*[P(a) for a in key_arrs])
        lv = np.array([k.level for k in keys] or [0], dtype=np.uint32)
        ge = np.array([self.galois_elt(k) for k in range(1, n)] or [1], dtype=np.uint32)
        d_scale = self.scale if scale is None else float(scale)
        if merged:
            out = np.zeros((2, level - 1, self.N), dtype=np.uint64)
            lib().orc_vecmat_dh_rs(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, n,
                                   P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
            return Ct(out, level - 1, ct.scale * d_scale / float(self.q[level - 1]))
        out = np.zeros((2, level, self.N), dtype=np.uint64)
        lib().orc_vecmat_dh(self._ctx, P(np.ascontiguousarray(ct.data)), P(digits), level, n,
                            P(np.ascontiguousarray(diags_ext)), ptrs, P(lv), P(ge), P(out))
        return self.rescale(Ct(out, level, ct.scale * d_scale))

    @staticmethod
    def im2col(img: np.ndarray, kh: int, kw: int, stride: int, slots: int):
        """Client-side im2col (§3.2): windows as rows (row-major windows, row-major taps), flattened
        by a vertical scan: slot t*W + w holds tap t of window w. Returns (slot vector, W)."""
        H, Wd = img.shape
        oh = (H - kh) // stride + 1
        ow = (Wd - kw) // stride + 1
        windows = oh * ow
        taps = kh * kw
        if taps * windows > slots:
            raise ValueError("image does not fit the slots")
        v = np.zeros(slots, dtype=np.float64)
        for r in range(oh):
            for c in range(ow):
                w = r * ow + c
                for t in range(taps):
                    v[t * windows + w] = img[stride * r + t // kw][stride * c + t % kw]
        return v, windows

    def conv_steps(self, taps: int, windows: int) -> list[int]:
        return [windows * (1 << m) for m in range(int(math.ceil(math.log2(taps))))]

    def conv2d_im2col_pt(self, ct: Ct, kernel_pt: Pt, taps: int, windows: int) -> Ct:
        """One kernel of the im2col convolution (§3.2): one multiplication by the replicated kernel,
        rescale, then log2(taps) left rotate-and-adds by windows * 2^m. Block-w of every 'windows'
        slots then holds the output for window w."""
        out = self.rescale(self.mul_plain(ct, kernel_pt))
        for st in self.conv_steps(taps, windows):
            out = self.add(out, self.rotate(out, st))
        return out

    def kernel_slots(self, kernel: np.ndarray, windows: int) -> np.ndarray:
        """Plain kernel laid out to match the vertical scan: slot t*W + w holds kernel tap t."""
        k = np.asarray(kernel, dtype=np.float64).reshape(-1)
        v = np.zeros(self.slots, dtype=np.float64)
        for t in range(len(k)):
            v[t * windows: (t + 1) * windows] = k[t]
        return v

    def conv2d_im2col(self, ct: Ct, kernel, windows: int) -> Ct:
        k = np.asarray(kernel, dtype=np.float64).reshape(-1)
        pt = self.encode(self.kernel_slots(k, windows), level=ct.level)
        return self.conv2d_im2col_pt(ct, pt, len(k), windows)


@dataclass
class CNNWeights:
    """Weights of the MNIST-shaped network of §5: conv 4x7x7 stride 3, square, FC 256->64, square,
    FC 64->10."""
    conv_w: np.ndarray  # [4][49]
    conv_b: np.ndarray  # [4]
    fc1_w: np.ndarray   # [64][256]
    fc1_b: np.ndarray   # [64]
    fc2_w: np.ndarray   # [10][64]
    fc2_b: np.ndarray   # [10]


@dataclass
class EncodedCNN:
    """Plaintexts of the CNN schedule, encoded at the levels the schedule uses them."""
    conv: list = field(default_factory=list)   # per kernel, level L
    masks: list = field(default_factory=list)  # per kernel, level L-1
    fc1: list = field(default_factory=list)    # 256 diagonals, level L-3
    fc2: list = field(default_factory=list)    # 64 diagonals, level L-5
    fc1_ext: np.ndarray | None = None          # the same over the extended basis [256][L-2][N]
    fc2_ext: np.ndarray | None = None          # [64][L-4][N]
    windows: int = 64
    taps: int = 49
    rect: bool = False                         # fully connected layers by rectangular diagonals
    biases: list | None = None                 # pre-encoded biases (Pt) in place of encoding them here
    conv_hoist: bool = False                   # convolution sums by hoisted baby-step giant-step rotation sums
    conv_shared: bool = False                  # baby steps on the input's rotations, shared by the kernels
    conv_baby_ext: list = field(default_factory=list)  # per kernel, its baby-step diagonals [B][L+1][N]
    pack_first: bool = False                   # channels packed after the baby steps, one giant-step sum
    fold: bool = False                         # the masks folded into the shared baby-step diagonals
    conv_baby_fold_ext: np.ndarray | None = None  # sum_k mask_k * (kernel k's baby diagonal b): [B][L+1][N]


def cnn_galois_steps(o: OracleCKKS, windows=64, taps=49, n1=256, n2=64, classes=10, rect=False, conv_hoist=False,
                     conv_shared=False, pack_first=False):
    """Galois steps of the CNN schedule with the level each is used at (key trimming). rect: the fully
    connected layers by rectangular diagonals (FC2 takes FC1's output as it comes, replicated)."""
    L = o.L
    need = {}

    def use(steps, level):
        for s in steps:
            s %= o.slots
            if s:
                need[s] = max(need.get(s, 0), level)

    period = None
    if pack_first:  # the giant steps rotate the packed vector at L - 2, which repeats with period B windows
        baby, giant = o.conv_bsgs_steps(taps, windows)
        use(baby, L if conv_shared else L - 1)
        use(giant, L - 2)
        period = (len(baby) + 1) * windows
    elif conv_shared:  # baby steps rotate the input at level L
        baby, giant = o.conv_bsgs_steps(taps, windows)
        use(baby, L)
        use(giant, L - 1)
    elif conv_hoist:
        baby, giant = o.conv_bsgs_steps(taps, windows)
        use(baby + giant, L - 1)
    else:
        use(o.conv_steps(taps, windows), L - 1)
    if rect:
        m1w, m2w = o.rect_width(n2), o.rect_width(classes)
        use(o.replicate_steps(n1, period) + list(range(1, m1w)), L - 3)
        use([m1w << j for j in range(int(math.log2(n1 // m1w)))], L - 4)
        use(list(range(1, m2w)), L - 5)
        use([m2w << j for j in range(int(math.log2(n2 // m2w)))], L - 6)
        return need
    use(o.replicate_steps(n1, period) + list(range(1, n1)), L - 3)
    use(o.vecmat_steps(n2), L - 5)
    return need


def cnn_mask_slots(o: OracleCKKS, k: int, windows: int, nb: int, pack_first: bool) -> np.ndarray:
    """The 0/1 mask that selects kernel k's output for the pack: its own block of windows, or, when the
    channels are packed before the giant steps, the windows-blocks k + nb g (what the giant-step sum
    gathers into block k)."""
    mask = np.zeros(o.slots)
    if pack_first:
        blk = np.arange(o.slots) // windows
        mask[blk % nb == k] = 1.0
    else:
        mask[k * windows: (k + 1) * windows] = 1.0
    return mask


def cnn_encode(o: OracleCKKS, w: CNNWeights, windows=64, rect=False, conv_hoist=False,
               conv_shared=False, pack_first=False, fold=False) -> EncodedCNN:
    L = o.L
    if fold and not (conv_shared and pack_first):
        raise ValueError("folding the masks needs the shared baby steps and the pack before the giant steps")
    e = EncodedCNN(windows=windows, taps=w.conv_w.shape[1], conv_hoist=conv_hoist, conv_shared=conv_shared,
                   pack_first=pack_first, fold=fold)
    nb = len(o.conv_bsgs_steps(e.taps, windows)[0]) + 1
    if fold:
        # reading A27: mask_k * sum_b rot(x, s_b) * d_kb summed over k is sum_b rot(x, s_b) * (sum_k mask_k * d_kb)
        # slot by slot, so one diagonal-method sum over the folded diagonals gives the packed vector
        baby, _ = o.conv_bsgs_steps(e.taps, windows)
        kern = [o.kernel_slots(w.conv_w[k], windows) for k in range(w.conv_w.shape[0])]
        masks = [cnn_mask_slots(o, k, windows, nb, True) for k in range(w.conv_w.shape[0])]
        e.conv_baby_fold_ext = np.stack([
            o.encode_ext(sum(masks[k] * np.roll(kern[k], -s) for k in range(len(kern))), L) for s in [0] + baby])
    for k in range(w.conv_w.shape[0]):
        e.conv.append(o.encode(o.kernel_slots(w.conv_w[k], windows), level=L))
        if conv_shared:
            e.conv_baby_ext.append(o.conv_baby_diagonals_ext(o.kernel_slots(w.conv_w[k], windows), e.taps,
                                                             windows, L))
        e.masks.append(o.encode(cnn_mask_slots(o, k, windows, nb, pack_first), level=L - 1))
    if rect:
        e.fc1 = o.encode_matrix_rect(w.fc1_w.T, L - 3)
        e.fc2 = o.encode_matrix_rect(w.fc2_w.T, L - 5)
        e.fc1_ext = o.encode_matrix_rect_ext(w.fc1_w.T, L - 3)
        e.fc2_ext = o.encode_matrix_rect_ext(w.fc2_w.T, L - 5)
        e.rect = True
        return e
    e.fc1 = o.encode_matrix(w.fc1_w.T, L - 3)
    e.fc2 = o.encode_matrix(w.fc2_w.T, L - 5)
    e.fc1_ext = o.encode_matrix_ext(w.fc1_w.T, L - 3)
    e.fc2_ext = o.encode_matrix_ext(w.fc2_w.T, L - 5)
    return e


def _pack(o: OracleCKKS, chans, masks, merged: bool) -> Ct:
    """The masked channels summed: each product rescaled, then added; merged (A25): the products added
    first and rescaled once."""
    v = None
    for c, mk in zip(chans, masks):
        t = o.mul_plain(c, mk) if merged else o.rescale(o.mul_plain(c, mk))
        v = t if v is None else o.add(v, t)
    return o.rescale(v) if merged else v


def cnn_bias_slots(o: OracleCKKS, w: CNNWeights, enc: EncodedCNN) -> list[np.ndarray]:
    """The three bias vectors as slot values, laid out where the schedule's ciphertexts hold the
    layers' outputs: the conv bias on each kernel's block of windows (repeated with the packed
    vector's period when the channels are packed before the giant steps), the FC biases in the first
    m slots (repeated with period rect_width(m) in the rectangular form, whose outputs come out
    replicated)."""
    W = enc.windows
    K = len(w.conv_b)
    b0 = np.zeros(o.slots)
    if enc.pack_first:
        baby, _ = o.conv_bsgs_steps(enc.taps, W)
        period = (len(baby) + 1) * W
        for r in range(o.slots // period):
            for k in range(K):
                b0[r * period + k * W: r * period + (k + 1) * W] = w.conv_b[k]
    else:
        for k in range(K):
            b0[k * W: (k + 1) * W] = w.conv_b[k]
    out = [b0]
    for b in (w.fc1_b, w.fc2_b):
        v = np.zeros(o.slots)
        v[:len(b)] = b
        if enc.rect:
            v = np.resize(v[:o.rect_width(len(b))], o.slots)
        out.append(v)
    return out


def cnn_forward(o: OracleCKKS, ct: Ct, w: CNNWeights, enc: EncodedCNN, trace: dict | None = None,
                double_hoist: bool = False, merged: bool = False) -> Ct:
    """The encrypted CNN schedule (§5): conv (im2col, one multiplication per kernel) -> pack the
    four channel outputs with masks -> square -> FC1 (vector x plain matrix) -> square -> FC2.
    Six multiplicative levels; biases are added as plaintexts at the ciphertext's scale and level.
    double_hoist: the two vector x matrix products take the ModDown once after their rotation sums."""
    def fc(v, diags, diags_ext, n, m, replicate=True, period=None):
        if enc.rect:
            return (o.vecmat_rect(v, n, m, diags_ext=diags_ext, replicate=replicate, period=period, merged=merged)
                    if double_hoist else o.vecmat_rect(v, n, m, diags=diags, replicate=replicate, period=period))
        return (o.vecmat_dh(v, diags_ext, n, m, period=period, merged=merged) if double_hoist
                else o.vecmat(v, diags, n, m, period=period))

    W = enc.windows
    K = len(enc.conv)
    period = None
    bias, b1, b2 = cnn_bias_slots(o, w, enc)
    if enc.pack_first:
        # baby-step sums z_k, masks on the blocks k + B g, the pack, then one giant-step sum: block k of
        # the result gathers blocks k + B g of z_k, the full tap sum of kernel k (reading A23)
        baby, giant = o.conv_bsgs_steps(enc.taps, W)
        if enc.fold:
            # one sum over the folded diagonals is the packed vector at level L - 1; the limb the pack's
            # rescale would have dropped is dropped by a modulus switch, so every later level is unchanged
            v = (o.dh_sum(ct, baby, enc.conv_baby_fold_ext, merged=True) if merged
                 else o.rescale(o.dh_sum(ct, baby, enc.conv_baby_fold_ext)))
            v = o.mod_switch(v, v.level - 1)
        else:
            if enc.conv_shared:
                zs = [o.dh_sum(ct, baby, enc.conv_baby_ext[k], merged=True) if merged
                      else o.rescale(o.dh_sum(ct, baby, enc.conv_baby_ext[k])) for k in range(K)]
            else:
                zs = [o.rotsum_dh(o.rescale(o.mul_plain(ct, enc.conv[k])), baby) for k in range(K)]
            v = _pack(o, zs, enc.masks, merged)
        v = o.rotsum_dh(v, giant)
        period = (len(baby) + 1) * W  # blocks [K, B) are zero, the pattern repeats every B blocks
    else:
        if enc.conv_shared:
            chans = [o.conv2d_im2col_shared(ct, enc.conv_baby_ext[k], enc.taps, W) for k in range(K)]
        else:
            conv = o.conv2d_im2col_hoisted if enc.conv_hoist else o.conv2d_im2col_pt
            chans = [conv(ct, enc.conv[k], enc.taps, W) for k in range(K)]
        v = _pack(o, chans, enc.masks, merged)
    if trace is not None:
        trace["bias_scales"] = [v.scale]
    def bias_pt(i, values, v):
        if enc.biases is not None:
            return enc.biases[i]
        return o.encode(values, scale=v.scale, level=v.level)

    v = o.add_plain(v, bias_pt(0, bias, v))
    v = o.mul(v, v, merged=merged)
    n1, m1 = w.fc1_w.shape[1], w.fc1_w.shape[0]
    v = fc(v, enc.fc1, enc.fc1_ext, n1, m1, period=period)
    if trace is not None:
        trace["bias_scales"].append(v.scale)
    v = o.add_plain(v, bias_pt(1, b1, v))
    v = o.mul(v, v, merged=merged)
    n2, m2 = w.fc2_w.shape[1], w.fc2_w.shape[0]
    v = fc(v, enc.fc2, enc.fc2_ext, n2, m2, replicate=not enc.rect)
    if trace is not None:
        trace["bias_scales"].append(v.scale)
    v = o.add_plain(v, bias_pt(2, b2, v))
    return v


def cnn_plain(img: np.ndarray, w: CNNWeights, stride=3) -> np.ndarray:
    """The same network evaluated directly in FP64 (the accuracy reference)."""
    kh = kw = int(round(math.sqrt(w.conv_w.shape[1])))
    H, Wd = img.shape
    oh = (H - kh) // stride + 1
    ow = (Wd - kw) // stride + 1
    conv = np.zeros((w.conv_w.shape[0], oh, ow))
    for k in range(w.conv_w.shape[0]):
        ker = w.conv_w[k].reshape(kh, kw)
        for r in range(oh):
            for c in range(ow):
                conv[k, r, c] = np.sum(img[stride * r: stride * r + kh, stride * c: stride * c + kw] * ker) + w.conv_b[k]
    x = conv.reshape(-1) ** 2
    x = w.fc1_w @ x + w.fc1_b
    x = x ** 2
    return w.fc2_w @ x + w.fc2_b
