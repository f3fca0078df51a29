"""Wire format of a ciphertext (TEST INFRASTRUCTURE ONLY: the oracle of the library's serializer).

The paper reports the communication of one encrypted inference (encrypted input plus encrypted output,
§5). A ciphertext travels as residues packed with exactly bit_length(q_i) bits each:

  header (16 bytes, little-endian): b"TCKS", version 1 (u8), kind 0 = ciphertext (u8), log2 N (u8),
  level (u8), scale (f64);
  payload: for component b = 0, 1 and limb i = 0 .. level-1, the N residues of that limb (NTT form),
  residue k in bits [k w_i, (k + 1) w_i) of the limb's segment, w_i = bit_length(q_i), bits numbered
  from the least significant bit of the segment's first byte; each segment is ceil(N w_i / 8) bytes.
  Kind 1 (a secret-key ciphertext, (-a s + e + m, a) with a the uniform polynomial of a public seed):
  the header, the seed (u64), then component 0 only, packed the same way.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"TCKS"
HEADER = 16


def limb_bytes(n: int, q: int) -> int:
    return (n * int(q).bit_length() + 7) // 8


def size(n: int, primes, level: int) -> int:
    return HEADER + 2 * sum(limb_bytes(n, q) for q in primes[:level])


def pack_limb(x: np.ndarray, w: int) -> bytes:
    """Residues -> bits (least significant first) -> bytes (least significant bit first)."""
    x = np.asarray(x, dtype=np.uint64)
    bits = ((x[:, None] >> np.arange(w, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)
    return np.packbits(bits.reshape(-1), bitorder="little").tobytes()


def unpack_limb(buf: bytes, n: int, w: int) -> np.ndarray:
    bits = np.unpackbits(np.frombuffer(buf, dtype=np.uint8), bitorder="little")[: n * w].reshape(n, w)
    return (bits.astype(np.uint64) << np.arange(w, dtype=np.uint64)[None, :]).sum(axis=1, dtype=np.uint64)


def serialize(data: np.ndarray, level: int, scale: float, log_n: int, primes) -> bytes:
    """data [2][level][N] canonical residues."""
    n = 1 << log_n
    out = [MAGIC, struct.pack("<BBBBd", 1, 0, log_n, level, scale)]
    for b in range(2):
        for i in range(level):
            out.append(pack_limb(data[b][i], int(primes[i]).bit_length()))
    return b"".join(out)


def size_seeded(n: int, primes, level: int) -> int:
    return HEADER + 8 + sum(limb_bytes(n, q) for q in primes[:level])


def serialize_seeded(c0: np.ndarray, level: int, scale: float, log_n: int, primes, seed_a: int) -> bytes:
    """Kind 1, a secret-key ciphertext whose c1 is the uniform polynomial of seed_a: header, seed_a
    (u64, little-endian), then the level limbs of c0 packed as in kind 0. Half the bytes."""
    out = [MAGIC, struct.pack("<BBBBd", 1, 1, log_n, level, scale), struct.pack("<Q", seed_a)]
    for i in range(level):
        out.append(pack_limb(c0[i], int(primes[i]).bit_length()))
    return b"".join(out)


def deserialize_seeded(buf: bytes, primes):
    """-> (c0 [level][N], seed_a, level, scale, log_n) of a kind-1 buffer; ValueError otherwise."""
    if len(buf) < HEADER + 8 or buf[:4] != MAGIC:
        raise ValueError("not a serialized ciphertext")
    version, kind, log_n, level, scale = struct.unpack("<BBBBd", buf[4:16])
    if version != 1 or kind != 1 or level < 1 or level > len(primes) - 1:
        raise ValueError("unsupported header")
    n = 1 << log_n
    if len(buf) != size_seeded(n, primes, level):
        raise ValueError("size mismatch")
    (seed_a,) = struct.unpack("<Q", buf[16:24])
    c0 = np.zeros((level, n), dtype=np.uint64)
    off = HEADER + 8
    for i in range(level):
        lb = limb_bytes(n, primes[i])
        c0[i] = unpack_limb(buf[off:off + lb], n, int(primes[i]).bit_length())
        if np.any(c0[i] >= np.uint64(primes[i])):
            raise ValueError("residue out of range")
        off += lb
    return c0, seed_a, level, scale, log_n


def deserialize(buf: bytes, primes):
    """-> (data [2][level][N], level, scale, log_n); ValueError on a bad header, size or residue."""
    if len(buf) < HEADER or buf[:4] != MAGIC:
        raise ValueError("not a serialized ciphertext")
    version, kind, log_n, level, scale = struct.unpack("<BBBBd", buf[4:16])
    if version != 1 or kind != 0 or level < 1 or level > len(primes) - 1:
        raise ValueError("unsupported header")
    n = 1 << log_n
    if len(buf) != size(n, primes, level):
        raise ValueError("size mismatch")
    data = np.zeros((2, level, n), dtype=np.uint64)
    off = HEADER
    for b in range(2):
        for i in range(level):
            lb = limb_bytes(n, primes[i])
            data[b][i] = unpack_limb(buf[off:off + lb], n, int(primes[i]).bit_length())
            if np.any(data[b][i] >= np.uint64(primes[i])):
                raise ValueError("residue out of range")
            off += lb
    return data, level, scale, log_n
