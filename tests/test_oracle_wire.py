"""Pins of the oracle's wire format: a hand-worked packing, the closed-form size of the paper's CNN
traffic, and round trips."""
import numpy as np
import pytest

import oracle
from oracle import wire
from paper_2104_03152_gb300 import inputs


def test_pack_worked_example():
    # residues 5, 3, 7, 1 at w = 3, each least significant bit first: 1,0,1 | 1,1,0 | 1,1,1 | 1,0,0;
    # byte 0 = bits 0..7 = 1,0,1,1,1,0,1,1 = 0xDD, byte 1 = bits 8..11 = 1,1,0,0 = 0x03
    assert wire.pack_limb(np.array([5, 3, 7, 1]), 3) == bytes([0xDD, 0x03])
    assert list(wire.unpack_limb(bytes([0xDD, 0x03]), 4, 3)) == [5, 3, 7, 1]


def test_cnn_traffic_closed_form():
    """C2 chain: the encrypted input at level 7 and the output at level 1 (§5's 427 KB figure, with
    the configs' 218-bit chain instead of the paper's 206-bit one)."""
    primes = oracle.gen_primes(13, [31, 26, 26, 26, 26, 26, 26, 31])
    n = 8192
    assert wire.size(n, primes, 7) == 16 + 2 * n * (31 + 6 * 26) // 8 == 16 + 382976
    assert wire.size(n, primes, 1) == 16 + 2 * n * 31 // 8 == 16 + 63488


@pytest.mark.parametrize("log_n,bits", [(5, [30, 30, 31]), (12, [36, 36, 36, 37]), (13, [31, 26, 26, 31])])
def test_roundtrip_and_rejects(log_n, bits):
    primes = oracle.gen_primes(log_n, bits)
    level = len(primes) - 1
    data = np.stack([inputs.random_limbs(primes[:level], 1 << log_n, 9 + b, polys=1)[0] for b in range(2)])
    buf = wire.serialize(data, level, 2.0 ** 30, log_n, primes)
    assert len(buf) == wire.size(1 << log_n, primes, level)
    back, lv, sc, ln = wire.deserialize(buf, primes)
    assert np.array_equal(back, data) and lv == level and sc == 2.0 ** 30 and ln == log_n
    with pytest.raises(ValueError):
        wire.deserialize(buf[:-1], primes)
    bad = bytearray(buf)
    bad[16:16 + 8] = b"\xff" * 8  # the first residues all ones: >= q_0
    with pytest.raises(ValueError):
        wire.deserialize(bytes(bad), primes)


def test_secret_key_encryption_equation():
    """(-a s + e + m, a): c1 is the uniform polynomial of the public seed, c0 + c1 s - m has the small
    CBD coefficients of e (|e_i| <= 21) as a polynomial (checked exactly by CRT), and it decrypts."""
    o = oracle.OracleCKKS(12, [36, 36, 36, 37], 2.0 ** 30).keygen()
    z = inputs.uniform_slots(o.slots, 5)
    pt = o.encode(z)
    ct = o.encrypt_symmetric(pt, 1234, 98765)
    assert np.array_equal(ct.data[1], o.sample_sym_a(pt.level, 1234))
    lv = pt.level
    diff = np.zeros((lv, o.N), dtype=np.uint64)
    for l in range(lv):
        q = o.primes[l]
        cs = (ct.data[1][l].astype(object) * o.s[l].astype(object) + ct.data[0][l].astype(object)
              - pt.data[l].astype(object)) % q
        diff[l] = np.array(cs, dtype=np.uint64)
    coeffs = o.crt_compose(o.intt_limbs(diff, lv), lv)
    Q = 1
    for q in o.primes[:lv]:
        Q *= q
    bal = [c - Q if c > Q // 2 else c for c in coeffs]
    assert max(abs(b) for b in bal) <= 21 and any(b != 0 for b in bal)
    assert np.max(np.abs(o.decrypt_values(ct, o.slots) - z)) < 1e-6
    other = o.encrypt_symmetric(pt, 1234, 98766)  # another private seed: same a, another e
    assert np.array_equal(other.data[1], ct.data[1]) and not np.array_equal(other.data[0], ct.data[0])


def test_seeded_wire_roundtrip_and_cnn_traffic():
    primes = oracle.gen_primes(13, [31, 26, 26, 26, 26, 26, 26, 31])
    n = 8192
    # the encrypted CNN input travels as c0 and the seed: 24 + 191,488 bytes instead of 16 + 382,976
    assert wire.size_seeded(n, primes, 7) == 16 + 8 + n * (31 + 6 * 26) // 8 == 191512
    o = oracle.OracleCKKS(12, [36, 36, 36, 37], 2.0 ** 30).keygen()
    ct = o.encrypt_symmetric(o.encode(inputs.uniform_slots(o.slots, 6)), 777, 888)
    buf = wire.serialize_seeded(ct.data[0], ct.level, ct.scale, o.log_n, o.primes, 777)
    assert len(buf) == wire.size_seeded(o.N, o.primes, ct.level)
    c0, seed, lv, sc, ln = wire.deserialize_seeded(buf, o.primes)
    assert seed == 777 and lv == ct.level and sc == ct.scale and ln == o.log_n
    assert np.array_equal(c0, ct.data[0]) and np.array_equal(o.sample_sym_a(lv, seed), ct.data[1])
    with pytest.raises(ValueError):
        wire.deserialize(buf, o.primes)  # kind 1 is not a full ciphertext
    with pytest.raises(ValueError):
        wire.deserialize_seeded(buf[:-1], o.primes)
