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
    """C2 chain: the encrypted input at level 7 and the output at level 1 (§4's 427 KB figure, with
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
