"""The bit-packed wire format on the GPU: byte-identical to the oracle's serializer, round trips, the
range and header checks, and the size of one encrypted CNN inference's traffic (§5)."""
import numpy as np
import pytest

import oracle
from oracle import wire
import paper_2104_03152_gb300 as tk
from gpu_common import SEED, Pair
from paper_2104_03152_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("log_n,bits", [(5, [30, 30, 31]), (12, [36, 36, 36, 37]), (13, [31, 26, 26, 26, 26, 26, 26, 31]),
                                        (14, [60, 40, 40, 60])])
def test_serialize_matches_oracle_and_roundtrips(log_n, bits):
    ctx = tk.Context(tk.Params(log_n, bits, 2.0 ** 26), seed=SEED)
    for level in (ctx.L, 1):
        data = np.stack([inputs.random_limbs(ctx.primes[:level], ctx.N, 40 + level + b, polys=1)[0] for b in range(2)])
        ct = ctx.ct_import(data, 2.0 ** 26)
        got = ct.serialize()
        assert got == wire.serialize(data, level, 2.0 ** 26, log_n, ctx.primes)
        back = ctx.ct_deserialize(got)
        assert np.array_equal(back.export(), data) and back.info() == (level, 2.0 ** 26)


def test_deserialize_rejects_bad_input():
    ctx = tk.Context(tk.Params(12, [36, 36, 36, 37], 2.0 ** 30), seed=SEED)
    data = np.stack([inputs.random_limbs(ctx.primes[:3], ctx.N, 7 + b, polys=1)[0] for b in range(2)])
    buf = ctx.ct_import(data, 1.0).serialize()
    bad = bytearray(buf)
    bad[16:24] = b"\xff" * 8  # residues >= q_0
    for blob in (buf[:-1], bytes(bad), b"XXXX" + buf[4:]):
        with pytest.raises(tk.TcksError) as e:
            ctx.ct_deserialize(blob)
        assert e.value.name == "INVALID_ARG"


def test_cnn_inference_traffic():
    """Encrypted input at level 7 plus encrypted output at level 1 for the C2 chain: 446,496 bytes
    (436 KiB; the paper's 427 KB is for its 206-bit chain)."""
    ctx = tk.Context(tk.Params(13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26), seed=SEED)
    x = ctx.encrypt_values(inputs.uniform_slots(8, 1), 3)
    y = ctx.ct_import(x.export()[:, :1], x.info()[1])
    assert len(x.serialize()) + len(y.serialize()) == 16 + 382976 + 16 + 63488


def test_batch_import_export_roundtrip():
    ctx = tk.Context(tk.Params(12, [36, 36, 36, 37], 2.0 ** 30), seed=SEED)
    data = np.stack([np.stack([inputs.random_limbs(ctx.primes[:3], ctx.N, 60 + 2 * i + b, polys=1)[0]
                               for b in range(2)]) for i in range(5)])
    cts = ctx.ct_import_batch(data, 2.0 ** 30)
    for i, c in enumerate(cts):
        assert np.array_equal(c.export(), data[i]) and c.info() == (3, 2.0 ** 30)
    out = np.zeros_like(data)
    handles = (tk._vp * len(cts))(*[c.h.value for c in cts])
    tk.check(tk.lib().tcks_ct_export_batch(handles, len(cts), tk._p(out), out.size))
    assert np.array_equal(out, data)


@pytest.mark.parametrize("name", ["C1", "C2"])
def test_secret_key_encryption_and_seeded_wire(name):
    """tcks_encrypt_symmetric equals the oracle's secret-key encryption bit for bit; its seeded wire form
    equals the oracle's byte for byte, deserializes to the same ciphertext (c1 regenerated on the
    device), and a ciphertext that has been computed on is refused."""
    log_n, bits, scale = {"C1": (12, [36, 36, 36, 37], 2.0 ** 30), "C2": (13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26)}[name]
    p = Pair(log_n, bits, scale)
    o, g = p.o, p.g
    pt = o.encode(inputs.uniform_slots(o.slots, 3))
    ref = o.encrypt_symmetric(pt, 4242, 17)
    ct = g.encrypt_symmetric(p.import_pt(pt), 4242, 17)
    assert np.array_equal(ct.export(), ref.data)
    buf = ct.serialize_seeded(4242)
    assert buf == wire.serialize_seeded(ref.data[0], ref.level, ref.scale, o.log_n, o.primes, 4242)
    assert len(buf) == wire.size_seeded(o.N, o.primes, ref.level) == (len(ct.serialize()) - 16) // 2 + 24
    back = g.ct_deserialize(buf)
    assert np.array_equal(back.export(), ref.data)
    with pytest.raises(tk.TcksError) as e:
        ct.serialize_seeded(4243)  # not the seed of its c1
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(tk.TcksError):
        ct.add(ct).serialize_seeded(4242)
