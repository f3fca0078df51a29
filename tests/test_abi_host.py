"""The C-ABI library without a GPU: it builds, loads, exports every symbol include/tcks.h declares, and
its host-only logic (prime chain, argument checks, client-side im2col) agrees with the oracle."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_2104_03152_gb300 as tk
from paper_2104_03152_gb300 import build as tkbuild
from paper_2104_03152_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tcks.h")


@pytest.fixture(scope="module")
def built():
    return tkbuild.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tcks_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 50
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(tcks_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = tk.lib()
    for n in names:
        assert getattr(L, n) is not None


def test_binding_covers_header(built):
    names = declared_functions()
    assert set(names) <= set(tk._SIGS), sorted(set(names) - set(tk._SIGS))


def test_status_strings(built):
    L = tk.lib()
    assert L.tcks_status_string(0) == b"OK"
    assert L.tcks_status_string(-3) == b"NO_GALOIS_KEY"
    assert L.tcks_status_string(-11) == b"VALUE_OVERFLOW"


@pytest.mark.parametrize("log_n,bits", [(12, [36, 36, 36, 37]), (13, [31, 26, 26, 26, 26, 26, 26, 31]),
                                        (14, [60, 40, 40, 60]), (16, [59, 58, 57, 56, 60]), (13, [50, 50, 50, 50, 51])])
def test_prime_chain_matches_oracle(built, log_n, bits):
    p = tk.Params(log_n, bits, 2.0 ** 30)
    assert p.primes == oracle.gen_primes(log_n, bits)


def test_bad_params_rejected(built):
    with pytest.raises(tk.TcksError) as e:
        tk.Params(13, [31], 2.0 ** 26)  # no special prime
    assert e.value.name == "BAD_PARAMS"
    with pytest.raises(tk.TcksError):
        tk.Params(20, [40, 40], 2.0 ** 26)  # N too large
    with pytest.raises(tk.TcksError):
        tk.Params(13, [62, 40], 2.0 ** 26)  # prime too large


def test_explicit_prime_chain(built):
    """One chain of primes == 1 (mod 2^17) serves every N <= 2^16; the checks reject what O1 excludes."""
    chain = oracle.gen_primes(16, [59 - (i % 10) for i in range(32)] + [60])
    for log_n in (13, 14, 15, 16):
        assert tk.Params(log_n, primes=chain, scale=2.0 ** 50).primes == chain
    q = chain[0]
    bad = {
        "composite": [(2 ** 14 + 1) * (2 ** 15 + 1), chain[-1]],  # == 1 (mod 2^14), not prime
        "not 1 mod 2N": [next(p for p in range(2 ** 40 + 1, 2 ** 40 + 10 ** 6, 2) if oracle.is_prime(p)
                              and p % 2 ** 14 != 1), chain[-1]],
        "repeated": [q, q],
        "too wide": [2 ** 61 + 2 ** 17 * 3 + 1, q],
        "one prime": [q],
    }
    for why, primes in bad.items():
        with pytest.raises(tk.TcksError) as e:
            tk.Params(13, primes=primes, scale=2.0 ** 40)
        assert e.value.name == "BAD_PARAMS", why


def test_im2col_matches_oracle(built):
    img = inputs.mnist_like_image(3)
    v, w = tk.im2col_encode(img, 7, 7, 3, 4096)
    ref, wref = oracle.OracleCKKS.im2col(img, 7, 7, 3, 4096)
    assert w == wref == 64
    assert np.array_equal(v, ref)
    with pytest.raises(tk.TcksError):
        tk.im2col_encode(img, 7, 7, 3, 1000)


@pytest.mark.slow
def test_debug_build_compiles_and_reports_itself(built):
    """The debug build (TCKS_DEBUG_CHECKS: descriptor-table asserts, device range checks) compiles,
    exports the same symbols, and reports itself; the default build does not."""
    dbg = tkbuild.build(debug=True)
    assert dbg != built
    out = subprocess.run(["nm", "-D", "--defined-only", dbg], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(tcks_\w+)", out))
    assert not [n for n in declared_functions() if n not in exported]
    code = "import paper_2104_03152_gb300 as tk; print(int(tk.debug_checks()))"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                       env=dict(os.environ, TCKS_DEBUG_CHECKS="1"), check=True)
    assert r.stdout.strip() == "1"
    assert tk.debug_checks() is False
