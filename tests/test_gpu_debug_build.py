"""The debug build (TCKS_DEBUG_CHECKS): its device range checks skip and report descriptor entries
outside their declared range, its host checks refuse a job list whose buffers overlap before any
launch, and a well-formed mixed batch passes every check with the single calls' results. The checks
run in a child process (tests/debug_build_checks.py) that builds and loads the debug library; this
process keeps the default build, where the self-test entry is UNSUPPORTED."""
import json
import os
import subprocess
import sys

import pytest

import paper_2104_03152_gb300 as tk

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
DBG_LIMB_RANGE = 2


@pytest.fixture(scope="module")
def results():
    env = dict(os.environ, TCKS_DEBUG_CHECKS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_checks.py")], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_reports_itself(results):
    assert results["debug_checks"] is True
    assert tk.debug_checks() is False


@pytest.mark.parametrize("case", ["selftest_n13", "selftest_n14"])
def test_device_range_checks_skip_and_report(results, case):
    r = results[case]
    assert r["word"] == DBG_LIMB_RANGE
    assert r["transformed_equal"] and r["skipped_unchanged"]


def test_overlapping_jobs_refused_before_launch(results):
    assert results["overlap"] == {"refused": "DEBUG_CHECK", "launches": 0}


def test_clean_batch_passes_checks(results):
    assert results["clean"] and all(results["clean"].values()), results["clean"]


def test_selftest_unsupported_in_default_build():
    g = tk.Context(tk.Params(13, [50, 40, 60], 2.0 ** 30))
    d = torch.zeros((1, 2, g.N), dtype=torch.int64, device="cuda")
    torch.cuda.current_stream().synchronize()
    before = tk.launch_count()
    with pytest.raises(tk.TcksError) as e:
        tk.debug_selftest(g, d.data_ptr(), 1, 2, 1)
    assert e.value.name == "UNSUPPORTED" and tk.launch_count() == before
