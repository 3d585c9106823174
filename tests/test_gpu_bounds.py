"""The bounds-check build (libgbcg_check.so, -DGBCG_BOUNDS_CHECK) on the
ragged SpMV cases and a small solve through every kernel family.

Its kernels test every column index they gather through and every staged row
range they walk, count a bad one instead of trapping, and report the count
through cg_bounds_faults.  On well-formed inputs the count must be 0 and the
results must meet the same bars as the normal build's (SpMV within its
summation-order bound, solves at the tolerance).  The check build runs in a
child process (GBCG_LIBRARY=check selects it), so this process keeps the
normal library.
"""
import json
import os
import subprocess
import sys

import pytest

from paper_1107_0538_gb300 import build as nvbuild
from paper_1107_0538_gb300 import gbcg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_check_build_counts_no_fault_on_wellformed_inputs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvbuild.build()
    assert os.path.exists(nvbuild.OUT_CHECK)
    env = dict(os.environ, GBCG_LIBRARY="check")
    res = subprocess.run([sys.executable, os.path.join(HERE, "bounds_worker.py")], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["faults"] == 0, out
    assert out["spmv_err_over_bound"] <= 1.0, out
    for s in out["solves"]:
        assert s["status"] == gbcg.CG_OK and s["relres_true"] <= 1.05e-8, s
    assert {s["plan"] for s in out["solves"]} == {0, 1, 2}, out["solves"]
    assert out["batch"] == [gbcg.CG_OK, gbcg.CG_OK] and out["learned_status"] == gbcg.CG_OK, out


def test_normal_build_reports_no_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert gbcg.cg_bounds_faults() == -1
