"""CPU checks of the host tile planner that cg_create runs (csrc/plan.h).

The kernels derive every TMA source range, copy size, shared-memory offset
and window gather from this plan; plan_check.cpp runs the planner on a CSR
pattern and check_plan verifies each of those indices against the matrix,
so that no plan the library builds can send a copy or a read out of bounds.
"""
import json
import os
import subprocess

import numpy as np
import pytest

from paper_1107_0538_gb300 import problems

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1107_0538_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    d = tmp_path_factory.mktemp("plan")
    exe = d / "plan_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe),
                    os.path.join(ROOT, "tests", "plan_check.cpp")], check=True)
    return exe, d


def run_plan(checker, rowptr, colidx, n):
    exe, d = checker
    path = d / f"csr_{n}_{len(colidx)}.bin"
    with open(path, "wb") as f:
        np.array([n, len(colidx)], np.int32).tofile(f)
        np.asarray(rowptr, np.int32).tofile(f)
        np.asarray(colidx, np.int32).tofile(f)
    res = subprocess.run([str(exe), str(path)], capture_output=True, text=True)
    out = json.loads(res.stdout)
    assert res.returncode == 0, out["error"]
    return out


@pytest.mark.parametrize("e", [1, 2, 7, 20, 50, 100])
def test_stencil_plans_are_sound_and_windowed(checker, e):
    A = problems.cube_uniform(e).A if e <= 20 else problems.q1_matrix(problems.nu_uniform(e, e, e), 1.0 / e)[0]
    out = run_plan(checker, A.rowptr, A.colidx, A.n)
    assert out["windowed"] == out["tiles"] and out["long"] == 0
    assert out["max_segments"] <= 18


@pytest.mark.parametrize("ex,ey,ez", [(3, 40, 2), (60, 1, 1), (1, 1, 70), (33, 9, 4)])
def test_uneven_boxes(checker, ex, ey, ez):
    A, _ = problems.q1_matrix(problems.nu_uniform(ex, ey, ez), 0.1)
    out = run_plan(checker, A.rowptr, A.colidx, A.n)
    assert out["windowed"] == out["tiles"]


def random_pattern(n, seed, long_rows=(), long_len=0, empty=(), dup=False):
    rng = np.random.default_rng(seed)
    rowptr, cols = [0], []
    for i in range(n):
        m = 0 if i in empty else (long_len if i in long_rows else int(rng.integers(1, 40)))
        c = np.sort(rng.choice(n, size=min(m, n), replace=False)) if m else np.zeros(0, int)
        if dup and len(c) > 2:
            c = np.concatenate([c, c[:2]])
        cols.extend(c.tolist())
        rowptr.append(len(cols))
    return rowptr, cols


@pytest.mark.parametrize("n,seed,extra", [
    (1, 0, {}), (2, 1, {}), (129, 2, {}), (3001, 3, {"long_rows": {5, 3000}, "long_len": 2000}),
    (2000, 4, {"empty": set(range(0, 2000, 3))}), (999, 5, {"dup": True}),
    (5000, 6, {"long_rows": {10, 11}, "long_len": 896}), (5000, 7, {"long_rows": {0}, "long_len": 897}),
])
def test_random_patterns(checker, n, seed, extra):
    rowptr, cols = random_pattern(n, seed, **extra)
    run_plan(checker, rowptr, cols, n)


def test_banded_windows_with_odd_tail(checker):
    # columns reaching n - 1 with n odd exercise the tail column of a window
    n = 1001
    rowptr, cols = [0], []
    for i in range(n):
        c = sorted({max(0, i - 1), i, min(n - 1, i + 1), n - 1})
        cols.extend(c)
        rowptr.append(len(cols))
    out = run_plan(checker, rowptr, cols, n)
    assert out["windowed"] == out["tiles"]


def test_empty_matrix(checker):
    run_plan(checker, [0], [], 0)
    run_plan(checker, [0] * 51, [], 50)


def test_sell_column_widths(checker):
    # 16-bit column offsets when every |col - row| < 2^15, else 32-bit columns
    e = 20
    A = problems.q1_matrix(problems.nu_uniform(e, e, e), 1.0 / e)[0]
    out = run_plan(checker, A.rowptr, A.colidx, A.n)
    assert out["sell_rel16"] == 1
    assert out["sell_entries"] >= A.nnz and out["sell_entries"] % 32 == 0
    rowptr, cols = random_pattern(70000, 8)   # random columns reach past 2^15
    out = run_plan(checker, rowptr, cols, 70000)
    assert out["sell_rel16"] == 0


def test_slice_split_balances_cost(checker):
    # contiguous slice ranges, at most 31 slices per CTA, largest CTA cost
    # between the lower bound (mean, largest slice) and the bound plus one slice
    e = 20
    A = problems.q1_matrix(problems.nu_uniform(e, e, e), 1.0 / e)[0]
    out = run_plan(checker, A.rowptr, A.colidx, A.n)
    assert out["error"] == ""
    assert out["slice_bound"] <= out["slice_cost"] <= out["slice_bound"] + 27 + 8
    # 4713 slices: more than 152 x 31, no split
    n = 152 * 31 * 32 + 1
    rowptr = np.arange(n + 1, dtype=np.int32)
    out = run_plan(checker, rowptr, np.arange(n, dtype=np.int32), n)
    assert out["error"] == "" and out["slice_cost"] == -1
    n = 152 * 31 * 32
    rowptr = np.arange(n + 1, dtype=np.int32)
    out = run_plan(checker, rowptr, np.arange(n, dtype=np.int32), n)
    assert out["error"] == "" and out["slice_cost"] == 31 * (1 + 8)
