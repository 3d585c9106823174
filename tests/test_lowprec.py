"""Byte-exact check of the library's low-precision inner matrix (csrc/lowprec.h)
against the oracle's, which is written independently (the oracle rounds with
frexp/ldexp and nearbyint; the library rounds BF16 from the double's bits and
FP32 with the IEEE conversion)."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1107_0538_gb300 import problems

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1107_0538_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("lowprec")
    exe = d / "lowprec_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe),
                    os.path.join(ROOT, "tests", "lowprec_check.cpp")], check=True)
    return exe, d


def library_inner(driver, A, fmt_code):
    exe, d = driver
    path, out = d / "A.bin", d / "out.bin"
    with open(path, "wb") as f:
        np.array([A.n, len(A.colidx)], np.int32).tofile(f)
        np.asarray(A.rowptr, np.int32).tofile(f)
        np.asarray(A.colidx, np.int32).tofile(f)
        np.asarray(A.vals, np.float64).tofile(f)
    subprocess.run([str(exe), str(path), str(fmt_code), str(out)], check=True)
    return np.fromfile(out, dtype=np.float64)


def extreme_matrix():
    """Values over the whole BF16 range: subnormals, ties, overflow, signs."""
    rng = np.random.default_rng(3)
    n = 300
    rowptr, cols, vals = [0], [], []
    specials = [1e-41, -3e-40, 2.0 ** -133 * 1.5, 2.0 ** -126 * (1 + 2 ** -8), 3.4e38, -3.39e38,
                1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 0.0, -0.0]
    for i in range(n):
        c = sorted(set(rng.choice(n, size=12, replace=False).tolist()) | {i})
        for j in c:
            cols.append(j)
            if j == i:
                vals.append(50.0)
            elif rng.random() < 0.1:
                vals.append(specials[int(rng.integers(len(specials)))])
            else:
                vals.append(-abs(rng.standard_normal()) * 10.0 ** rng.integers(-30, 30))
        rowptr.append(len(cols))
    return problems.CSR(n, np.array(rowptr, np.int32), np.array(cols, np.int32), np.array(vals))


@pytest.mark.parametrize("fmt_code,fmt", [(1, oracle.FP32_FORMAT), (2, oracle.BF16_FORMAT)])
@pytest.mark.parametrize("case", ["blobs6", "uniform20", "extreme"])
def test_inner_matrix_matches_oracle_bitwise(driver, fmt_code, fmt, case):
    A = {"blobs6": lambda: problems.cube_blobs(6).A, "uniform20": lambda: problems.cube_uniform(20).A,
         "extreme": extreme_matrix}[case]()
    got = library_inner(driver, A, fmt_code)
    want = oracle.lowprec_values(A, fmt)
    with np.errstate(invalid="ignore"):
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), \
            np.flatnonzero(got.view(np.uint64) != want.view(np.uint64))[:10]
