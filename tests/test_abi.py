"""CPU checks of the C ABI boundary: the library loads, exports every function
include/gbcg.h declares, the ctypes structures match the C layout, and the
host-side argument validation answers without touching a GPU."""
import ctypes
import json
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1107_0538_gb300 import build as nvbuild
from paper_1107_0538_gb300 import gbcg, problems

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbcg.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    return gbcg.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(cg_\w+)\s*\(", text, flags=re.M))


def test_header_and_binding_agree():
    assert declared_functions() == set(gbcg.EXPORTS)


def test_every_declared_symbol_is_exported():
    out = subprocess.run(["nm", "-D", "--defined-only", gbcg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    names = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - names
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(gbcg.lib(), f)


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gbcg.h"
#define F(T, m) printf("\\"%s.%s\\": [%zu, %zu],", #T, #m, offsetof(T, m), sizeof(((T*)0)->m));
int main(void) {
  printf("{");
  F(cg_csr, n) F(cg_csr, nnz) F(cg_csr, rowptr) F(cg_csr, colidx) F(cg_csr, vals) F(cg_csr, mem)
  F(cg_opts, precond) F(cg_opts, true_residual) F(cg_opts, wait_limit_s) F(cg_opts, grid_ctas)
  F(cg_opts, debug_phantom_arrivals) F(cg_opts, vectors_in_memory)
  F(cg_opts, inner_values) F(cg_opts, inner_tol) F(cg_opts, max_outer) F(cg_opts, max_inner)
  F(cg_info, iters) F(cg_info, status) F(cg_info, relres) F(cg_info, relres_true)
  F(cg_info, kernel_ms) F(cg_info, launches) F(cg_info, outer) F(cg_info, reverted_at) F(cg_info, reserved)
  F(cg_plan, n) F(cg_plan, nnz) F(cg_plan, ctas) F(cg_plan, threads) F(cg_plan, tiles)
  F(cg_plan, tile_nnz) F(cg_plan, stages) F(cg_plan, smem_bytes) F(cg_plan, lanes_per_row)
  F(cg_plan, l2_evict_first) F(cg_plan, reg_rows) F(cg_plan, window_tiles) F(cg_plan, device_bytes)
  F(cg_plan, slice_solve) F(cg_plan, inner_solve)
  F(cg_batch_result, iters) F(cg_batch_result, outer) F(cg_batch_result, status) F(cg_batch_result, reserved)
  F(cg_batch_result, relres)
  F(cg_batch_tuning, inner_tol) F(cg_batch_tuning, gather_tiles) F(cg_batch_tuning, trials) F(cg_batch_tuning, best_ms)
  F(cg_batch_tuning, lanes_per_row) F(cg_batch_tuning, static_split)
  F(cg_learn_set, ninst) F(cg_learn_set, inst) F(cg_learn_set, npairs) F(cg_learn_set, pair_inst)
  F(cg_learn_set, r) F(cg_learn_set, e)
  printf("\\"sizes\\": [%zu, %zu, %zu, %zu]}", sizeof(cg_csr), sizeof(cg_opts), sizeof(cg_info), sizeof(cg_plan));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    c = json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)
    for T in (gbcg.cg_csr, gbcg.cg_opts, gbcg.cg_info, gbcg.cg_plan, gbcg.cg_batch_result, gbcg.cg_batch_tuning,
              gbcg.cg_learn_set):
        for name, ctype in T._fields_:
            off, size = c[f"{T.__name__}.{name}"]
            assert getattr(T, name).offset == off, (T.__name__, name)
            assert ctypes.sizeof(ctype) == size, (T.__name__, name)
    assert c["sizes"] == [ctypes.sizeof(T) for T in (gbcg.cg_csr, gbcg.cg_opts, gbcg.cg_info, gbcg.cg_plan)]


def test_defaults_and_strerror():
    o = gbcg.cg_opts_default()
    assert o.precond == gbcg.CG_PRECOND_NONE and o.true_residual == 1
    assert o.wait_limit_s == 5.0 and o.grid_ctas == 0 and o.debug_phantom_arrivals == 0
    for code in range(8):
        assert gbcg.cg_strerror(code) != "unknown status"
    assert gbcg.cg_strerror(99) == "unknown status"
    assert gbcg.cg_version() >= 10000


def _csr(n, rowptr, colidx, vals, nnz=None):
    rowptr = np.asarray(rowptr, np.int32)
    colidx = np.asarray(colidx, np.int32)
    vals = np.asarray(vals, np.float64)
    c = gbcg.cg_csr(n, len(colidx) if nnz is None else nnz, rowptr.ctypes.data, colidx.ctypes.data,
                    vals.ctypes.data, gbcg.CG_MEM_HOST)
    return c, (rowptr, colidx, vals)


@pytest.mark.parametrize("case", ["rowptr0", "decreasing", "nnz_mismatch", "col_high", "col_negative",
                                  "negative_n", "bad_mem", "null_rowptr"])
def test_malformed_csr_rejected_without_gpu(case):
    rowptr, colidx, vals = [0, 2, 3], [0, 1, 1], [2.0, -1.0, 2.0]
    n, nnz, mem = 2, None, gbcg.CG_MEM_HOST
    if case == "rowptr0":
        rowptr = [1, 2, 3]
    elif case == "decreasing":
        rowptr, colidx, vals = [0, 3, 2], [0, 1, 1], [1.0, 1.0, 1.0]
    elif case == "nnz_mismatch":
        nnz = 5
    elif case == "col_high":
        colidx = [0, 2, 1]
    elif case == "col_negative":
        colidx = [0, -1, 1]
    elif case == "negative_n":
        n = -1
    c, keep = _csr(n, rowptr, colidx, vals, nnz)
    if case == "bad_mem":
        c.mem = 7
    if case == "null_rowptr":
        c.rowptr = None
    rc, h = gbcg.cg_create(c, None, None)
    assert rc == gbcg.CG_EINVAL and h is None


def test_bad_options_rejected_without_gpu():
    A = problems.cube_uniform(2).A
    c, keep = gbcg.host_csr(A)
    for field, value in [("precond", 3), ("wait_limit_s", 0.0), ("wait_limit_s", float("nan")),
                         ("grid_ctas", -1), ("debug_phantom_arrivals", -2),
                         ("vectors_in_memory", 2), ("inner_values", 3), ("inner_tol", 1.5),
                         ("inner_tol", -1.0), ("max_outer", 0), ("max_inner", -1)]:
        o = gbcg.cg_opts_default()
        setattr(o, field, value)
        rc, h = gbcg.cg_create(c, o, None)
        assert rc == gbcg.CG_EINVAL and h is None, field


def test_jacobi_requires_positive_diagonal_without_gpu():
    c, keep = _csr(2, [0, 1, 2], [0, 1], [1.0, -1.0])
    o = gbcg.cg_opts_default()
    o.precond = gbcg.CG_PRECOND_JACOBI
    rc, h = gbcg.cg_create(c, o, None)
    assert rc == gbcg.CG_EINVAL
    c, keep = _csr(2, [0, 1, 1], [0], [1.0])  # row 1 has no diagonal
    rc, h = gbcg.cg_create(c, o, None)
    assert rc == gbcg.CG_EINVAL


def test_null_handles():
    gbcg.cg_destroy(None)  # no-op
    rc, info = gbcg.cg_solve(0, 0, 0, 1e-8, 0)
    assert rc == gbcg.CG_EINVAL
    # a call that fails before the solve still reports its code in info
    assert info.status == gbcg.CG_EINVAL and info.iters == 0 and info.launches == 0
    assert info.relres_true == -1.0 and info.reverted_at == -1
    rc, info = gbcg.cg_solve_host(0, 0, 0, 1e-8, 0)
    assert rc == gbcg.CG_EINVAL and info.status == gbcg.CG_EINVAL
    assert gbcg.cg_spmv(0, 0, 0) == gbcg.CG_EINVAL
    L = gbcg.lib()
    assert L.cg_create(None, None, None, None) == gbcg.CG_EINVAL
    assert L.cg_opts_default(None) == gbcg.CG_EINVAL
    assert L.cg_get_plan(None, None) == gbcg.CG_EINVAL


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1107_0538_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "cg_oracle" not in text and "liboracle" not in text, f


def test_noalloc_rejects_sizes_beyond_its_workspace_without_gpu():
    c = gbcg.cg_csr(gbcg.CG_NOALLOC_MAX_N + 1, 0, 1, 1, 1, gbcg.CG_MEM_DEVICE)
    rc, info = gbcg.cg_solve_noalloc(c, 8, 16, 1e-8, 0, None)
    assert rc == gbcg.CG_EINVAL
    assert info.status == gbcg.CG_EINVAL and info.iters == 0 and info.reverted_at == -1
    c = gbcg.cg_csr(10, 0, 1, 1, 1, gbcg.CG_MEM_HOST)  # host arrays are not accepted
    rc, _ = gbcg.cg_solve_noalloc(c, 8, 16, 1e-8, 0, None)
    assert rc == gbcg.CG_EINVAL


def test_batch_rejects_bad_arguments_without_gpu():
    A = problems.cube_uniform(2).A
    c, keep = gbcg.host_csr(A)
    arr = (gbcg.cg_csr * 2)(c, c)
    bad = gbcg.cg_opts_default()
    bad.inner_values = 7
    assert gbcg.cg_batch_create(arr, bad, None)[0] == gbcg.CG_EINVAL
    broken = (gbcg.cg_csr * 1)(gbcg.cg_csr(A.n, A.nnz + 1, c.rowptr, c.colidx, c.vals, gbcg.CG_MEM_HOST))
    assert gbcg.cg_batch_create(broken, None, None)[0] == gbcg.CG_EINVAL
    assert gbcg.lib().cg_batch_create(None, 0, None, None, None) == gbcg.CG_EINVAL
    gbcg.cg_batch_destroy(None)


def test_learned_entry_points_reject_bad_arguments_without_gpu():
    L = gbcg.lib()
    bad = np.full(gbcg.CG_LEARN_PARAMS, np.nan, dtype=np.float32)
    h = ctypes.c_void_p()
    assert L.cg_net_create(None, ctypes.byref(h)) == gbcg.CG_EINVAL
    assert L.cg_net_create(ctypes.c_void_p(bad.ctypes.data), ctypes.byref(h)) == gbcg.CG_EINVAL
    assert L.cg_net_create(ctypes.c_void_p(bad.ctypes.data), None) == gbcg.CG_EINVAL
    assert L.cg_net_get_params(None, None) == gbcg.CG_EINVAL
    assert L.cg_net_set_params(None, None) == gbcg.CG_EINVAL
    gbcg.cg_net_destroy(None)
    assert gbcg.cg_set_learned(0, 0, 4, 4, 4, np.zeros(125)) == gbcg.CG_EINVAL
    assert gbcg.cg_precond_apply(0, 8, 16) == gbcg.CG_EINVAL
    assert gbcg.cg_learn_pairs(0, 8, 16, 4, 4, 32, 64) == gbcg.CG_EINVAL
    s = gbcg.cg_learn_set(0, None, 0, None, None, None)
    assert gbcg.cg_learn_grad(0, s, np.zeros(1, np.int64))[0] == gbcg.CG_EINVAL
    assert gbcg.cg_learn_train(0, s, np.zeros(1, np.int64), 1, 1, 1e-3)[0] == gbcg.CG_EINVAL
    # the learned preconditioner is FP64-only
    o = gbcg.cg_opts_default()
    o.precond = gbcg.CG_PRECOND_LEARNED
    o.inner_values = gbcg.CG_VALUES_FP32
    A = problems.cube_uniform(2).A
    c, keep = gbcg.host_csr(A)
    assert gbcg.cg_create(c, o, None)[0] == gbcg.CG_EINVAL
