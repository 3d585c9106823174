"""Builds libgbcg.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1107_0538_gb300.build [-v]

Three translation units, one -gencode, static CUDA runtime; the result sits next
to this file as libgbcg.so and is loaded by ``gbcg.lib()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
SOURCES = [os.path.join(_HERE, "csrc", f) for f in ("gbcg.cu", "noalloc.cu", "batch.cu")]
DEPS = SOURCES + [os.path.join(_HERE, "csrc", f) for f in ("cg_device.cuh", "layout.h", "plan.h")] + [
    os.path.join(ROOT, "include", "gbcg.h")]
OUT = os.path.join(_HERE, "libgbcg.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None) -> str:
    if (not force and not extra and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= max(os.path.getmtime(d) for d in DEPS)):
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [nvcc_path(), "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", ARCH, "-lineinfo",
           "-I", os.path.join(ROOT, "include"), "-o", tmp] + SOURCES
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    if extra:
        cmd[1:1] = extra
    res = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or res.returncode:
        sys.stderr.write(res.stdout + res.stderr)
    if res.returncode:
        raise RuntimeError(f"nvcc failed ({res.returncode}): {' '.join(cmd)}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
