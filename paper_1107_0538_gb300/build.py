"""Builds libgbcg.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1107_0538_gb300.build [-v]

Four translation units compiled in parallel (one -gencode each) into _build/,
then linked with the static CUDA runtime; the result sits next to this file as
libgbcg.so and is loaded by ``gbcg.lib()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
SOURCES = [os.path.join(_HERE, "csrc", f) for f in ("gbcg.cu", "noalloc.cu", "batch.cu", "learn.cu")]
DEPS = SOURCES + [os.path.join(_HERE, "csrc", f) for f in ("cg_device.cuh", "layout.h", "plan.h", "lowprec.h",
                                                           "handle.h", "sell.cuh")] + [
    os.path.join(ROOT, "include", "gbcg.h")]
OUT = os.path.join(_HERE, "libgbcg.so")
OBJDIR = os.path.join(_HERE, "_build")
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
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = nvcc_path()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", ARCH, "-lineinfo", "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.insert(0, "-Xptxas=-v")
    if extra:
        common = list(extra) + common
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, os.path.basename(src) + f".{os.getpid()}.o")
        objs.append(obj)
        cmd = [nvcc, "-c"] + common + ["-o", obj, src]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = None
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode:
            sys.stderr.write(out)
        if pr.returncode and failed is None:
            failed = (pr.returncode, cmd)
    if failed:
        raise RuntimeError(f"nvcc failed ({failed[0]}): {' '.join(failed[1])}")
    tmp = OUT + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", ARCH, "-o", tmp] + objs
    res = subprocess.run(link, capture_output=True, text=True)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    if verbose or res.returncode:
        sys.stderr.write(res.stdout + res.stderr)
    if res.returncode:
        raise RuntimeError(f"nvcc link failed ({res.returncode}): {' '.join(link)}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
