"""Builds libgbcg.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1107_0538_gb300.build [-v]

Four translation units, each compiled twice in parallel (one -gencode each):
once for libgbcg.so, the library, and once with -DGBCG_BOUNDS_CHECK for
libgbcg_check.so, the bounds-check build whose kernels test and count every
index they gather through.  Objects go to _build/; each library is linked
with the static CUDA runtime and sits next to this file (``gbcg.lib()``
loads libgbcg.so, or libgbcg_check.so when GBCG_LIBRARY=check).
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
                                                           "handle.h", "sell.cuh", "sellsolve.cuh",
                                                           "check.cuh")] + [
    os.path.join(ROOT, "include", "gbcg.h")]
OUT = os.path.join(_HERE, "libgbcg.so")
OUT_CHECK = os.path.join(_HERE, "libgbcg_check.so")
OBJDIR = os.path.join(_HERE, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
VARIANTS = {OUT: [], OUT_CHECK: ["-DGBCG_BOUNDS_CHECK"]}


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: str) -> bool:
    return not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(d) for d in DEPS)


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None) -> str:
    """Builds both libraries (only what is out of date unless force or extra
    flags are given) and returns the path of libgbcg.so."""
    outs = [o for o in VARIANTS if force or extra or _stale(o)]
    if not outs:
        return OUT
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = nvcc_path()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", ARCH, "-lineinfo", "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.insert(0, "-Xptxas=-v")
    if extra:
        common = list(extra) + common
    procs, objs = [], {o: [] for o in outs}
    for out in outs:
        tag = "check" if out == OUT_CHECK else "lib"
        for src in SOURCES:
            obj = os.path.join(OBJDIR, f"{os.path.basename(src)}.{tag}.{os.getpid()}.o")
            objs[out].append(obj)
            cmd = [nvcc, "-c"] + VARIANTS[out] + common + ["-o", obj, src]
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = None
    for cmd, pr in procs:
        text, _ = pr.communicate()
        if verbose or pr.returncode:
            sys.stderr.write(text)
        if pr.returncode and failed is None:
            failed = (pr.returncode, cmd)
    if failed:
        for ol in objs.values():
            for o in ol:
                if os.path.exists(o):
                    os.remove(o)
        raise RuntimeError(f"nvcc failed ({failed[0]}): {' '.join(failed[1])}")
    for out in outs:
        tmp = out + f".tmp{os.getpid()}"
        link = [nvcc, "-shared", ARCH, "-o", tmp] + objs[out]
        res = subprocess.run(link, capture_output=True, text=True)
        for o in objs[out]:
            try:
                os.remove(o)
            except OSError:
                pass
        if verbose or res.returncode:
            sys.stderr.write(res.stdout + res.stderr)
        if res.returncode:
            raise RuntimeError(f"nvcc link failed ({res.returncode}): {' '.join(link)}")
        os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
