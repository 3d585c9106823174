#!/usr/bin/env python
"""Benchmark of the CG hot path on the paper-sized system.

Workload: the Q1 hexahedral FEM matrix of a 50^3-element cube (N = 132651,
NNZ = 3442951, the sizes of the paper's Section IV matrix), nu = 1 air with
seeded iron blobs at nu = 1e-3, b = A x* for a seeded smooth x*, x0 = 0.
A step is one FP64 CG solve to ||r|| <= 1e-8 ||b|| through the C ABI
(one persistent kernel launch).  The L2 cache is flushed (a 2x L2 buffer
is written) before every timed solve, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbcg|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64
oracle (serial C) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ms per solve to rel. residual 1e-8; SpMV HBM GB/s; chosen form vs FP64 CG"
UNIT = "ms/solve"
TOL = 1e-8
WORKLOAD = ("q1-50^3 Q1 hex FEM, nu 1 / 1e-3 iron blobs (contrast 1e3), N=132651, NNZ=3442951, "
            "b = A x*, x0 = 0, FP64 CG to rel. residual 1e-8")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gbcg", "reference"], default="gbcg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 100^3 SpMV roofline, the other forms, the batch and the CPU baseline")
    ap.add_argument("--section", choices=["spmv", "forms", "forms100", "batched", "batched_small", "learned",
                                          "learned_iter", "learned_iter100", "fp64peak"],
                    help="run one extra section alone and print its JSON: the 100^3 SpMV roofline, the "
                         "other forms on the 50^3 workload, the forms on the 100^3 system, "
                         "the 256-system batch (edges 20..80), a 64-system batch (edges 20..40), "
                         "the learned preconditioner (training and tests), the time per flexible-CG "
                         "iteration with an untrained network at 50^3 and 100^3 (or 100^3 alone), or the "
                         "FP64 peak probe")
    ap.add_argument("--batched-full", action="store_true", help="same as --section batched")
    ap.add_argument("--learned-only", action="store_true", help="same as --section learned")
    return ap.parse_args()


def bytes_per_iteration(n: int, nnz: int, precond: bool) -> int:
    """Algorithmic bytes of one fused CG iteration: CSR stream (12 NNZ + 4(N+1))
    plus 11 FP64 vector passes (88 N); Jacobi adds a read of 1/diag and a write
    of z (16 N)."""
    return 12 * nnz + 4 * (n + 1) + 88 * n + (16 * n if precond else 0)


def flops_per_iteration(n: int, nnz: int, precond: bool) -> int:
    """The paper's count for one CG iteration (Table I): 2 NNZ + 10 N; Jacobi adds 3 N."""
    return 2 * nnz + 10 * n + (3 * n if precond else 0)


def fp64_peak(stream) -> dict:
    """FP64 throughput of this GPU, measured in this run (cg_fp64_peak: 4 x SMs
    CTAs x 512 threads, 8 independent FMA chains per thread, CUDA events),
    next to the nominal figure from the device's SM count and the maximum SM
    clock (2 FP64 FMA per clock per SM)."""
    import torch

    from paper_1107_0538_gb300 import gbcg
    rc, flops, ms = gbcg.cg_fp64_peak(stream.cuda_stream, 4000)
    if rc != gbcg.CG_OK or ms <= 0:
        raise RuntimeError(f"cg_fp64_peak failed: {gbcg.cg_strerror(rc)}")
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return {"tflops": round(flops / ms / 1e9, 4), "ms": round(ms, 3), "sms": sms,
            "method": "cg_fp64_peak: 4 x SMs CTAs x 512 threads x 8 independent FP64 FMA chains, CUDA events"}


def spmv_bytes(n: int, nnz: int) -> int:
    """Algorithmic bytes of y = A x: CSR stream, x read once, y written once."""
    return 12 * nnz + 4 * (n + 1) + 16 * n


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# Sources whose content fixes each kernel's code and launch plan: a capture in
# profiles/ncu_traffic.txt counts only while their digest is unchanged.
_COMMON = ["cg_device.cuh", "layout.h"]
KERNEL_SOURCES = {
    "cg_solve_kernel": ["gbcg.cu", "plan.h"] + _COMMON,
    "cg_sell_kernel": ["gbcg.cu", "sell.cuh", "sellsolve.cuh", "plan.h"] + _COMMON,
    "cg_sellmem_kernel": ["gbcg.cu", "sell.cuh", "sellsolve.cuh", "plan.h"] + _COMMON,
    "sell_spmv_kernel": ["gbcg.cu", "sell.cuh", "plan.h"],
    "cg_ir_kernel": ["gbcg.cu", "plan.h", "lowprec.h"] + _COMMON,
    "cg_irsell_kernel": ["gbcg.cu", "sell.cuh", "sellsolve.cuh", "plan.h", "lowprec.h"] + _COMMON,
    "cg_batch_kernel": ["batch.cu", "plan.h", "lowprec.h"] + _COMMON,
    "conv16_kernel": ["learn.cu"] + _COMMON,
    "conv16tc_kernel": ["learn.cu"] + _COMMON,
    "convout_kernel": ["learn.cu"] + _COMMON,
    "conv1_kernel": ["learn.cu"] + _COMMON,
    "fcg_spmv_kernel": ["learn.cu", "plan.h"] + _COMMON,
    "fcg_sell_kernel": ["learn.cu", "sell.cuh", "sellsolve.cuh"] + _COMMON,
}


def source_digest(kernel: str) -> str:
    """sha256 (first 16 hex digits) of the kernel's source files in order."""
    import hashlib
    src = os.path.join(ROOT, "paper_1107_0538_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str) -> dict | None:
    """DRAM bytes per launch of a kernel from the committed ncu capture summary
    (profiles/ncu_traffic.txt), if it was taken on the current kernel source
    (digest match), else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    digest = source_digest(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
            return {"dram_bytes_per_launch": float(parts[2])}
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device) -> float:
    """The largest `value` over the ranks of the default process group: the
    job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_solve(total_ms: float, steps: int, world: int) -> float:
    """Whole-job ms per solve: every rank solves `steps` systems in the
    slowest rank's `total_ms`."""
    return total_ms / (steps * world)


def run_reference(args) -> None:
    """The oracle (serial C, FP64) on the same workload, on the host cores."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    from paper_1107_0538_gb300 import problems
    pr = problems.cube_blobs(50)
    times, iters = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.cg(pr.A, pr.b, tol=TOL)
        dt = (time.perf_counter() - t0) * 1e3
        assert r["status"] == oracle.OK
        iters = r["iters"]
        if i >= args.warmup:
            times.append(dt)
    v = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": pr.A.n, "nnz": pr.A.nnz,
                                        "tol": TOL, "iters": iters},
        "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"full serial FP64 CG solves of the same system ({iters} iterations each)"},
        "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def generate_batch(nsys: int, emin: int, emax: int, seed0: int = 1000, threads: int = 16) -> list:
    """problems.batch_systems, one system per task on a thread pool (numpy
    releases the GIL in the array work): the same systems, generated faster."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1107_0538_gb300 import problems
    with ThreadPoolExecutor(max(1, min(threads, os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda i: problems.batch_systems(1, emin, emax, seed0=seed0 + i)[0], range(nsys)))


def measure_batched(nsys: int, emin: int, emax: int, steps: int, tune_sys: int, sample: int) -> dict:
    """Batched mixed-precision solves of nsys uneven Q1 boxes x 4 source-current
    right-hand sides in one persistent launch (FP32 inner CG with Jacobi, FP64
    refinement, rel. residual 1e-8): ms per batch, the same enqueue captured
    in a CUDA graph and replayed, the autotuner's choice on the first tune_sys
    systems, and the error of sampled pairs against a tight FP64 GPU solve."""
    import torch

    from paper_1107_0538_gb300 import gbcg
    t0 = time.perf_counter()
    sl = generate_batch(nsys, emin, emax)
    gen_s = time.perf_counter() - t0
    n_tot = sum(s["A"].n for s in sl)
    nnz_tot = sum(s["A"].nnz for s in sl)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"workload": f"{nsys} Q1 boxes, edges U{{{emin}..{emax}}}, contrast log-U[1e2, 1e4], 4 source-current rhs "
                       f"each, FP32 inner CG (Jacobi) + FP64 refinement to rel. residual {TOL:g}",
           "systems": nsys, "rhs": 4, "n_total": n_tot, "nnz_total": nnz_tot, "generate_s": round(gen_s, 2)}
    choice = None
    if tune_sys:
        sub = sl[:tune_sys]
        with gbcg.BatchSolver([x["A"] for x in sub], inner_values=gbcg.CG_VALUES_FP32,
                              precond=gbcg.CG_PRECOND_JACOBI) as tb:
            Bt = torch.from_numpy(np.concatenate([x["B"] for x in sub], axis=1)).to(dev).contiguous()
            rc, ch = tb.tune(Bt, torch.zeros_like(Bt), TOL)
            out["tuned"] = {"on": f"the first {tune_sys} systems", "status": rc, "inner_tol": ch.inner_tol,
                            "gather_tiles": ch.gather_tiles, "lanes_per_row": ch.lanes_per_row,
                            "trials": ch.trials, "best_ms": round(ch.best_ms, 3),
                            "space": "inner tol {1e-2, 3e-3, 1e-3, 1e-4} x tiles {x-window, gather} x "
                                     "rows per warp step {32, 16, 8}"}
            choice = (ch.inner_tol, ch.gather_tiles, ch.lanes_per_row) if rc == gbcg.CG_OK else None
            del Bt
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    bs = gbcg.BatchSolver([x["A"] for x in sl], inner_values=gbcg.CG_VALUES_FP32, precond=gbcg.CG_PRECOND_JACOBI,
                          stream=stream)
    out["create_s"] = round(time.perf_counter() - t0, 2)
    if tune_sys and choice is not None:
        bs.set_tuning(*choice)   # the sub-batch's choice applied to the whole batch
    B = torch.from_numpy(np.concatenate([x["B"] for x in sl], axis=1)).to(dev).contiguous()
    X = torch.zeros_like(B)
    torch.cuda.synchronize()
    rc, res, ms = bs.solve(B, X, TOL)  # warm-up
    times = []
    for _ in range(steps):
        X.zero_()
        torch.cuda.synchronize()
        rc, res, ms = bs.solve(B, X, TOL)
        times.append(ms)
    ok = sum(1 for r in res if r.status == gbcg.CG_OK)
    batch_ms = statistics.median(times)
    out.update({"status": rc, "pairs_converged": ok, "pairs": len(res), "ms_per_batch": round(batch_ms, 3),
                "ms_per_solve_amortised": round(batch_ms / len(res), 4),
                "inner_iters_max": max(r.iters for r in res), "outer_max": max(r.outer for r in res),
                "relres_max": max(r.relres for r in res)})
    # the same solve with the inner loop keeping the creation-time split of
    # the tiles instead of re-splitting the active ones over the CTAs
    if choice is not None:
        bs.set_tuning(*choice, 1)
        X.zero_()
        torch.cuda.synchronize()
        rcs, ress, ms_static = bs.solve(B, X, TOL)
        out["static_split"] = {"ms_per_batch": round(ms_static, 3), "status": rcs,
                               "pairs_converged": sum(1 for r in ress if r.status == gbcg.CG_OK)}
        bs.set_tuning(*choice, 0)
    # the whole batch's enqueue (copies, memsets, the cooperative launch)
    # captured in one CUDA graph and replayed
    try:
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            rcq = bs.enqueue(B, X, TOL)
        X.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
        e1.synchronize()
        rcg, resg = bs.results(4)
        out["graph"] = {"captured": rcq == gbcg.CG_OK, "replay_ms": round(e0.elapsed_time(e1), 3),
                        "replay_status": rcg, "pairs_converged": sum(1 for r in resg if r.status == gbcg.CG_OK),
                        "systems": nsys}
        del g
    except Exception as exc:  # report, do not hide
        out["graph"] = {"captured": False, "error": str(exc)[:200]}
    # error of sampled pairs against a tight FP64 CG solve on the GPU
    Xh = X.cpu().numpy()
    errs = []
    offs = np.concatenate([[0], np.cumsum([s["A"].n for s in sl])])
    order = sorted(range(nsys), key=lambda i: sl[i]["A"].n)[:sample]
    for i in order:
        fs = gbcg.Solver(sl[i]["A"], precond=gbcg.CG_PRECOND_JACOBI)
        for r in range(4):
            bt = torch.from_numpy(sl[i]["B"][r]).to(dev)
            xt = torch.zeros_like(bt)
            fs.solve(bt, xt, 1e-13)
            ref = xt.cpu().numpy()
            x = Xh[r, offs[i]:offs[i + 1]]
            errs.append(float(np.linalg.norm(x - ref) / np.linalg.norm(ref)))
        fs.close()
    out["err_vs_fp64_cg_max"] = max(errs) if errs else None
    out["err_sample"] = (f"{len(errs)} pairs of the {len(order)} smallest systems (graph replay's X), against "
                         f"FP64 Jacobi-PCG on the GPU to rel. residual 1e-13")
    bs.close()
    del B, X
    torch.cuda.empty_cache()
    return out


def measure_learned(ninst: int = 40, per: int = 500, seg: int = 8, batch: int = 8, lr: float = 1e-3,
                    reps: int = 3, epochs: int = 3, nheld: int = 2) -> dict:
    """The learned preconditioner end to end on the GPU: training pairs from
    restarted FP64 CG on ninst random 50^3 instances (contrast 1e3, seeds
    10000+), `epochs` epochs of Adam through the project's kernels with the
    loss on held-out pairs (nheld instances never trained on, seeds 15000+)
    after each, then flexible CG with the network against FP64 CG and
    Jacobi-PCG on the 50^3 workload and on an unseen 100^3 instance (seed
    20000), to rel. residual 1e-8."""
    import torch

    from paper_1107_0538_gb300 import gbcg, problems
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"workload": f"train: {ninst} q1-50^3 blob instances x {per} (residual, error) pairs from restarted "
                       f"FP64 CG (segments of {seg}); test: flexible CG to rel. residual {TOL:g}"}
    t0 = time.perf_counter()
    train = [problems.learn_instance(50, 10000 + i) for i in range(ninst)]
    out["instances_s"] = round(time.perf_counter() - t0, 2)
    net = gbcg.Net(problems.learn_init_params())
    solvers = []
    for inst in train:
        s = gbcg.Solver(inst.A, precond=gbcg.CG_PRECOND_LEARNED)
        s.set_learned(net, inst.grid, inst.lognu.astype(np.float32))
        solvers.append(s)
    n = train[0].A.n
    R = torch.empty((ninst * per, n), dtype=torch.float32, device=dev)
    E = torch.empty_like(R)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, (inst, s) in enumerate(zip(train, solvers)):
        s.learn_pairs(torch.from_numpy(inst.b).to(dev), torch.from_numpy(inst.xstar).to(dev), seg, per,
                      R[k * per:(k + 1) * per], E[k * per:(k + 1) * per])
    torch.cuda.synchronize()
    out["pairs"] = ninst * per
    out["pairs_s"] = round(time.perf_counter() - t0, 2)
    pinst = np.repeat(np.arange(ninst), per)
    lset = gbcg.LearnSet(solvers, pinst, R, E)
    # held-out pairs: the same recipe on instances the network never trains on
    held_inst = [problems.learn_instance(50, 15000 + i) for i in range(nheld)]
    held_solvers = []
    Rh = torch.empty((nheld * per, n), dtype=torch.float32, device=dev)
    Eh = torch.empty_like(Rh)
    for k, inst in enumerate(held_inst):
        s = gbcg.Solver(inst.A, precond=gbcg.CG_PRECOND_LEARNED)
        s.set_learned(net, inst.grid, inst.lognu.astype(np.float32))
        s.learn_pairs(torch.from_numpy(inst.b).to(dev), torch.from_numpy(inst.xstar).to(dev), seg, per,
                      Rh[k * per:(k + 1) * per], Eh[k * per:(k + 1) * per])
        held_solvers.append(s)
    hset = gbcg.LearnSet(held_solvers, np.repeat(np.arange(nheld), per), Rh, Eh)
    held = np.arange(nheld * per)
    sample = np.arange(0, len(pinst), max(1, len(pinst) // 256))
    steps = len(pinst) // batch
    curve = [{"epoch": 0, "held_out_loss": round(net.grad(hset, held)[0], 5),
              "train_sample_loss": round(net.grad(lset, sample)[0], 5)}]
    train_s = 0.0
    for ep in range(epochs):
        order = (problems.splitmix64(77 + ep, steps * batch) % np.uint64(len(pinst))).astype(np.int64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.train(lset, order, steps, batch, lr)
        torch.cuda.synchronize()
        train_s += time.perf_counter() - t0
        curve.append({"epoch": ep + 1, "held_out_loss": round(net.grad(hset, held)[0], 5),
                      "train_sample_loss": round(net.grad(lset, sample)[0], 5)})
    out["train"] = {"steps_per_epoch": steps, "batch": batch, "lr": lr, "epochs": epochs, "s": round(train_s, 2),
                    "loss_by_epoch": curve,
                    "held_out": f"{nheld * per} pairs from {nheld} 50^3 instances not trained on (seeds 15000+)",
                    "train_sample": f"{len(sample)} training pairs, every {max(1, len(pinst) // 256)}th"}
    del R, E, lset, Rh, Eh, hset
    for s in solvers + held_solvers:
        s.close()
    torch.cuda.empty_cache()

    def run(A, b, mk):
        s = mk()
        bt = torch.from_numpy(b).to(dev)
        x = torch.zeros_like(bt)
        s.solve(bt, x, TOL)
        ts, info = [], None
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            info = s.solve(bt, x, TOL)
            ts.append(info.kernel_ms)
        s.close()
        return {"ms_per_solve": round(statistics.median(ts), 3), "iters": info.iters, "status": info.status,
                "relres_true": info.relres_true, "reverted_at": info.reverted_at}

    def learned_solver(A, grid, lognu):
        def mk():
            s = gbcg.Solver(A, precond=gbcg.CG_PRECOND_LEARNED)
            s.set_learned(net, grid, lognu.astype(np.float32))
            return s
        return mk

    c2 = problems.cube_blobs(50)
    test100 = problems.learn_instance(100, 20000)
    for key, A, b, grid, lognu in (("q1_50cube_c2", c2.A, c2.b, c2.grid, problems.node_log_nu(c2.grid, c2.nu)),
                                   ("q1_100cube_unseen", test100.A, test100.b, test100.grid, test100.lognu)):
        res = {"fp64_cg": run(A, b, lambda: gbcg.Solver(A)),
               "jacobi_pcg": run(A, b, lambda: gbcg.Solver(A, precond=gbcg.CG_PRECOND_JACOBI)),
               "learned_fcg": run(A, b, learned_solver(A, grid, lognu))}
        lf = res["learned_fcg"]
        lf["speedup_vs_fp64_cg"] = round(res["fp64_cg"]["ms_per_solve"] / lf["ms_per_solve"], 3)
        lf["speedup_vs_jacobi_pcg"] = round(res["jacobi_pcg"]["ms_per_solve"] / lf["ms_per_solve"], 3)
        lf["iters_vs_jacobi_pcg"] = round(lf["iters"] / max(res["jacobi_pcg"]["iters"], 1), 3)
        out[key] = res
    net.close()
    return out


def timed_solves(solver, b, x, count, flush, record=True):
    """count solves of b from x = 0 with the L2 flushed before each, timed by
    CUDA events on the current stream: [(ms, info), ...]."""
    import torch

    from paper_1107_0538_gb300 import gbcg
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(count):
        x.zero_()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = solver.solve(b, x, tol=TOL)
        e1.record(stream)
        e1.synchronize()
        if info.status != gbcg.CG_OK:
            raise RuntimeError(f"solve failed: {gbcg.cg_strerror(info.status)}")
        if record:
            out.append((e0.elapsed_time(e1), info))
    return out


def l2_flush_buffer():
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    l2 = int(getattr(props, "L2_cache_size", 126 * 2 ** 20))
    return torch.empty(2 * l2 // 4, dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))


def measure_forms(pr, ms_fp64: float, iters_fp64: int, count: int, x_ref, flush) -> dict:
    """Jacobi-PCG and FP32/BF16 refinement (with and without Jacobi) on the
    50^3 workload: ms per solve, iterations, true residual, error against the
    oracle's solution (x_ref, from the CPU baseline leg; None: against x*)."""
    import torch

    from paper_1107_0538_gb300 import gbcg
    dev = torch.device("cuda", torch.cuda.current_device())
    b = torch.from_numpy(pr.b).to(dev)
    x = torch.zeros_like(b)
    ref = x_ref if x_ref is not None else pr.xstar
    key = "err_vs_fp64_oracle" if x_ref is not None else "err_vs_xstar"
    forms = {"fp64_cg": {"ms_per_solve": round(ms_fp64, 4), "iters": iters_fp64}}
    variants = [("jacobi_pcg", dict(precond=gbcg.CG_PRECOND_JACOBI)),
                ("fp32_ir", dict(inner_values=gbcg.CG_VALUES_FP32)),
                ("bf16_ir", dict(inner_values=gbcg.CG_VALUES_BF16)),
                ("fp32_ir_jacobi", dict(inner_values=gbcg.CG_VALUES_FP32, precond=gbcg.CG_PRECOND_JACOBI)),
                ("bf16_ir_jacobi", dict(inner_values=gbcg.CG_VALUES_BF16, precond=gbcg.CG_PRECOND_JACOBI))]
    for name, kw in variants:
        vs = gbcg.Solver(pr.A, **kw)
        timed_solves(vs, b, x, 2, flush, False)
        res_v = timed_solves(vs, b, x, count, flush)
        v_ms = statistics.mean(t for t, _ in res_v)
        xv = x.cpu().numpy()
        info_v = res_v[-1][1]
        forms[name] = {"ms_per_solve": round(v_ms, 4), "iters": info_v.iters, "outer": info_v.outer,
                       "relres_true": info_v.relres_true,
                       key: float(np.linalg.norm(xv - ref) / np.linalg.norm(ref)),
                       "speedup_vs_fp64_cg": round(ms_fp64 / v_ms, 3)}
        vs.close()
    return forms


def measure_forms_100cube(flush, fp64_tflops: float, count: int = 2) -> dict:
    """The mixed-precision forms on the 100^3 system (N=1030301, NNZ=27270901,
    contrast 1e3, b = A x*): the FP64 matrix (327 MB of CSR) no longer fits
    the L2, so the 8- and 6-byte inner entries of FP32/BF16 refinement cut
    the bytes each inner iteration streams. ms per solve to rel. residual
    1e-8, iterations, true residual, and the error against the GPU FP64 CG
    solution (parity-tested against the oracle) and against x*."""
    import torch

    from paper_1107_0538_gb300 import gbcg, problems
    dev = torch.device("cuda", torch.cuda.current_device())
    big = problems.cube_blobs(100)
    b = torch.from_numpy(big.b).to(dev)
    x = torch.zeros_like(b)
    out = {"workload": "q1-100^3 blobs (contrast 1e3), N=1030301, NNZ=27270901, b = A x*, x0 = 0, "
                       "rel. residual 1e-8, L2 flushed before each solve"}
    x_fp64 = None
    ms_fp64 = None
    variants = [("fp64_cg", {}), ("jacobi_pcg", dict(precond=gbcg.CG_PRECOND_JACOBI)),
                ("fp32_ir", dict(inner_values=gbcg.CG_VALUES_FP32)),
                ("bf16_ir", dict(inner_values=gbcg.CG_VALUES_BF16)),
                ("fp32_ir_jacobi", dict(inner_values=gbcg.CG_VALUES_FP32, precond=gbcg.CG_PRECOND_JACOBI)),
                ("bf16_ir_jacobi", dict(inner_values=gbcg.CG_VALUES_BF16, precond=gbcg.CG_PRECOND_JACOBI))]
    for name, kw in variants:
        # refinement forms: the inner tolerance that solves fastest (the
        # others are listed), as the batched solver's tuner picks it
        tols = ([1e-2, 3e-3, 1e-3] if kw.get("inner_values") == gbcg.CG_VALUES_FP32 else
                [1e-2, 3e-3] if kw.get("inner_values") == gbcg.CG_VALUES_BF16 else [None])
        best = None
        tried = {}
        for it in tols:
            vs = gbcg.Solver(big.A, **kw, **({} if it is None else {"inner_tol": it}))
            timed_solves(vs, b, x, 1, flush, False)
            res_v = timed_solves(vs, b, x, count, flush)
            v_ms = statistics.mean(t for t, _ in res_v)
            if it is not None:
                tried[f"{it:g}"] = round(v_ms, 3)
            if best is None or v_ms < best[0]:
                best = (v_ms, res_v[-1][1], x.cpu().numpy(), vs.plan(), it)
            vs.close()
        v_ms, info_v, xv, plan_v, it_best = best
        if name == "fp64_cg":
            x_fp64, ms_fp64 = xv.copy(), v_ms
            # FP64-ALU roofline of the solve kernel (Table I's flop count)
            kern = "cg_sellmem_kernel" if plan_v["slice_solve"] == 2 else "cg_solve_kernel"
            kern_s = statistics.mean(i.kernel_ms for _, i in res_v) / 1e3
            flops = info_v.iters * flops_per_iteration(big.A.n, big.A.nnz, False)
            tr = ncu_traffic(kern)
            nbytes = info_v.iters * bytes_per_iteration(big.A.n, big.A.nnz, False)
            hbm = measured_peaks()["hbm_gbs"]
            out["roofline"] = {"bound": "hbm", "kernel": kern, "achieved": round(nbytes / kern_s / 1e9, 1),
                               "peak": hbm, "unit": "GB/s", "frac": round(nbytes / kern_s / 1e9 / hbm, 4),
                               "traffic": (round(tr["dram_bytes_per_launch"]) if tr else None),
                               "algorithmic_bytes_per_launch": nbytes,
                               "fp64_achieved_tflops": round(flops / kern_s / 1e12, 4),
                               "fp64_peak_tflops": fp64_tflops,
                               "fp64_frac": round(flops / kern_s / 1e12 / fp64_tflops, 4)}
        out[name] = {"ms_per_solve": round(v_ms, 3), "iters": info_v.iters, "outer": info_v.outer,
                     "relres_true": info_v.relres_true,
                     "err_vs_fp64_cg": float(np.linalg.norm(xv - x_fp64) / np.linalg.norm(x_fp64)),
                     "err_vs_xstar": float(np.linalg.norm(xv - big.xstar) / np.linalg.norm(big.xstar)),
                     "speedup_vs_fp64_cg": round(ms_fp64 / v_ms, 3)}
        if tried:
            out[name]["inner_tol"] = it_best
            out[name]["ms_by_inner_tol"] = tried
    return out


def measure_spmv_hbm(peaks: dict, flush, fp64_tflops: float) -> dict:
    """One FP64 SpMV (cg_spmv: the SELL-32 kernel) on the 100^3 system (27.3M
    entries), L2 flushed before each of 20 launches, median time against the
    measured HBM peak."""
    import torch

    from paper_1107_0538_gb300 import gbcg, problems
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    big = problems.cube_blobs(100)
    bs = gbcg.Solver(big.A)
    xb = torch.from_numpy(np.random.default_rng(0).standard_normal(big.A.n)).to(dev)
    yb = torch.empty_like(xb)
    for _ in range(3):
        bs.spmv(xb, yb)
    ts = []
    for _ in range(20):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bs.spmv(xb, yb)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    bs.close()
    t_med = statistics.median(ts) / 1e3
    sb = spmv_bytes(big.A.n, big.A.nnz)
    gbs = sb / t_med / 1e9
    trs = ncu_traffic("sell_spmv_kernel")
    return {
        "workload": "q1-100^3 blobs, N=1030301, NNZ=27270901, FP64 SpMV, L2 flushed",
        "kernel": "sell_spmv_kernel", "us": round(t_med * 1e6, 2), "achieved": round(gbs, 1),
        "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4),
        "algorithmic_bytes": sb,
        "fp64_frac": round(2 * big.A.nnz / t_med / 1e12 / fp64_tflops, 4),
        "traffic": (round(trs["dram_bytes_per_launch"]) if trs else None),
    }


def measure_learned_iter(maxits=(12, 36), grids=(50, 100)) -> dict:
    """ms per flexible-CG iteration with the untrained network (the cost of an
    iteration does not depend on the weights): the slope between maxit = 12 and
    36 on the 50^3 workload grid and on a 100^3 instance."""
    import torch

    from paper_1107_0538_gb300 import gbcg, problems
    dev = torch.device("cuda", torch.cuda.current_device())
    net = gbcg.Net(problems.learn_init_params())
    out = {}
    for e in grids:
        inst = problems.learn_instance(e, 20001)
        s = gbcg.Solver(inst.A, precond=gbcg.CG_PRECOND_LEARNED, true_residual=False)
        s.set_learned(net, inst.grid, inst.lognu.astype(np.float32))
        b = torch.from_numpy(inst.b).to(dev)
        ms = {}
        for m in maxits:
            ts = []
            for _ in range(3):
                x = torch.zeros_like(b)
                ts.append(s.solve(b, x, 1e-14, maxit=m).kernel_ms)
            ms[m] = statistics.median(ts)
        s.close()
        out[f"q1_{e}cube"] = {"ms_per_iteration": round((ms[maxits[1]] - ms[maxits[0]]) / (maxits[1] - maxits[0]), 4),
                              "n": inst.A.n, "nnz": inst.A.nnz}
    net.close()
    return out


def run_section(args) -> None:
    """--section NAME: one extra section alone (no headline line)."""
    import torch

    from paper_1107_0538_gb300 import gbcg, problems
    torch.cuda.set_device(0)
    gbcg.lib()
    name = "batched" if args.batched_full else "learned" if args.learned_only else args.section
    if name == "spmv":
        out = measure_spmv_hbm(measured_peaks(), l2_flush_buffer(), fp64_peak(torch.cuda.current_stream())["tflops"])
    elif name == "forms":
        flush = l2_flush_buffer()
        pr = problems.cube_blobs(50)
        s = gbcg.Solver(pr.A)
        b = torch.from_numpy(pr.b).to(torch.device("cuda", 0))
        x = torch.zeros_like(b)
        timed_solves(s, b, x, 2, flush, False)
        res = timed_solves(s, b, x, 3, flush)
        s.close()
        out = measure_forms(pr, statistics.mean(t for t, _ in res), res[-1][1].iters, 3, None, flush)
    elif name == "forms100":
        out = measure_forms_100cube(l2_flush_buffer(), fp64_peak(torch.cuda.current_stream())["tflops"])
    elif name == "batched":
        out = measure_batched(256, 20, 80, 1, tune_sys=32, sample=2)
    elif name == "batched_small":
        out = measure_batched(64, 20, 40, 3, tune_sys=64, sample=2)
    elif name == "fp64peak":
        out = fp64_peak(torch.cuda.current_stream())
    elif name == "learned_iter":
        out = measure_learned_iter()
    elif name == "learned_iter100":
        out = measure_learned_iter(grids=(100,))
    else:
        out = measure_learned()
    print(json.dumps({"section": name, name: out}), flush=True)


def run_gbcg(args) -> None:
    import torch
    import torch.distributed as dist

    from paper_1107_0538_gb300 import gbcg, problems

    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbcg.lib()
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    l2 = int(getattr(props, "L2_cache_size", 126 * 2 ** 20))

    pr = problems.cube_blobs(50)
    n, nnz = pr.A.n, pr.A.nnz
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # ---------------------------------------------------- FP64 CG (the step)
    solver = gbcg.Solver(pr.A)
    b = torch.from_numpy(pr.b).to(dev)
    x = torch.zeros_like(b)
    timed_solves(solver, b, x, args.warmup, flush, False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        res = timed_solves(solver, b, x, args.steps, flush)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = sum(t for t, _ in res)
    kern_ms = [i.kernel_ms for _, i in res]
    iters = res[-1][1].iters
    relres_true = res[-1][1].relres_true
    launches = sum(i.launches for _, i in res)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    value = job_ms_per_solve(total_ms, args.steps, world)

    bpi = bytes_per_iteration(n, nnz, False)
    fpi = flops_per_iteration(n, nnz, False)
    kern_s = statistics.mean(kern_ms) / 1e3
    achieved_tflops = iters * fpi / kern_s / 1e12
    achieved_gbs = iters * bpi / kern_s / 1e9
    # the persistent solve kernel the plan picked: one SELL-32 slice per warp
    # (systems up to 31 slices per CTA) or the tiled kernel
    solve_kernel = "cg_sell_kernel" if solver.plan()["slice_solve"] else "cg_solve_kernel"
    tr = ncu_traffic(solve_kernel)
    fp64 = fp64_peak(stream)
    nominal = fp64["sms"] * 2 * 2 * (clk.summary()["sm_max_mhz"] or 2070.0) * 1e6 / 1e12
    # the bytes view of the CG iteration's algorithmic bytes (12 NNZ + 4(N+1) +
    # 88 N per iteration) against the measured HBM copy peak; at this size an
    # iteration's bytes stay in L2, so this is the L2-effective rate, and the
    # DRAM traffic (ncu) is the matrix read once per solve
    roofline = {
        "bound": "hbm", "kernel": solve_kernel, "achieved": round(achieved_gbs, 1),
        "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved_gbs / peaks["hbm_gbs"], 4),
        "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peaks['source']})",
        "traffic": (round(tr["dram_bytes_per_launch"]) if tr else None),
        "algorithmic_bytes_per_launch": iters * bpi, "bytes_per_iteration": bpi,
        "view": "L2-effective: the 53.5 MB an iteration moves stay in the L2",
        "fp64_achieved_tflops": round(achieved_tflops, 4), "fp64_peak_tflops": fp64["tflops"],
        "fp64_frac": round(achieved_tflops / fp64["tflops"], 4),
        "fp64_peak_source": "measured in this run: " + fp64["method"],
        "fp64_peak_nominal_tflops": round(nominal, 4),
        "algorithmic_flops_per_launch": iters * fpi,
    }

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": nnz, "tol": TOL, "iters": iters,
                   "relres_true": relres_true, "l2_flush": "2x L2 buffer written before each solve",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "solve_kernel_ms": round(statistics.mean(kern_ms), 4)},
        "roofline": roofline,
        "gpu_launches": launches,
    }

    # ------------------------------------------------------------- e2e
    bh = torch.from_numpy(pr.b.copy()).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    bn, xn = bh.numpy(), xh.numpy()
    for _ in range(args.warmup):
        xn[:] = 0.0
        solver.solve_host(bn, xn, TOL)
    e2e = []
    for _ in range(args.steps):
        xn[:] = 0.0
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = solver.solve_host(bn, xn, TOL)
        e2e.append((time.perf_counter() - t0) * 1e3)
        assert info.status == gbcg.CG_OK
    line["e2e"] = {"value": round(sum(e2e) / len(e2e), 4), "unit": UNIT,
                   "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n + 40,
                   "api": "cg_solve_host (pinned host b, x)"}
    line["clocks"] = clk.summary()
    solver.close()

    if not args.no_extras:
        # ------------------- CPU baselines: the OpenMP build on all host cores
        # and the serial oracle (whose solution the other forms' errors are
        # reported against)
        x_oracle = None
        if rank == 0 and world == 1:
            import oracle
            r = oracle.cg_omp(pr.A, pr.b, tol=TOL)   # warm-up (thread pool, pages)
            t0 = time.perf_counter()
            r = oracle.cg_omp(pr.A, pr.b, tol=TOL)
            dt = (time.perf_counter() - t0) * 1e3
            assert r["status"] == oracle.OK
            line["cpu_baseline"] = {
                "value": round(dt, 2), "unit": UNIT, "cores": oracle.omp_threads(), "kind": "oracle",
                "build": "OpenMP (row and vector loops over all host cores), beside the serial oracle",
                "sample": f"one full FP64 CG solve of the same system ({r['iters']} iterations)"}
            t0 = time.perf_counter()
            r = oracle.cg(pr.A, pr.b, tol=TOL)
            dt = (time.perf_counter() - t0) * 1e3
            x_oracle = r["x"]
            line["cpu_baseline_serial"] = {
                "value": round(dt, 2), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"one full serial FP64 CG solve of the same system ({r['iters']} iterations)"}
        forms = measure_forms(pr, ms_per_step, iters, max(3, args.steps // 2), x_oracle, flush)
        line["spmv_hbm"] = measure_spmv_hbm(peaks, flush, fp64["tflops"])
        line["roofline"]["spmv_hbm_frac"] = line["spmv_hbm"]["frac"]
        line["roofline"]["spmv_hbm_gbs"] = line["spmv_hbm"]["achieved"]
        line["forms_100cube"] = measure_forms_100cube(flush, fp64["tflops"])
        line["batched"] = measure_batched(256, 20, 80, 1, tune_sys=32, sample=2)
        line["learned"] = measure_learned()
        lf = line["learned"]["q1_50cube_c2"]["learned_fcg"]
        forms["learned_fcg"] = {"ms_per_solve": lf["ms_per_solve"], "iters": lf["iters"],
                                "relres_true": lf["relres_true"], "reverted_at": lf["reverted_at"],
                                "speedup_vs_fp64_cg": round(ms_per_step / lf["ms_per_solve"], 3)}
        line["forms"] = forms
        line["gpu_launches"] += 0  # extras are outside the timed region

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.section or args.batched_full or args.learned_only:
        run_section(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gbcg(args)


if __name__ == "__main__":
    main()
