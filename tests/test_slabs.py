"""Row-slab sharding of CG over ranks (the paper's 2- and 4-GPU runs,
Section V, Table I): the host plan, and the sharded iteration emulated with
gloo ranks on the CPU.

The plan (`slabs.slab_plan`) is checked against the definition of a halo:
the off-slab columns each rank's rows reference, grouped by owner.  The
emulation runs the CG recurrence of Section IV with each rank holding only
its slab.  Before each SpMV the ranks exchange the halo entries of the
gathered vector point-to-point, and the dot products are per-rank partial
sums added by an allreduce.  Its iterates must equal the single-process
oracle's within the parity bar of the GPU tests (rel. 1e-10 at a fixed
iteration count; full solves within +-2 iterations).
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1107_0538_gb300 import problems, slabs

torch = pytest.importorskip("torch")


def _q1(e):
    return problems.q1_matrix(problems.nu_uniform(e, e, e), 1.0 / e)[0]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
def test_plan_covers_rows_and_halos_are_the_off_slab_columns(world):
    A = _q1(6)
    plan = slabs.slab_plan(A.rowptr, A.colidx, world)
    assert plan.row0[0] == 0 and plan.row0[-1] == A.n
    assert np.all(np.diff(plan.row0) >= 1)
    nnz = np.diff(A.rowptr)
    per = [int(nnz[plan.row0[k]:plan.row0[k + 1]].sum()) for k in range(world)]
    assert max(per) - min(per) <= 2 * nnz.max()      # balanced by stored entries
    for k in range(world):
        r0, r1 = plan.rows(k)
        cols = set(A.colidx[A.rowptr[r0]:A.rowptr[r1]].tolist())
        off = sorted(c for c in cols if not r0 <= c < r1)
        assert plan.halo_rows(k).tolist() == off
        for j, rows in plan.recv[k].items():
            a, b = plan.rows(j)
            assert j != k and np.all((rows >= a) & (rows < b))
            assert np.array_equal(plan.send[j][k], rows)


def test_q1_slabs_exchange_with_neighbours_only():
    # x-fastest numbering: a row references at most one node plane (plus a
    # line and a node) on either side, so only adjacent ranks exchange
    e = 12
    A = _q1(e)
    plane = (e + 1) ** 2
    for world in (2, 4):
        plan = slabs.slab_plan(A.rowptr, A.colidx, world)
        for k in range(world):
            assert set(plan.recv[k]) <= {k - 1, k + 1}
            for rows in plan.recv[k].values():
                assert rows.size <= plane + (e + 1) + 1
    # the paper-sized system on 2 ranks: about one 51 x 51 plane each way
    A = problems.q1_matrix(problems.nu_uniform(50, 50, 50), 1.0 / 50)[0]
    plan = slabs.slab_plan(A.rowptr, A.colidx, 2)
    assert 2 * 51 * 51 <= plan.exchange_bytes() // 8 <= 2 * (51 * 51 + 52)


def test_more_ranks_than_rows():
    A = problems.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 2.0]))
    plan = slabs.slab_plan(A.rowptr, A.colidx, 3)
    assert plan.row0[0] == 0 and plan.row0[-1] == 2 and np.all(np.diff(plan.row0) >= 0)
    assert all(not r for r in plan.recv)


# ------------------------------------------- sharded CG on gloo ranks

def _case(name):
    if name == "uniform":
        return problems.cube_uniform(6)
    return problems.cube_blobs(7, contrast=1e2, tol=1e-10)


def _exchange(dist, plan, rank, g):
    """Halo exchange of the gathered vector g (full length; own rows valid)."""
    reqs, bufs = [], {}
    for j, rows in plan.send[rank].items():
        reqs.append(dist.isend(torch.from_numpy(g[rows].copy()), dst=j))
    for j, rows in plan.recv[rank].items():
        bufs[j] = torch.empty(rows.size, dtype=torch.float64)
        reqs.append(dist.irecv(bufs[j], src=j))
    for r in reqs:
        r.wait()
    for j, rows in plan.recv[rank].items():
        g[rows] = bufs[j].numpy()


def _allreduce(dist, *vals):
    t = torch.tensor(vals, dtype=torch.float64)
    dist.all_reduce(t)
    return t.numpy()


def _rank_main(rank, world, port, case, tol, maxit, precond, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = _case(case)
        A = pr.A
        plan = slabs.slab_plan(A.rowptr, A.colidx, world)
        r0, r1 = plan.rows(rank)
        rp = A.rowptr[r0:r1 + 1].astype(np.int64)
        cols, vals = A.colidx[rp[0]:rp[-1]], A.vals[rp[0]:rp[-1]]
        rows = np.repeat(np.arange(r1 - r0), np.diff(rp))
        diag = np.zeros(r1 - r0)
        np.add.at(diag, rows, np.where(cols == rows + r0, vals, 0.0))

        def spmv(g):   # own rows of A g (g valid on own rows and the halo)
            return np.bincount(rows, weights=vals * g[cols], minlength=r1 - r0)

        b = pr.b[r0:r1]
        g = np.zeros(A.n)                      # x0 = 0
        x = np.zeros(r1 - r0)
        _exchange(dist, plan, rank, g)
        r = b - spmv(g)
        z = r / diag if precond else r.copy()
        p = z.copy()
        rho, rr, bb = _allreduce(dist, r @ z, r @ r, b @ b)
        bnorm = np.sqrt(bb)
        k = 0
        while np.sqrt(rr) > tol * bnorm and k < maxit:
            g[r0:r1] = p
            _exchange(dist, plan, rank, g)
            q = spmv(g)
            (pq,) = _allreduce(dist, p @ q)
            alpha = rho / pq
            x += alpha * p
            r -= alpha * q
            z = r / diag if precond else r
            rr, rho_new = _allreduce(dist, r @ r, r @ z)
            k += 1
            if np.sqrt(rr) <= tol * bnorm or k >= maxit:
                break
            p = z + (rho_new / rho) * p
            rho = rho_new
        np.save(os.path.join(out_dir, f"x{rank}.npy"), x)
        np.save(os.path.join(out_dir, f"k{rank}.npy"), np.array([k, r0, r1]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded_cg(tmp_path, world, case, tol, maxit, precond):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), case, tol, maxit, precond, str(tmp_path)),
             nprocs=world, join=True)
    n = _case(case).A.n
    x = np.zeros(n)
    iters = set()
    for rank in range(world):
        k, r0, r1 = np.load(tmp_path / f"k{rank}.npy")
        x[r0:r1] = np.load(tmp_path / f"x{rank}.npy")
        iters.add(int(k))
    assert len(iters) == 1        # every rank took the same decisions
    return x, iters.pop()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precond", [0, 1])
def test_sharded_cg_matches_oracle_iterates(tmp_path, world, precond):
    pr = _case("blobs")
    k = 25
    ref = oracle.cg(pr.A, pr.b, tol=0.0, maxit=k, precond=precond)
    x, iters = _sharded_cg(tmp_path, world, "blobs", 0.0, k, precond)
    assert iters == k == ref["iters"]
    assert _rel(x, ref["x"]) <= 1e-10


def test_sharded_cg_full_solve(tmp_path):
    pr = _case("uniform")
    ref = oracle.cg(pr.A, pr.b, tol=1e-10)
    x, iters = _sharded_cg(tmp_path, 2, "uniform", 1e-10, pr.A.n, 0)
    assert abs(iters - ref["iters"]) <= 2
    assert _rel(x, ref["x"]) <= 1e-8
