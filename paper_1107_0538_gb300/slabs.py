"""Row-slab partition of a CSR system over ranks, with each rank's halo.

The paper runs its CG on 1, 2 and 4 GPUs by splitting the rows equally
between them (Section V, Table I).  This module is the host-side plan of that
split for a sharded solver:

* rank k owns the contiguous rows [row0[k], row0[k+1]), cut so that each rank
  holds about the same number of stored entries.  On a Q1 node grid numbered
  x-fastest a contiguous row range is a slab of z-planes, and its rows
  reference at most one node plane on either side;
* before each SpMV, rank k needs the entries of the gathered vector at the
  columns outside its own rows that its rows reference (its halo), each from
  the rank that owns them.  ``recv[k][j]`` lists those rows for owner j and
  ``send[j][k]`` is the same list seen from the sender;
* every dot product of the iteration is a sum of per-rank partial sums, so
  an iteration costs one halo exchange and two scalar allreduces (p.q and
  r.r; r.z too with Jacobi).

It is planning only: no solver arithmetic, no device code, no oracle.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SlabPlan:
    world: int
    row0: np.ndarray                 # world + 1 row boundaries
    recv: list[dict[int, np.ndarray]]  # recv[k][j]: rows rank k receives from rank j (sorted)
    send: list[dict[int, np.ndarray]]  # send[j][k]: rows rank j sends to rank k (== recv[k][j])

    def rows(self, k: int) -> tuple[int, int]:
        return int(self.row0[k]), int(self.row0[k + 1])

    def halo_rows(self, k: int) -> np.ndarray:
        """Every off-slab row rank k's SpMV reads, sorted."""
        parts = [self.recv[k][j] for j in sorted(self.recv[k])]
        return np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)

    def exchange_bytes(self, itemsize: int = 8) -> int:
        """Bytes all ranks send per halo exchange."""
        return itemsize * sum(int(v.size) for s in self.send for v in s.values())


def balanced_cuts(rowptr: np.ndarray, world: int) -> np.ndarray:
    """Row boundaries that give each of `world` ranks about nnz / world
    stored entries (each rank at least one row when n >= world)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    n = rowptr.size - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    targets = rowptr[-1] * np.arange(1, world) / world
    cuts = np.searchsorted(rowptr, targets, side="left")
    row0 = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    # keep the boundaries strictly increasing where there are enough rows
    for k in range(1, world):
        lo = row0[k - 1] + (1 if n >= world else 0)
        hi = n - (world - k if n >= world else 0)
        row0[k] = min(max(row0[k], lo), hi)
    return row0


def slab_plan(rowptr: np.ndarray, colidx: np.ndarray, world: int) -> SlabPlan:
    """The slab partition and halo lists of a CSR pattern over `world` ranks."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colidx = np.asarray(colidx, dtype=np.int64)
    row0 = balanced_cuts(rowptr, world)
    recv: list[dict[int, np.ndarray]] = []
    for k in range(world):
        r0, r1 = int(row0[k]), int(row0[k + 1])
        cols = np.unique(colidx[rowptr[r0]:rowptr[r1]])
        off = cols[(cols < r0) | (cols >= r1)]
        owner = np.searchsorted(row0, off, side="right") - 1
        recv.append({int(j): off[owner == j] for j in np.unique(owner)})
    send: list[dict[int, np.ndarray]] = [dict() for _ in range(world)]
    for k in range(world):
        for j, rows in recv[k].items():
            send[j][k] = rows
    return SlabPlan(world, row0, recv, send)
