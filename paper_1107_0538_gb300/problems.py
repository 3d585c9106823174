"""Seeded synthetic inputs: Q1 hexahedral FEM matrices in CSR and right-hand sides.

The case study of the paper (Section IV) solves a CSR system that comes from
a finite-element model of an electrical machine, with N = 132651 unknowns and
NNZ = 3442951 stored entries (Section IV; Table I caption).  That matrix is
not published, so every workload here is generated instead:

* the stiffness matrix of -div(nu grad u) discretised with trilinear (Q1)
  hexahedral elements on a box of Ex x Ey x Ez cubic elements of side h,
  plus a shift of 1e-2 times the lumped mass matrix, so every node is a free
  unknown and the matrix is symmetric positive definite;
* the CSR pattern holds every pair of nodes that share an element, explicit
  zeros included (the edge-neighbour couplings of a cube are exactly zero),
  so NNZ = (3Ex+1)(3Ey+1)(3Ez+1).  A 50^3-element cube gives N = 51^3 =
  132651 and NNZ = 151^3 = 3442951, the paper's sizes exactly;
* nu is either 1 everywhere or an "air" background at 1 with seeded random
  axis-aligned ellipsoidal "iron" blobs at a lower value (contrast 1e3);
* right-hand sides are seeded uniform[-1, 1] vectors or b = A x* for a seeded
  smooth x*.

Nodes are numbered x-fastest: node(i, j, k) = i + (Ex+1) (j + (Ey+1) k);
element (i, j, k) has its lower corner at node (i, j, k).  Every random draw
comes from splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based stream: draw t of the
stream with seed s is mix(s + (t + 1) * 0x9E3779B97F4A7C15).

This module is input generation only: it holds none of the solver's
arithmetic and imports neither the CUDA library nor the oracle.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Q1 element stiffness of -laplace on the unit cube, indexed by how many
# coordinates the two local vertices differ in (0: same vertex, 1: edge,
# 2: face diagonal, 3: body diagonal).  For a cube of side h the entries are h
# times these values.
Q1_UNIT_STIFFNESS = (1.0 / 3.0, 0.0, -1.0 / 12.0, -1.0 / 12.0)


# ---------------------------------------------------------------- random draws

def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the splitmix64 stream with this seed."""
    t = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + t * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal variates by the Box-Muller transform of draw pairs."""
    u = uniform01(seed, 2 * count, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------- CSR

@dataclasses.dataclass
class CSR:
    """A square CSR matrix: int32 row pointers and column indices, FP64 values."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if self.n > 0 else 0

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(d, (rows, self.colidx), self.vals)
        return d


@dataclasses.dataclass
class Grid:
    """Element counts of a box mesh and the element side h."""
    ex: int
    ey: int
    ez: int
    h: float

    @property
    def nodes(self) -> tuple[int, int, int]:
        return self.ex + 1, self.ey + 1, self.ez + 1

    @property
    def n(self) -> int:
        nx, ny, nz = self.nodes
        return nx * ny * nz

    def node_coords(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Coordinates of all nodes, each an array of shape (nz, ny, nx)."""
        nx, ny, nz = self.nodes
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return x * self.h, y * self.h, z * self.h


def _shared_choices(d: int) -> tuple[int, ...]:
    # Element offsets (relative to the first node) along one axis of the
    # elements that contain both a node and its neighbour at offset d.
    return {1: (0,), -1: (-1,), 0: (-1, 0)}[d]


def q1_matrix(nu: np.ndarray, h: float, shift: float = 1e-2) -> tuple[CSR, np.ndarray]:
    """Assemble A = K(nu) + shift * M_L on the element field nu[k, j, i].

    K is the Q1 stiffness of -div(nu grad u) with natural boundary conditions,
    M_L the lumped mass matrix (h^3 / 8 per element corner).  Entry (a, b) for
    nodes that share elements is h * Q1_UNIT_STIFFNESS[#differing coordinates]
    times the sum of nu over the shared elements; the sum always runs over the
    shared elements in the same order, so A is bitwise symmetric.
    Returns (A, lumped mass diagonal).
    """
    nu = np.asarray(nu, dtype=np.float64)
    ez, ey, ex = nu.shape
    nz, ny, nx = ez + 1, ey + 1, ex + 1
    n = nx * ny * nz
    pad = np.zeros((ez + 2, ey + 2, ex + 2))
    pad[1:-1, 1:-1, 1:-1] = nu
    ones = np.zeros_like(pad)
    ones[1:-1, 1:-1, 1:-1] = 1.0

    def shared_sum(field, dz, dy, dx):
        acc = None
        for sz in _shared_choices(dz):
            for sy in _shared_choices(dy):
                for sx in _shared_choices(dx):
                    part = field[1 + sz:1 + sz + nz, 1 + sy:1 + sy + ny, 1 + sx:1 + sx + nx]
                    acc = part.copy() if acc is None else acc + part
        return acc

    count = shared_sum(ones, 0, 0, 0)          # elements touching each node
    mass = (h ** 3 / 8.0) * count.reshape(-1)

    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    node = (ii + nx * (jj + ny * kk)).reshape(-1)
    offsets = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    vals2 = np.empty((n, 27))
    cols2 = np.empty((n, 27), dtype=np.int64)
    mask2 = np.empty((n, 27), dtype=bool)
    for t, (dz, dy, dx) in enumerate(offsets):
        nd = abs(dz) + abs(dy) + abs(dx)
        inside = ((kk + dz >= 0) & (kk + dz < nz) & (jj + dy >= 0) & (jj + dy < ny)
                  & (ii + dx >= 0) & (ii + dx < nx)).reshape(-1)
        v = (h * Q1_UNIT_STIFFNESS[nd]) * shared_sum(pad, dz, dy, dx).reshape(-1)
        if nd == 0:
            v = v + shift * mass
        vals2[:, t] = v
        cols2[:, t] = node + dx + nx * (dy + ny * dz)
        mask2[:, t] = inside
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask2.sum(axis=1), out=rowptr[1:])
    A = CSR(n=n, rowptr=rowptr.astype(np.int32), colidx=cols2[mask2].astype(np.int32),
            vals=vals2[mask2].astype(np.float64))
    return A, mass


def q1_nnz(ex: int, ey: int, ez: int) -> int:
    """Stored entries of the Q1 pattern: (3Ex+1)(3Ey+1)(3Ez+1)."""
    return (3 * ex + 1) * (3 * ey + 1) * (3 * ez + 1)


# ------------------------------------------------------------------ nu fields

def nu_uniform(ex: int, ey: int, ez: int, value: float = 1.0) -> np.ndarray:
    return np.full((ez, ey, ex), float(value))


def nu_blobs(grid: Grid, seed: int = 1, nblobs: int = 8, nu_iron: float = 1e-3,
             nu_air: float = 1.0) -> np.ndarray:
    """Air background with seeded axis-aligned ellipsoidal iron blobs.

    Blob m takes draws 6m .. 6m+5 of the stream: centre = 0.2 + 0.6 u on each
    axis, semi-axis = 0.05 + 0.15 u on each axis (unit-cube coordinates scaled
    by the box extent).  An element is iron when its centroid lies inside any
    blob.
    """
    u = uniform01(seed, 6 * nblobs).reshape(nblobs, 6)
    nx, ny, nz = grid.ex, grid.ey, grid.ez
    ext = np.array([nx * grid.h, ny * grid.h, nz * grid.h])
    kc, jc, ic = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = (ic + 0.5) * grid.h, (jc + 0.5) * grid.h, (kc + 0.5) * grid.h
    iron = np.zeros((nz, ny, nx), dtype=bool)
    for m in range(nblobs):
        c = (0.2 + 0.6 * u[m, 0:3]) * ext
        a = (0.05 + 0.15 * u[m, 3:6]) * ext
        s = ((cx - c[0]) / a[0]) ** 2 + ((cy - c[1]) / a[1]) ** 2 + ((cz - c[2]) / a[2]) ** 2
        iron |= s <= 1.0
    return np.where(iron, nu_iron, nu_air)


# ------------------------------------------------------------------------ RHS

def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """b_i = 2 u_i - 1 with u from the splitmix64 stream of this seed."""
    return 2.0 * uniform01(seed, n) - 1.0


def smooth_solution(grid: Grid, seed: int = 2, offset: float = 0.1) -> np.ndarray:
    """x*(x,y,z) = sum_{k in {1,2,3}^3} c_k sin(k1 pi x') sin(k2 pi y') sin(k3 pi z') + offset.

    c_k ~ N(0,1) / |k|^2 from the stream of this seed (k in lexicographic
    order), and x', y', z' are the node coordinates scaled to [0, 1].
    """
    x, y, z = grid.node_coords()
    x = x / max(grid.ex * grid.h, 1e-300)
    y = y / max(grid.ey * grid.h, 1e-300)
    z = z / max(grid.ez * grid.h, 1e-300)
    ks = [(a, b, c) for a in (1, 2, 3) for b in (1, 2, 3) for c in (1, 2, 3)]
    coef = normal(seed, len(ks))
    out = np.full(x.shape, offset)
    for (k1, k2, k3), cn in zip(ks, coef):
        w = cn / float(k1 * k1 + k2 * k2 + k3 * k3)
        out = out + w * np.sin(k1 * math.pi * x) * np.sin(k2 * math.pi * y) * np.sin(k3 * math.pi * z)
    return out.reshape(-1)


def csr_times(A: CSR, x: np.ndarray) -> np.ndarray:
    """A x for building b = A x* (input preparation, vectorised numpy)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return np.bincount(rows, weights=A.vals * x[A.colidx], minlength=A.n)


# ----------------------------------------------------------------- workloads

@dataclasses.dataclass
class Problem:
    name: str
    grid: Grid
    A: CSR
    b: np.ndarray
    xstar: np.ndarray | None
    tol: float
    mass: np.ndarray
    nu: np.ndarray


def cube_uniform(e: int = 20, seed: int = 0) -> Problem:
    """Q1 cube of e^3 elements, nu = 1, h = 1/e, RHS uniform[-1, 1] (seed 0), tol 1e-10."""
    g = Grid(e, e, e, 1.0 / e)
    nu = nu_uniform(e, e, e)
    A, mass = q1_matrix(nu, g.h)
    return Problem(f"q1-{e}^3-uniform", g, A, rhs_uniform(A.n, seed), None, 1e-10, mass, nu)


def cube_blobs(e: int = 50, blob_seed: int = 1, x_seed: int = 2, contrast: float = 1e3,
               tol: float = 1e-8) -> Problem:
    """Q1 cube of e^3 elements, iron blobs at nu = 1/contrast, b = A x* for a smooth x*."""
    g = Grid(e, e, e, 1.0 / e)
    nu = nu_blobs(g, seed=blob_seed, nu_iron=1.0 / contrast)
    A, mass = q1_matrix(nu, g.h)
    xs = smooth_solution(g, seed=x_seed)
    return Problem(f"q1-{e}^3-blobs-c{contrast:g}", g, A, csr_times(A, xs), xs, tol, mass, nu)


def source_currents(grid: Grid, mass: np.ndarray, seed: int, nsteps: int = 4, ncoils: int = 3) -> np.ndarray:
    """Right-hand sides of time-stepped source currents, shape (nsteps, n).

    Coil c is an axis-aligned box (corner U[0.1, 0.6]^3, size U[0.1, 0.4]^3 of
    the box extent) with amplitude U[0.5, 2] and phase U[0, 2 pi), 8 draws of
    the stream of `seed`; at step s the current density is
    J = sum_c amp_c sin(2 pi s / nsteps + phase_c) 1[node in coil c] and the
    right-hand side is b = M_L J (lumped mass).
    """
    u = uniform01(seed, 8 * ncoils).reshape(ncoils, 8)
    x, y, z = grid.node_coords()
    ext = np.array([grid.ex * grid.h, grid.ey * grid.h, grid.ez * grid.h])
    out = np.zeros((nsteps, grid.n))
    for c in range(ncoils):
        lo = (0.1 + 0.5 * u[c, 0:3]) * ext
        hi = lo + (0.1 + 0.3 * u[c, 3:6]) * ext
        amp = 0.5 + 1.5 * u[c, 6]
        phase = 2.0 * math.pi * u[c, 7]
        inside = ((x >= lo[0]) & (x <= hi[0]) & (y >= lo[1]) & (y <= hi[1]) & (z >= lo[2]) & (z <= hi[2]))
        inside = inside.reshape(-1).astype(np.float64)
        for s in range(nsteps):
            out[s] += amp * math.sin(2.0 * math.pi * s / nsteps + phase) * inside
    return out * mass[None, :]


def batch_systems(nsys: int, emin: int = 20, emax: int = 80, seed0: int = 1000, nrhs: int = 4):
    """Independent systems of uneven Q1 boxes for batched solves.

    System i uses seed s = seed0 + i: draws 0-2 of that stream give the
    element counts Ex, Ey, Ez ~ U{emin..emax}, draw 3 the contrast
    (log-uniform on [1e2, 1e4]; iron at nu = 1 / contrast); the iron blobs use
    the stream of seed 10 s + 1 and the source currents (nrhs time steps) the
    stream of seed 10 s + 2; h = 1 / max(Ex, Ey, Ez).  Returns a list of dicts
    with A, B (nrhs x n), grid, mass and contrast.
    """
    out = []
    for i in range(nsys):
        s = seed0 + i
        u = uniform01(s, 4)
        ex, ey, ez = (emin + np.minimum((u[:3] * (emax - emin + 1)).astype(int), emax - emin)).tolist()
        contrast = 10.0 ** (2.0 + 2.0 * u[3])
        g = Grid(int(ex), int(ey), int(ez), 1.0 / max(ex, ey, ez))
        nu = nu_blobs(g, seed=10 * s + 1, nu_iron=1.0 / contrast)
        A, mass = q1_matrix(nu, g.h)
        B = source_currents(g, mass, seed=10 * s + 2, nsteps=nrhs)
        out.append({"A": A, "B": B, "grid": g, "mass": mass, "contrast": contrast})
    return out


def node_log_nu(grid: Grid, nu: np.ndarray) -> np.ndarray:
    """log nu at the nodes: the mean of log nu over the (1 to 8) elements that
    share each node, node order x fastest (float64, length n).  This is the
    second input field of the learned preconditioner."""
    ex, ey, ez = grid.ex, grid.ey, grid.ez
    ln = np.log(np.asarray(nu, dtype=np.float64)).reshape(ez, ey, ex)
    acc = np.zeros((ez + 1, ey + 1, ex + 1))
    cnt = np.zeros_like(acc)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                acc[dz:dz + ez, dy:dy + ey, dx:dx + ex] += ln
                cnt[dz:dz + ez, dy:dy + ey, dx:dx + ex] += 1.0
    return (acc / cnt).reshape(-1)


LEARN_PARAMS = 7792  # W1 16x27, W2 16x16x27, Wg 16x27, bg 16


def bf16_representable(v: np.ndarray) -> np.ndarray:
    """Round float values to the nearest BF16 (ties to even), returned as float32."""
    f = np.asarray(v, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def learn_init_params(seed: int = 7, noise: float = 0.01, gate_bias: float = 2.0) -> np.ndarray:
    """Initial parameters of the learned preconditioner (float32, BF16-representable).

    W1 and W2 start at the identity on the centre tap (channel 0 of W1, the
    diagonal of W2) plus noise * N(0, 1) from the splitmix64 stream of ``seed``;
    the gate convolution starts at zero and its bias at ``gate_bias``, so the
    untrained preconditioner is sigmoid(gate_bias)^2 D^-1 plus small noise."""
    ch, ntap, centre = 16, 27, 13
    w1 = np.zeros((ch, ntap))
    w1[0, centre] = 1.0
    w2 = np.zeros((ch, ch, ntap))
    for o in range(ch):
        w2[o, o, centre] = 1.0
    z = normal(seed, w1.size + w2.size)
    w1 += noise * z[:w1.size].reshape(w1.shape)
    w2 += noise * z[w1.size:].reshape(w2.shape)
    wg = np.zeros((ch, ntap))
    bg = np.full(ch, gate_bias)
    theta = np.concatenate([w1.ravel(), w2.ravel(), wg.ravel(), bg])
    assert theta.size == LEARN_PARAMS
    return bf16_representable(theta)


@dataclasses.dataclass
class LearnInstance:
    name: str
    grid: Grid
    A: CSR
    b: np.ndarray
    xstar: np.ndarray
    lognu: np.ndarray


def learn_instance(e: int, seed: int, contrast: float = 1e3) -> LearnInstance:
    """A random-reluctivity instance for the learned preconditioner.

    Q1 cube of e^3 elements (h = 1/e) with iron blobs from the stream of
    ``seed`` at nu = 1/contrast, x* uniform[-1, 1] from the stream of
    seed + 1 and b = A x*, so the true error of any iterate is known.
    Training instances use seeds 10000 and up, test instances 20000 and up."""
    g = Grid(e, e, e, 1.0 / e)
    nu = nu_blobs(g, seed=seed, nu_iron=1.0 / contrast)
    A, _ = q1_matrix(nu, g.h)
    xs = 2.0 * uniform01(seed + 1, A.n) - 1.0
    return LearnInstance(f"q1-{e}^3-blobs-c{contrast:g}-s{seed}", g, A, csr_times(A, xs), xs,
                         node_log_nu(g, nu))


def flops_per_iteration(n: int, nnz: int) -> int:
    """One SpMV (2 NNZ), two dot products (4 N) and three axpys (6 N): 2 NNZ + 10 N."""
    return 2 * nnz + 10 * n
