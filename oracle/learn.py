"""FP64 oracle of the learned preconditioner and of flexible CG (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; the product path never does, and this module never
imports the product path.  Plain numpy in float64, one readable step per line;
scipy's CSR matrix-vector product is the only library primitive used for A v.

The paper (Section IV) solves A x = b by CG and has no preconditioner beyond
the identity.  This module follows the extension built on top of it:

* The preconditioner.  With D = diag(A), s = D^-1/2 r, sigma = rms(s) and
  s_hat = s / sigma, the network computes
      a1 = C1(s_hat)            1 -> 16 channels, 3x3x3 taps
      h1 = g * a1               g = sigmoid(Cg(lognu / 8) + bg), 16 channels
      h2 = C2(h1)               16 -> 16
      k  = C2^T(h2)             the adjoint of C2 (flipped taps, swapped channels)
      k1 = g * k
      u  = C1^T(k1)             16 -> 1
  and z = sigma D^-1/2 u, i.e. z = D^-1/2 L^T L D^-1/2 r with L = C2 g C1:
  linear in r, symmetric and positive semi-definite by construction.  Every
  convolution is a correlation over the 27 neighbours of a node of the
  (Ex+1) x (Ey+1) x (Ez+1) node grid with zeros outside the grid.
* The loss of one (residual r, error e) pair with A e = r: with
  e_hat = D^1/2 e / sigma (so that A_hat e_hat = s_hat, A_hat = D^-1/2 A D^-1/2),
      loss = (u - e_hat)^T A_hat (u - e_hat) / (2 n),
  the energy-norm error of the network's error estimate; its gradient with
  respect to u is A_hat (u - e_hat) / n.
* Flexible CG (Notay's FCG with one stored direction, equivalently the
  Polak-Ribiere form of Golub and Ye): alpha = rho / (p.q),
  beta = -alpha (z_new . q) / rho, p = z_new + beta p.  A stall (no residual
  norm of the last W = 50 iterations is below 0.9 times the smallest one
  before them) or r.z <= 0 switches the solve, for the rest of it, to
  Jacobi-PCG restarted from the current x.

Parameter vector (float, 7792 entries): W1[o][t] (16 x 27), W2[o][c][t]
(16 x 16 x 27), Wg[o][t] (16 x 27), bg[o] (16).  Tap t = 9 (dz+1) + 3 (dy+1)
+ (dx+1) reads the node at offset (dx, dy, dz).

Parity status: conv (pinned: library correlation), conv_adjoint (pinned:
adjoint identity), apply (pinned: symmetry, linearity, the identity network
reduces to Jacobi), loss_grad (pinned: central finite differences), fcg
(pinned: identity preconditioner reproduces CG, Jacobi reproduces PCG).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

CH = 16
NTAP = 27
LOGNU_SCALE = 0.125
N_W1 = CH * NTAP
N_W2 = CH * CH * NTAP
N_WG = CH * NTAP
N_PARAMS = N_W1 + N_W2 + N_WG + CH
TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]

OK, ENOCONV, EBREAKDOWN, ENAN = 0, 4, 5, 6


def split_params(theta):
    """Views W1 (16,1,27), W2 (16,16,27), Wg (16,1,27), bg (16,) of the flat vector."""
    t = np.asarray(theta, dtype=np.float64)
    assert t.shape == (N_PARAMS,)
    w1 = t[:N_W1].reshape(CH, 1, NTAP)
    w2 = t[N_W1:N_W1 + N_W2].reshape(CH, CH, NTAP)
    wg = t[N_W1 + N_W2:N_W1 + N_W2 + N_WG].reshape(CH, 1, NTAP)
    bg = t[N_W1 + N_W2 + N_WG:]
    return w1, w2, wg, bg


def join_params(w1, w2, wg, bg):
    return np.concatenate([np.ravel(w1), np.ravel(w2), np.ravel(wg), np.ravel(bg)])


def _pad(x):
    c, nz, ny, nx = x.shape
    xp = np.zeros((c, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    return xp


def conv(x, w):
    """y[o, p] = sum_{c, t} w[o, c, t] x[c, p + off(t)], zeros outside the grid.

    x has shape (C, nz, ny, nx) and w (O, C, 27)."""
    c, nz, ny, nx = x.shape
    xp = _pad(x)
    y = np.zeros((w.shape[0], nz, ny, nx))
    for t, (dx, dy, dz) in enumerate(TAPS):
        xs = xp[:, 1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        y += np.einsum("oc,czyx->ozyx", w[:, :, t], xs)
    return y


def conv_adjoint(y, w):
    """The adjoint of ``conv`` with the same weights: x[c, q] = sum_{o, t} w[o, c, t] y[o, q - off(t)]."""
    o, nz, ny, nx = y.shape
    yp = _pad(y)
    x = np.zeros((w.shape[1], nz, ny, nx))
    for t, (dx, dy, dz) in enumerate(TAPS):
        ys = yp[:, 1 - dz:1 - dz + nz, 1 - dy:1 - dy + ny, 1 - dx:1 - dx + nx]
        x += np.einsum("oc,ozyx->czyx", w[:, :, t], ys)
    return x


def weight_grad(dy, x):
    """d/dw of sum(dy * conv(x, w)): G[o, c, t] = sum_p dy[o, p] x[c, p + off(t)]."""
    o, nz, ny, nx = dy.shape
    xp = _pad(x)
    g = np.zeros((o, x.shape[0], NTAP))
    for t, (dx, dy_, dz) in enumerate(TAPS):
        xs = xp[:, 1 + dz:1 + dz + nz, 1 + dy_:1 + dy_ + ny, 1 + dx:1 + dx + nx]
        g[:, :, t] = np.einsum("ozyx,czyx->oc", dy, xs)
    return g


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-v))


def gates(theta, lognu):
    """g = sigmoid(Cg(lognu / 8) + bg) on the node grid, shape (16, nz, ny, nx)."""
    _, _, wg, bg = split_params(theta)
    a = conv(LOGNU_SCALE * lognu[None], wg) + bg[:, None, None, None]
    return sigmoid(a)


def forward(theta, s_hat, lognu):
    """All intermediates of the network for a normalised input s_hat (shape (nz, ny, nx))."""
    w1, w2, _, _ = split_params(theta)
    g = gates(theta, lognu)
    a1 = conv(s_hat[None], w1)
    h1 = g * a1
    h2 = conv(h1, w2)
    k = conv_adjoint(h2, w2)
    k1 = g * k
    u = conv_adjoint(k1, w1)[0]
    return dict(g=g, a1=a1, h1=h1, h2=h2, k=k, k1=k1, u=u)


def scale_input(r, diag):
    """s = D^-1/2 r, sigma = rms(s), s_hat = s / sigma."""
    s = np.asarray(r, dtype=np.float64) / np.sqrt(diag)
    sigma = np.sqrt(np.dot(s, s) / s.size)
    return s, sigma


def apply(theta, r, diag, lognu, shape):
    """z = M r for a residual in node order (x fastest); shape = (nz, ny, nx)."""
    s, sigma = scale_input(r, diag)
    if sigma == 0.0:
        return np.zeros_like(s)
    f = forward(theta, (s / sigma).reshape(shape), lognu.reshape(shape))
    return sigma * f["u"].reshape(-1) / np.sqrt(diag)


def loss_grad(theta, A, diag, lognu, shape, r, e):
    """Energy-norm loss of one pair and its gradient with respect to the parameters.

    A is a scipy CSR matrix (or anything with ``@``); r and e are in node order."""
    w1, w2, wg, bg = split_params(theta)
    n = r.size
    s, sigma = scale_input(r, diag)
    s_hat = (s / sigma).reshape(shape)
    e_hat = (np.sqrt(diag) * e / sigma).reshape(shape)
    f = forward(theta, s_hat, lognu.reshape(shape))
    g = f["g"]
    v = (f["u"] - e_hat).reshape(-1)
    av = (A @ (v / np.sqrt(diag))) / np.sqrt(diag)     # A_hat v
    loss = 0.5 * np.dot(v, av) / n
    du = (av / n).reshape((1,) + tuple(shape))
    # u = C1^T(k1)
    dw1 = weight_grad(f["k1"], du)
    dk1 = conv(du, w1)
    # k1 = g k
    dk = g * dk1
    dg = f["k"] * dk1
    # k = C2^T(h2)
    dw2 = weight_grad(f["h2"], dk)
    dh2 = conv(dk, w2)
    # h2 = C2(h1)
    dw2 += weight_grad(dh2, f["h1"])
    dh1 = conv_adjoint(dh2, w2)
    # h1 = g a1
    da1 = g * dh1
    dg += f["a1"] * dh1
    # a1 = C1(s_hat)
    dw1 += weight_grad(da1, s_hat[None])
    # g = sigmoid(Cg(lognu / 8) + bg)
    dag = dg * g * (1.0 - g)
    dwg = weight_grad(dag, LOGNU_SCALE * lognu.reshape((1,) + tuple(shape)))
    dbg = dag.sum(axis=(1, 2, 3))
    return loss, join_params(dw1, dw2, dwg, dbg)


def batch_loss_grad(theta, samples):
    """Mean loss and gradient over samples = [(A, diag, lognu, shape, r, e), ...]."""
    tot, grad = 0.0, np.zeros(N_PARAMS)
    for A, diag, lognu, shape, r, e in samples:
        l, gr = loss_grad(theta, A, diag, lognu, shape, r, e)
        tot += l
        grad += gr
    return tot / len(samples), grad / len(samples)


def csr_matrix(A):
    """scipy CSR view of a problems.CSR."""
    return sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n))


def diagonal(A):
    """Diagonal of a problems.CSR (duplicates summed)."""
    return csr_matrix(A).diagonal()


def fcg(A, b, precond, tol=1e-8, maxit=0, x0=None, diag=None, stall_window=50, stall_factor=0.9):
    """Flexible CG with the stall switch to Jacobi-PCG.

    ``precond`` maps a residual to z, or is the string "jacobi" or "none".
    Returns dict(x, iters, relres, status, reverted_at) where reverted_at is
    the iteration at which the solve switched to Jacobi (-1: never).
    """
    S = A if sp.issparse(A) else csr_matrix(A)
    n = S.shape[0]
    d = S.diagonal() if diag is None else diag
    jac = lambda v: v / d
    ident = lambda v: v.copy()
    if precond == "jacobi":
        M, learned = jac, False
    elif precond == "none":
        M, learned = ident, False
    else:
        M, learned = precond, True
    maxit = n if maxit <= 0 else maxit
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - S @ x
    bnorm = np.sqrt(np.dot(b, b))
    out = dict(x=x, iters=0, relres=0.0, status=OK, reverted_at=-1)
    if bnorm == 0.0:
        out["x"] = np.zeros(n)
        return out
    hist = [np.sqrt(np.dot(r, r))]
    if hist[0] <= tol * bnorm:
        out["relres"] = hist[0] / bnorm
        return out
    z = M(r)
    rho = np.dot(r, z)
    if learned and not rho > 0.0:
        M, learned, out["reverted_at"] = jac, False, 0
        z = M(r)
        rho = np.dot(r, z)
    p = z.copy()
    mode_start = 0
    for k in range(1, maxit + 1):
        q = S @ p
        pq = np.dot(p, q)
        if not np.isfinite(pq):
            out.update(status=ENAN, iters=k - 1)
            break
        if pq <= 0.0:
            out.update(status=EBREAKDOWN, iters=k - 1)
            break
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        rn = np.sqrt(np.dot(r, r))
        hist.append(rn)
        out["iters"] = k
        if rn <= tol * bnorm:
            break
        if k == maxit:
            out["status"] = ENOCONV
            break
        restart = False
        if (learned and k - mode_start >= stall_window
                and min(hist[k - stall_window + 1:k + 1]) > stall_factor * min(hist[:k - stall_window + 1])):
            restart = True
        else:
            z = M(r)
            rho_new = np.dot(r, z)
            if learned and not rho_new > 0.0:
                restart = True
        if restart:
            M, learned, out["reverted_at"] = jac, False, k
            mode_start = k
            z = M(r)
            rho = np.dot(r, z)
            p = z.copy()
            continue
        if not rho_new > 0.0:
            out["status"] = EBREAKDOWN
            break
        beta = -alpha * np.dot(z, q) / rho
        p = z + beta * p
        rho = rho_new
    out["x"] = x
    out["relres"] = hist[-1] / bnorm
    return out
