"""Pins of the learned-preconditioner and flexible-CG oracle (CPU only).

Each check compares the oracle with something other than itself: a library
correlation, the adjoint identity, linearity, central finite differences, a
closed form of the loss, or the CG oracle written in C.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import learn as L
from paper_1107_0538_gb300 import problems as P


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_library_correlation():
    x = _rand((2, 4, 5, 6), 1)
    w = _rand((3, 2, 27), 2)
    y = L.conv(x, w)
    for o in range(3):
        ref = np.zeros(x.shape[1:])
        for c in range(2):
            k = np.zeros((3, 3, 3))
            for t, (dx, dy, dz) in enumerate(L.TAPS):
                k[dz + 1, dy + 1, dx + 1] = w[o, c, t]
            ref += ndimage.correlate(x[c], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_conv_adjoint_identity():
    x = _rand((16, 5, 4, 7), 3)
    y = _rand((16, 5, 4, 7), 4)
    w = _rand((16, 16, 27), 5)
    lhs = np.vdot(L.conv(x, w), y)
    rhs = np.vdot(x, L.conv_adjoint(y, w))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) * 100


def test_weight_grad_is_derivative_of_conv():
    x = _rand((2, 4, 3, 5), 6)
    dy = _rand((3, 4, 3, 5), 7)
    v = _rand((3, 2, 27), 8)
    # conv is linear in w: <dy, conv(x, v)> = <weight_grad(dy, x), v>
    assert abs(np.vdot(dy, L.conv(x, v)) - np.vdot(L.weight_grad(dy, x), v)) < 1e-10


def _instance(e=4, seed=10000):
    inst = P.learn_instance(e, seed)
    S = L.csr_matrix(inst.A)
    d = S.diagonal()
    shape = (e + 1, e + 1, e + 1)
    return inst, S, d, shape


def _random_theta(seed):
    rng = np.random.default_rng(seed)
    th = P.learn_init_params(seed=seed, noise=0.3).astype(np.float64)
    th[L.N_W1 + L.N_W2:L.N_W1 + L.N_W2 + L.N_WG] = 0.5 * rng.standard_normal(L.N_WG)
    th[-L.CH:] = rng.standard_normal(L.CH)
    return th


def test_apply_is_symmetric_linear_and_positive():
    inst, S, d, shape = _instance()
    th = _random_theta(11)
    r1, r2 = _rand(inst.A.n, 12), _rand(inst.A.n, 13)
    m1 = L.apply(th, r1, d, inst.lognu, shape)
    m2 = L.apply(th, r2, d, inst.lognu, shape)
    assert abs(np.dot(m1, r2) - np.dot(r1, m2)) <= 1e-12 * np.linalg.norm(m1) * np.linalg.norm(r2)
    assert np.dot(m1, r1) > 0 and np.dot(m2, r2) > 0
    np.testing.assert_allclose(L.apply(th, 2.5 * r1, d, inst.lognu, shape), 2.5 * m1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(L.apply(th, -r1, d, inst.lognu, shape), -m1, rtol=1e-12, atol=1e-14)
    # superposition (linearity in r)
    m12 = L.apply(th, r1 + r2, d, inst.lognu, shape)
    np.testing.assert_allclose(m12, m1 + m2, rtol=1e-10, atol=1e-12 * np.abs(m12).max())


def test_identity_network_is_scaled_jacobi():
    inst, S, d, shape = _instance()
    w1 = np.zeros((16, 1, 27))
    w1[0, 0, 13] = 1.0
    w2 = np.zeros((16, 16, 27))
    for o in range(16):
        w2[o, o, 13] = 1.0
    b = 0.7
    th = L.join_params(w1, w2, np.zeros((16, 1, 27)), np.full(16, b))
    r = _rand(inst.A.n, 14)
    g = 1.0 / (1.0 + np.exp(-b))
    np.testing.assert_allclose(L.apply(th, r, d, inst.lognu, shape), g * g * r / d, rtol=1e-13)


def test_gradient_matches_central_differences():
    inst, S, d, shape = _instance(e=3, seed=10001)
    th = _random_theta(21)
    r = _rand(inst.A.n, 22)
    e = np.linalg.solve(S.toarray(), r)
    loss, grad = L.loss_grad(th, S, d, inst.lognu, shape, r, e)
    assert loss > 0
    rng = np.random.default_rng(23)
    h = 1e-5
    # random directions over the whole vector and over each block separately
    blocks = [slice(0, L.N_W1), slice(L.N_W1, L.N_W1 + L.N_W2),
              slice(L.N_W1 + L.N_W2, L.N_W1 + L.N_W2 + L.N_WG), slice(L.N_PARAMS - L.CH, L.N_PARAMS)]
    for blk in [slice(0, L.N_PARAMS)] + blocks:
        v = np.zeros(L.N_PARAMS)
        v[blk] = rng.standard_normal(v[blk].size)
        lp, _ = L.loss_grad(th + h * v, S, d, inst.lognu, shape, r, e)
        lm, _ = L.loss_grad(th - h * v, S, d, inst.lognu, shape, r, e)
        fd = (lp - lm) / (2 * h)
        an = np.dot(grad, v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * abs(loss)), (blk, fd, an)


def test_loss_of_zero_network_is_half_energy_of_error():
    inst, S, d, shape = _instance(e=3, seed=10002)
    th = np.zeros(L.N_PARAMS)          # W1 = 0, so u = 0
    r = _rand(inst.A.n, 31)
    e = np.linalg.solve(S.toarray(), r)
    loss, grad = L.loss_grad(th, S, d, inst.lognu, shape, r, e)
    s, sigma = L.scale_input(r, d)
    # u = 0: loss = e_hat^T A_hat e_hat / 2n = e^T r / (2 n sigma^2)
    assert abs(loss - np.dot(e, r) / (2 * r.size * sigma ** 2)) <= 1e-12 * loss
    # and the loss is invariant under r, e -> c r, c e
    l2, _ = L.loss_grad(th, S, d, inst.lognu, shape, 3.0 * r, 3.0 * e)
    assert abs(l2 - loss) <= 1e-12 * loss


@pytest.fixture(scope="module")
def c1_small():
    return P.cube_uniform(6)


def test_fcg_identity_reproduces_cg(c1_small):
    pr = c1_small
    ref = oracle.cg(pr.A, pr.b, tol=1e-10)
    out = L.fcg(pr.A, pr.b, lambda v: v.copy(), tol=1e-10)
    assert out["status"] == L.OK and out["reverted_at"] == -1
    assert abs(out["iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(out["x"] - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


def test_fcg_jacobi_reproduces_pcg():
    pr = P.cube_blobs(8, contrast=1e2, tol=1e-10)
    d = L.diagonal(pr.A)
    ref = oracle.cg(pr.A, pr.b, tol=1e-10, precond=1)
    for pre in ("jacobi", lambda v: v / d):
        out = L.fcg(pr.A, pr.b, pre, tol=1e-10)
        assert out["status"] == L.OK
        assert abs(out["iters"] - ref["iters"]) <= 2
        assert np.linalg.norm(out["x"] - ref["x"]) <= 1e-9 * np.linalg.norm(ref["x"])


def test_fcg_reverts_on_nonpositive_and_on_stall():
    pr = P.cube_blobs(8, contrast=1e2, tol=1e-10)
    d = L.diagonal(pr.A)
    jac = L.fcg(pr.A, pr.b, "jacobi", tol=1e-10)
    neg = L.fcg(pr.A, pr.b, lambda v: -v / d, tol=1e-10)     # r.z < 0 at once
    assert neg["reverted_at"] == 0 and neg["status"] == L.OK
    assert neg["iters"] == jac["iters"]
    np.testing.assert_allclose(neg["x"], jac["x"], rtol=0, atol=1e-12 * np.abs(jac["x"]).max())
    w = _rand(pr.A.n, 41)

    def useless(v):  # positive (r.z = 1e-6 |r|^2) but nearly orthogonal to r
        return 1e-6 * v + np.linalg.norm(v) * (w - np.dot(w, v) / np.dot(v, v) * v)
    st = L.fcg(pr.A, pr.b, useless, tol=1e-10)
    assert st["reverted_at"] >= 50 and st["status"] == L.OK
    true = np.linalg.norm(pr.b - P.csr_times(pr.A, st["x"])) / np.linalg.norm(pr.b)
    assert st["relres"] <= 1e-10 and true <= 1e-9
