"""Pins for the sparse oracle (oracle/sparse.py): dense matrix products, exact
termination and conjugacy of CG, scipy's CG, and the true residual."""
import numpy as np
import pytest

from oracle import sparse as osp
from paper_1304_5553_gb300 import inputs


def _dense(rowptr, col, val, n, m):
    A = np.zeros((n, m))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            A[i, col[k]] += val[k]
    return A


def test_spmv_is_the_dense_product():
    for seed, empty in ((1, 0), (2, 5)):
        rp, c, v = inputs.random_spd(200, seed, max_degree=40, empty_every=empty)
        x = np.random.default_rng(seed).standard_normal(200)
        A = _dense(rp, c, v, 200, 200)
        y, ab = osp.spmv(rp, c, v, x)
        assert np.allclose(y, A @ x, rtol=1e-13, atol=1e-13)
        assert np.allclose(ab, np.abs(A) @ np.abs(x), rtol=1e-13, atol=1e-13)  # no duplicates
        assert np.all(ab >= np.abs(y) - 1e-12)
        if empty:
            assert np.all(y[::empty] == 0) and np.all(ab[::empty] == 0)


def test_cg_terminates_in_n_steps_and_directions_are_conjugate():
    n = 40
    rp, c, v = inputs.random_spd(n, 3, max_degree=10)
    A = _dense(rp, c, v, n, n)
    b = np.random.default_rng(4).standard_normal(n)
    x, k, hist, dirs = osp.cg(rp, c, v, b, np.zeros(n), 1e-12, 10 * n, directions=True)
    assert k <= n
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    P = np.array(dirs[:-1])
    G = P @ A @ P.T
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) <= 1e-8 * np.max(np.abs(np.diag(G)))
    # the recurrence's residual is the true residual
    assert abs(hist[-1] - np.linalg.norm(b - A @ x)) <= 1e-9 * np.linalg.norm(b)


def test_cg_matches_scipy():
    sla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    rp, c, v = inputs.poisson2d(48, 40, np.float64)
    n = 48 * 40
    A = sp.csr_matrix((v, c, rp), shape=(n, n))
    b = np.random.default_rng(5).standard_normal(n)
    x, k, hist = osp.cg(rp, c, v, b, np.zeros(n), 1e-8, 5000)
    steps = []
    xs, info = sla.cg(A, b, x0=np.zeros(n), rtol=1e-8, atol=0.0, maxiter=5000,
                      callback=lambda xk: steps.append(1))
    assert info == 0 and abs(len(steps) - k) <= 1
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.001


def test_cg_edge_cases():
    rp, c, v = inputs.poisson2d(8, 8, np.float64)
    n = 64
    x, k, _ = osp.cg(rp, c, v, np.zeros(n), np.zeros(n), 1e-6, 100)
    assert k == 0 and np.all(x == 0)
    xs, _, _ = osp.cg(rp, c, v, np.ones(n), np.zeros(n), 1e-14, 1000)
    x, k, _ = osp.cg(rp, c, v, np.ones(n), xs, 1e-6, 100)   # already solved
    assert k == 0
    x, k, hist = osp.cg(rp, c, v, np.ones(n), np.zeros(n), 1e-14, 3)
    assert k == 3 and len(hist) == 4


def _rank_one_plus_identity(n, seed):
    """A = I + u u^T (dense pattern, CSR): eigenvalues 1 (n - 1 times) and 1 + |u|^2."""
    u = np.random.default_rng(seed).standard_normal(n)
    A = np.eye(n) + np.outer(u, u)
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    c = np.tile(np.arange(n, dtype=np.int32), n)
    return rp, c, A.ravel(), A


def test_cg_two_eigenvalues_two_steps():
    """CG's residual polynomial of degree k can vanish on k distinct eigenvalues, so a
    matrix with two of them is solved in two steps (to rounding); one step is not
    enough unless b happens to be an eigenvector."""
    n = 60
    rp, c, v, A = _rank_one_plus_identity(n, 7)
    b = np.random.default_rng(8).standard_normal(n)
    x, k, hist = osp.cg(rp, c, v, b, np.zeros(n), 1e-12, 50)
    assert k == 2
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    assert hist[1] > 1e-3 * hist[0]
