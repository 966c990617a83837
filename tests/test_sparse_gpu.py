"""CSR matrix-vector products and the CG solver on the GPU (Sec. 3.2.6),
against the binary64 sparse oracle."""
import numpy as np
import pytest
import torch

from oracle import sparse as osp
from paper_1304_5553_gb300 import inputs, pyc

pytestmark = pytest.mark.gpu

U = {pyc.PYC_F32: 2.0 ** -24, pyc.PYC_F64: 2.0 ** -53}
NP = {pyc.PYC_F32: np.float32, pyc.PYC_F64: np.float64}


class Mat:
    def __init__(self, rp, c, v, n, vt):
        self.rp, self.c, self.v, self.n, self.vt = rp, c, v.astype(NP[vt]), n, vt
        self.d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rp, c, self.v)]
        self.h = pyc.pyc_csr_create(n, n, c.size, *(t.data_ptr() for t in self.d), vt)

    def vec(self, a):
        return torch.from_numpy(np.ascontiguousarray(a, NP[self.vt])).cuda()

    def __del__(self):
        pyc.pyc_csr_destroy(self.h)


def _mixed(n, seed):
    """Rows of 3 entries, every 7th empty, and a band of 40-entry rows."""
    rng = np.random.default_rng(seed)
    deg = np.full(n, 3, np.int64)
    deg[2560:3840] = 40
    deg[::7] = 0
    rp = np.r_[0, np.cumsum(deg)].astype(np.int64)
    c = rng.integers(0, n, rp[-1]).astype(np.int32)
    v = rng.uniform(-1, 1, rp[-1])
    return rp, c, v


def _padding_over_limit(rp):
    """True if slices of 32 rows padded to their longest row would hold more than
    2 nnz + 32 entries per slice (the tuner's limit for the sliced copy)."""
    n = rp.size - 1
    nch = (n + 31) // 32
    d = np.zeros(nch * 32, np.int64)
    d[:n] = np.diff(rp)
    return 32 * d.reshape(nch, 32).max(1).sum() > 2 * rp[-1] + 32 * nch


def _matrices(vt):
    return [Mat(*inputs.poisson2d(300, 200), 60000, vt),
            Mat(*inputs.random_spd(50000, 7, max_degree=2000, empty_every=11), 50000, vt),
            Mat(*_mixed(20011, 17), 20011, vt)]


@pytest.mark.parametrize("vt", [pyc.PYC_F32, pyc.PYC_F64])
def test_spmv_every_width_within_bound(vt):
    s = torch.cuda.current_stream().cuda_stream
    for m in _matrices(vt):
        x = np.random.default_rng(90).uniform(-1, 1, m.n).astype(NP[vt])
        dx = m.vec(x)
        dy = torch.empty(m.n, dtype=dx.dtype, device="cuda")
        y64, ab = osp.spmv(m.rp, m.c, m.v, x)
        length = np.diff(m.rp)
        got = {}
        for w in (0, 1, 2, 4, 8, 16, 32):
            pyc.pyc_csr_set_width(m.h, w)
            dy.fill_(np.nan)
            pyc.pyc_spmv(m.h, dx.data_ptr(), dy.data_ptr(), s)
            got[w] = dy.cpu().numpy()
            y = got[w].astype(np.float64)
            # a row is folded in at most len + 5 steps (lane runs, then a 5-level tree)
            assert np.all(np.abs(y - y64) <= (length + 6) * U[vt] * ab), w
        # the sliced copy adds each row in entry order, as one lane per row does
        assert np.array_equal(got[0], got[1])
        pyc.pyc_spmv_autotune(m.h, dx.data_ptr(), dy.data_ptr(), s)
        assert pyc.pyc_csr_width(m.h) in (0, 1, 2, 4, 8, 16, 32)
        if _padding_over_limit(m.rp):   # the tuner does not try the sliced copy
            assert pyc.pyc_csr_width(m.h) != 0


def test_sliced_copy_is_a_snapshot():
    """Width 0 multiplies by the matrix as it was when the width was set; setting
    it again takes the caller's current values.  Row lengths wider than a byte
    (a 300-entry row) take the 2-byte length table."""
    s = torch.cuda.current_stream().cuda_stream
    rp, c, v = _mixed(5003, 21)
    deg = np.diff(rp)
    deg[100] = 300
    rp = np.r_[0, np.cumsum(deg)].astype(np.int64)
    rng = np.random.default_rng(22)
    c = rng.integers(0, 5003, rp[-1]).astype(np.int32)
    v = rng.uniform(-1, 1, rp[-1])
    m = Mat(rp, c, v, 5003, pyc.PYC_F64)
    x = rng.uniform(-1, 1, 5003)
    dx = m.vec(x)
    dy = torch.empty(5003, dtype=torch.float64, device="cuda")
    pyc.pyc_csr_set_width(m.h, 1)
    pyc.pyc_spmv(m.h, dx.data_ptr(), dy.data_ptr(), s)
    y1 = dy.cpu().numpy()
    pyc.pyc_csr_set_width(m.h, 0)
    pyc.pyc_spmv(m.h, dx.data_ptr(), dy.data_ptr(), s)
    assert np.array_equal(dy.cpu().numpy(), y1)
    m.d[2].mul_(2.0)      # the caller changes its values
    pyc.pyc_spmv(m.h, dx.data_ptr(), dy.data_ptr(), s)
    assert np.array_equal(dy.cpu().numpy(), y1)   # the snapshot
    pyc.pyc_csr_set_width(m.h, 0)
    pyc.pyc_spmv(m.h, dx.data_ptr(), dy.data_ptr(), s)
    assert np.array_equal(dy.cpu().numpy(), 2.0 * y1)   # exact: a power of two


def _true_residual(m, b, x):
    return np.linalg.norm(b.astype(np.float64) - osp.spmv(m.rp, m.c, m.v, x)[0])


@pytest.mark.parametrize("width", [None, 0])
def test_cg_f64_matches_the_oracle(width):
    s = torch.cuda.current_stream().cuda_stream
    rp, c, v = inputs.poisson2d(64, 64, np.float64)
    m = Mat(rp, c, v, 4096, pyc.PYC_F64)
    if width is not None:
        pyc.pyc_csr_set_width(m.h, width)
    b = np.random.default_rng(91).standard_normal(4096)
    db, dx = m.vec(b), m.vec(np.zeros(4096))
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), dx.data_ptr(), 1e-8, 5000, s)
    x = dx.cpu().numpy()
    xo, k, hist = osp.cg(rp, c, v, b, np.zeros(4096), 1e-8, 5000)
    assert info["converged"] and abs(info["iterations"] - k) <= 2, (info, k)
    assert _true_residual(m, b, x) <= 1e-8 * np.linalg.norm(b) * 1.01
    assert abs(info["residual"] - hist[min(info["iterations"], len(hist) - 1)] /
               np.linalg.norm(b)) <= 1e-9


def test_cg_f32_and_irregular():
    s = torch.cuda.current_stream().cuda_stream
    rp, c, v = inputs.poisson2d(256, 256, np.float32)
    m = Mat(rp, c, v, 65536, pyc.PYC_F32)
    b = np.random.default_rng(92).uniform(-1, 1, 65536).astype(np.float32)
    db, dx = m.vec(b), m.vec(np.zeros(65536))
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), dx.data_ptr(), 1e-4, 20000, s)
    _, k, _ = osp.cg(rp, c, v.astype(np.float64), b, np.zeros(65536), 1e-4, 20000)
    assert info["converged"] and 0.8 * k <= info["iterations"] <= 1.25 * k, (info, k)
    assert _true_residual(m, b, dx.cpu().numpy()) <= 2e-4 * np.linalg.norm(b.astype(np.float64))
    # irregular rows (log-uniform degrees up to 300), binary64
    rp, c, v = inputs.random_spd(30000, 8, max_degree=300)
    m2 = Mat(rp, c, v, 30000, pyc.PYC_F64)
    pyc.pyc_csr_set_width(m2.h, 0)   # the sliced copy (slices padded to 300-entry rows)
    b2 = np.random.default_rng(93).standard_normal(30000)
    db2, dx2 = m2.vec(b2), m2.vec(np.zeros(30000))
    info2 = pyc.pyc_cg_solve(m2.h, db2.data_ptr(), dx2.data_ptr(), 1e-10, 1000, s)
    _, k2, _ = osp.cg(rp, c, v, b2, np.zeros(30000), 1e-10, 1000)
    assert info2["converged"] and abs(info2["iterations"] - k2) <= 2
    assert _true_residual(m2, b2, dx2.cpu().numpy()) <= 1e-10 * np.linalg.norm(b2) * 1.01


@pytest.mark.parametrize("width", [1, 0])
def test_cg_two_eigenvalues_two_steps(width):
    """A = I + u u^T has two distinct eigenvalues: CG solves it in two steps."""
    n = 60
    u = np.random.default_rng(7).standard_normal(n)
    A = np.eye(n) + np.outer(u, u)
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    c = np.tile(np.arange(n, dtype=np.int32), n)
    m = Mat(rp, c, A.ravel(), n, pyc.PYC_F64)
    pyc.pyc_csr_set_width(m.h, width)
    b = np.random.default_rng(8).standard_normal(n)
    db, dx = m.vec(b), m.vec(np.zeros(n))
    s = torch.cuda.current_stream().cuda_stream
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), dx.data_ptr(), 1e-12, 50, s)
    assert info["converged"] and info["iterations"] == 2
    assert np.allclose(dx.cpu().numpy(), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_cg_edge_cases():
    s = torch.cuda.current_stream().cuda_stream
    rp, c, v = inputs.poisson2d(32, 32, np.float64)
    m = Mat(rp, c, v, 1024, pyc.PYC_F64)
    zero = m.vec(np.zeros(1024))
    dx = m.vec(np.zeros(1024))
    info = pyc.pyc_cg_solve(m.h, zero.data_ptr(), dx.data_ptr(), 1e-6, 100, s)
    assert info["iterations"] == 0 and info["converged"] and not dx.any().item()
    b = np.ones(1024)
    xs, _, _ = osp.cg(rp, c, v, b, np.zeros(1024), 1e-13, 5000)
    db, dx = m.vec(b), m.vec(xs)
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), dx.data_ptr(), 1e-6, 100, s)  # already solved
    assert info["iterations"] == 0 and info["converged"]
    # x not 16-byte aligned (an offset view): the element-wise update kernel
    buf = m.vec(np.zeros(1025))
    xv = buf[1:]
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), xv.data_ptr(), 1e-9, 5000, s)
    assert info["converged"]
    assert _true_residual(m, b, xv.cpu().numpy()) <= 1e-9 * np.linalg.norm(b) * 1.01
    assert buf[0].item() == 0
    dx = m.vec(np.zeros(1024))
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), dx.data_ptr(), 1e-12, 5, s)
    assert info["iterations"] == 5 and not info["converged"]
    _, _, hist = osp.cg(rp, c, v, b, np.zeros(1024), 1e-12, 5)
    assert abs(info["residual"] - hist[5] / np.linalg.norm(b)) <= 1e-9


@pytest.mark.parametrize("vt", [pyc.PYC_F32, pyc.PYC_F64])
def test_full_size_laplacian(vt):
    """The bench's system, the 5-point Laplacian on 2048 x 2048 (4.19 M rows),
    tuned as the bench tunes it: the product on every 1024th row and the last
    1024 within the bound; 20 CG steps from x = 0 with b = 1 against the
    oracle's 20 steps (binary64: to 1e-9; binary32: to 1e-3)."""
    s = torch.cuda.current_stream().cuda_stream
    nx = 2048
    n = nx * nx
    rp, c, v = inputs.poisson2d(nx, nx, NP[vt])
    m = Mat(rp, c, v, n, vt)
    x = np.random.default_rng(9).uniform(-1, 1, n).astype(NP[vt])
    dx = m.vec(x)
    dy = torch.empty(n, dtype=dx.dtype, device="cuda")
    pyc.pyc_spmv_autotune(m.h, dx.data_ptr(), dy.data_ptr(), s)
    pyc.pyc_spmv(m.h, dx.data_ptr(), dy.data_ptr(), s)
    y = dy.cpu().numpy().astype(np.float64)
    y64, ab = osp.spmv(rp, c, v, x)
    idx = np.concatenate([np.arange(0, n, 1024), np.arange(n - 1024, n)])
    length = np.diff(rp)[idx]
    assert np.all(np.abs(y[idx] - y64[idx]) <= (length + 6) * U[vt] * ab[idx])
    b = np.ones(n)
    db, dxs = m.vec(b), m.vec(np.zeros(n))
    info = pyc.pyc_cg_solve(m.h, db.data_ptr(), dxs.data_ptr(), 0.0, 20, s)
    assert info["iterations"] == 20 and not info["converged"]
    xo, k, hist = osp.cg(rp, c, v.astype(np.float64), b, np.zeros(n), 0.0, 20)
    assert k == 20
    tol = 1e-9 if vt == pyc.PYC_F64 else 1e-3
    xg = dxs.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - xo) <= tol * np.linalg.norm(xo)
    r20 = hist[20] / np.linalg.norm(b)
    assert abs(info["residual"] - r20) <= tol * r20
    del m, dx, dy, db, dxs
    torch.cuda.empty_cache()
