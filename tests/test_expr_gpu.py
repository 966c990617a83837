"""Fused array expressions on the GPU (Sec. 3.2.3-3.2.4): one kernel per
expression, checked against the expression oracle element by element."""
import numpy as np
import pytest
import torch

import oracle
from oracle import expr as ox
from paper_1304_5553_gb300 import gpuarray as ga
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu


def _dev(a):
    return ga.GArray(torch.from_numpy(np.ascontiguousarray(a)).cuda())


def _host(g):
    return g.tensor.cpu().numpy()


def _arrays(seed, n, k, lo=-2.0, hi=2.0):
    return [inputs.uniform_f32(seed, s, n, lo, hi) for s in range(k)]


@pytest.mark.parametrize("n", [1, 7, 1000, 65536 + 13, 1 << 22])
def test_correctly_rounded_trees_are_bit_exact(n):
    """+ - * / sqrt neg abs min max: each operation rounds once in source order, so
    the fused kernel equals binary32 evaluation bit for bit."""
    x, y, z = _arrays(60, n, 3)
    X, Y, Z = (_dev(a) for a in (x, y, z))
    a, b = np.float32(2.5), np.float32(-0.75)
    cases = [
        (lambda: 2.5 * X + (-0.75) * Y, ("+", ("*", a, x), ("*", b, y))),
        (lambda: (X * Y - Z) / (ga.fabs(Y) + 1.0),
         ("/", ("-", ("*", x, y), z), ("+", ("abs", y), np.float32(1)))),
        (lambda: ga.sqrt(X * X + Y * Y) - ga.maximum(X, -Z),
         ("-", ("sqrt", ("+", ("*", x, x), ("*", y, y))), ("max", x, ("neg", z)))),
        (lambda: ga.minimum(X, Y) * (X - (-Y)), ("*", ("min", x, y), ("-", x, ("neg", y)))),
    ]
    for build, tree in cases:
        got = _host(ga.evaluate(build()))
        want = np.broadcast_to(ox.eval_f32(tree), (n,))
        assert np.array_equal(got, want)


def test_transcendental_trees_within_bound():
    n = (1 << 20) + 5
    x, y, w = _arrays(61, n, 3)
    u = inputs.uniform_f32(61, 3, n, 0.1, 3.0)
    X, Y, W, V = (_dev(a) for a in (x, y, w, u))
    cases = [
        (lambda: X * ga.exp(-Y * Y) + ga.sin(W) * V,
         ("+", ("*", x, ("exp", ("neg", ("*", y, y)))), ("*", ("sin", w), u))),
        (lambda: ga.log(V + 0.5) * ga.tanh(X) - ga.cos(Y * 3.0),
         ("-", ("*", ("log", ("+", u, np.float32(0.5))), ("tanh", x)),
          ("cos", ("*", y, np.float32(3))))),
        (lambda: ga.exp2(X) / ga.sqrt(V) + ga.log2(V),
         ("+", ("/", ("exp2", x), ("sqrt", u)), ("log2", u))),
    ]
    for build, tree in cases:
        got = _host(ga.evaluate(build())).astype(np.float64)
        v, e = ox.eval_bound(tree)
        assert np.all(np.abs(got - v) <= e * (1 + 1e-6) + 1e-30)


def test_fused_equals_the_hand_written_map():
    """The four-input expression fused from operators is the same computation as
    the stock map z[i] = x[i]*exp(-y[i]*y[i]) + sin(u[i])*w[i]: identical bits."""
    n = (1 << 21) + 3
    arrs = _arrays(62, n, 4)
    X, Y, U_, W = (_dev(a) for a in arrs)
    fused = _host(ga.evaluate(X * ga.exp(-(Y * Y)) + ga.sin(U_) * W))
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    h = stock.create("gauss_sin_f32")
    pyc.pyc_map_launch(h, n, [X.tensor.data_ptr(), Y.tensor.data_ptr(), U_.tensor.data_ptr(),
                              W.tensor.data_ptr(), z.data_ptr()], None,
                       torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(fused, z.cpu().numpy())


def test_eager_equals_fused_and_counts_kernels():
    n = 100003
    x, y = _arrays(63, n, 2)
    X, Y = _dev(x), _dev(y)
    e = (X * Y + 2.5) * (X - Y) / (ga.fabs(Y) + 1.0)
    fused = _host(ga.evaluate(e))
    eager, kernels = ga.evaluate_eager(e)
    assert kernels == 7 and np.array_equal(fused, _host(eager))


def test_bf16_storage_and_int_wrap():
    n = 50021
    xb = inputs.to_bf16_values(inputs.uniform_f32(64, 0, n, -2, 2))
    yb = inputs.to_bf16_values(inputs.uniform_f32(64, 1, n, -2, 2))
    Xb = ga.GArray(torch.from_numpy(xb).to(torch.bfloat16).cuda())
    Yb = ga.GArray(torch.from_numpy(yb).to(torch.bfloat16).cuda())
    out = ga.evaluate(2.5 * Xb - 0.75 * Yb, dtype=pyc.PYC_BF16)
    assert out.tensor.dtype == torch.bfloat16
    # binary32 arithmetic in source order, then one rounding to bfloat16 on the store
    z = oracle.map_lin_comb_f32ops(2.5, xb, -0.75, yb, out_bf16=True)
    assert np.array_equal(out.tensor.float().cpu().numpy(), z)
    a = np.random.default_rng(65).integers(-2 ** 31, 2 ** 31, n).astype(np.int32)
    b = np.random.default_rng(66).integers(-2 ** 31, 2 ** 31, n).astype(np.int32)
    A, B = _dev(a), _dev(b)
    got = _host(ga.evaluate(A * B - (A + B) * 3))
    assert got.dtype == np.int32
    assert np.array_equal(got, ox.eval_int(("-", ("*", a, b), ("*", ("+", a, b), np.int32(3)))))


def test_in_place_and_offsets():
    n = 70001
    x, y = _arrays(67, n + 8, 2)
    t = torch.from_numpy(x).cuda()
    u = torch.from_numpy(y).cuda()
    X = ga.GArray(t[1:n + 1])   # unaligned view
    Y = ga.GArray(u[3:n + 3])
    X.assign(X * 2.0 + Y)
    want = ox.eval_f32(("+", ("*", x[1:n + 1], np.float32(2)), y[3:n + 3]))
    assert np.array_equal(t[1:n + 1].cpu().numpy(), want)
    assert t[0].item() == x[0] and t[n + 1].item() == x[n + 1]


def test_reductions():
    n = (1 << 22) + 17
    x, y = _arrays(68, n, 2, -1.0, 1.0)
    X, Y = _dev(x), _dev(y)
    d = ga.dot(X, Y).item()
    s64, ab = oracle.dot_f32(x, y)
    assert abs(d - s64) <= 8 * 2.0 ** -24 * ab
    m = ga.max(ga.fabs(X - Y)).item()
    assert m == float(np.max(np.abs(ox.eval_f32(("-", x, y)))))
    xi = inputs.int_uniform_i32(68, 2, n)
    assert ga.sum(_dev(xi)).item() == oracle.sum_i32_i64(xi)
    # a transcendental map inside the reduction: |r - S| <= sum of term bounds + 8u sum|t|
    v, e = ox.eval_bound(("*", x, ("exp", ("neg", ("*", y, y)))))
    r = ga.sum(X * ga.exp(-(Y * Y))).item()
    assert abs(r - v.sum()) <= e.sum() + 8 * 2.0 ** -24 * (np.abs(v).sum() + e.sum())


def test_one_compile_per_shape():
    n = 4096
    x, y = _arrays(69, n, 2)
    X, Y = _dev(x), _dev(y)
    ga.evaluate(X * 1.5 + Y)
    before = pyc.pyc_cache_stats()
    for c in (0.5, 2.0, -3.25):  # new scalar values: same kernel, no compilation
        got = _host(ga.evaluate(X * c + Y))
        assert np.array_equal(got, ox.eval_f32(("+", ("*", x, np.float32(c)), y)))
    assert pyc.pyc_cache_stats()["compiled"] == before["compiled"]


def test_full_size_sampled():
    """The bench's expressions at n = 2^28, tuned as the bench tunes them: every
    4096th element and the last 4096 against the oracle (bit-exact for the
    correctly rounded tree, within the first-order bound for the other)."""
    n = 1 << 28
    xs = [inputs.uniform_f32(1, s, n, -2.0, 2.0) for s in range(4)]
    X, Y, U, W = (_dev(a) for a in xs)
    idx = np.concatenate([np.arange(0, n, 4096), np.arange(n - 4096, n)])
    x, y, u, w = (a[idx] for a in xs)
    out = ga.GArray(torch.empty(n, dtype=torch.float32, device="cuda"))
    e = 2.5 * X - 0.75 * Y
    ga.autotune(e)
    ga.evaluate(e, out=out)
    want = ox.eval_f32(("-", ("*", np.float32(2.5), x), ("*", np.float32(0.75), y)))
    assert np.array_equal(_host(out)[idx], want)
    e = X * ga.exp(-(Y * Y)) + ga.sin(U) * W
    ga.autotune(e)
    ga.evaluate(e, out=out)
    v, err = ox.eval_bound(("+", ("*", x, ("exp", ("neg", ("*", y, y)))), ("*", ("sin", u), w)))
    assert np.all(np.abs(_host(out)[idx].astype(np.float64) - v) <= err * (1 + 1e-6) + 1e-30)
    del X, Y, U, W, out
    torch.cuda.empty_cache()
