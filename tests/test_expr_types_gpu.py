"""Fused array expressions over mixed storage types (Sec. 3.2.3-3.2.4) on the
GPU: trees mixing binary64, binary32, binary16 / bfloat16 (read as binary32),
int32 and int64 arrays with Python scalars compile to one kernel each and
equal the typed expression oracle bit for bit -- the result type, the
promotion of every operand, true division and the float64 math of integers,
int32 comparisons, two's-complement wrap-around and one rounding per
operation in its own type."""
import numpy as np
import pytest
import torch

from oracle import expr as ox
from paper_1304_5553_gb300 import gpuarray as ga
from paper_1304_5553_gb300 import inputs

pytestmark = pytest.mark.gpu

_NP = {torch.float32: np.float32, torch.float64: np.float64, torch.int32: np.int32,
       torch.int64: np.int64}


def _data(n):
    x32 = inputs.uniform_f32(70, 0, n, -4.0, 4.0)
    x64 = inputs.unit_f64(70, 1, n) * 8.0 - 4.0
    i32 = inputs.int_uniform_i32(70, 2, n, -(2 ** 31) + 1, 2 ** 31 - 1)   # no INT_MIN
    i64 = (inputs.int_uniform_i32(70, 3, n).astype(np.int64) << 40) + inputs.int_uniform_i32(
        70, 4, n)
    d = inputs.int_uniform_i32(70, 5, n, 1, 100) * np.where(
        inputs.int_uniform_i32(70, 6, n, 0, 1) > 0, 1, -1).astype(np.int32)  # nonzero divisors
    h16 = inputs.to_f16_values(inputs.uniform_f32(70, 7, n, -4.0, 4.0))
    b16 = inputs.to_bf16_values(inputs.uniform_f32(70, 8, n, -4.0, 4.0))
    host = dict(x32=x32, x64=x64, i32=i32, i64=i64, d=d.astype(np.int32),
                h16=h16.astype(np.float32), b16=b16)          # halves enter as their values
    dev = dict(x32=torch.from_numpy(x32), x64=torch.from_numpy(x64), i32=torch.from_numpy(i32),
               i64=torch.from_numpy(i64), d=torch.from_numpy(host["d"]),
               h16=torch.from_numpy(h16), b16=torch.from_numpy(b16).to(torch.bfloat16))
    return host, {k: ga.GArray(v.cuda()) for k, v in dev.items()}


def _cases(G, h):
    X32, X64, I32, I64, D, H16, B16 = (G[k] for k in ("x32", "x64", "i32", "i64", "d", "h16",
                                                     "b16"))
    f32, f64, s32 = np.float32, np.float64, np.int32
    return [
        # (GPU expression, oracle tree); Python floats are binary64 scalars when a
        # binary64 array is in the tree, else binary32; Python ints are int32
        (X64 * 2.5 + I32, ("+", ("*", h["x64"], f64(2.5)), h["i32"])),
        (I32 / D, ("/", h["i32"], h["d"])),
        (I64 * 3 - I32, ("-", ("*", h["i64"], s32(3)), h["i32"])),
        (X32 * I32 + 0.5, ("+", ("*", h["x32"], h["i32"]), f32(0.5))),
        (ga.sqrt(abs(I32)), ("sqrt", ("abs", h["i32"]))),
        (H16 * X32 - 1.25, ("-", ("*", h["h16"], h["x32"]), f32(1.25))),
        (ga.where(X32 > 0, X64, I64), ("where", (">", h["x32"], s32(0)), h["x64"], h["i64"])),
        (ga.maximum(I64, I32) + ga.minimum(X64, X32),
         ("+", ("max", h["i64"], h["i32"]), ("min", h["x64"], h["x32"]))),
        (X64.astype(torch.float32) * X32, ("*", ("f32", h["x64"]), h["x32"])),
        (B16 * 3 + I32 / 7, ("+", ("*", h["b16"], s32(3)), ("/", h["i32"], s32(7)))),
        ((I32 - I64) * (I32 + 1), ("*", ("-", h["i32"], h["i64"]), ("+", h["i32"], s32(1)))),
        (-I32 + I32 * I32, ("+", ("neg", h["i32"]), ("*", h["i32"], h["i32"]))),
        ((X32 <= H16) + (I64 != I32), ("+", ("<=", h["x32"], h["h16"]), ("!=", h["i64"],
                                                                           h["i32"]))),
    ]


@pytest.mark.parametrize("n", [1, 1000, 65536 + 13, (1 << 20) + 3])
def test_mixed_type_trees_bit_exact(n):
    host, G = _data(n)
    for k, (expr, tree) in enumerate(_cases(G, host)):
        got = ga.evaluate(expr).tensor.cpu()
        want = np.asarray(ox.eval_typed(tree))
        assert _NP[got.dtype] == want.dtype.type, (k, got.dtype, want.dtype)
        g = got.numpy()
        # bit for bit: compare each element's bytes
        bad = np.flatnonzero((g.view(np.uint8).reshape(n, -1) !=
                              want.view(np.uint8).reshape(n, -1)).any(axis=1))
        assert bad.size == 0, (k, n, bad[:4], g[bad[:4]], want[bad[:4]])


def _random_tree(rng, G, h, depth):
    """A random expression over the arrays of _data (and Python scalars), built as
    a GPU expression and as a record of its tree side by side.  No division by
    zero (divisors are |e| + 1), square roots of |e|, small integer leaves; the
    only cast is to binary64."""
    names = ["x32", "x64", "i32", "i64", "h16", "b16"]
    if depth == 0 or rng.random() < 0.25:
        r = rng.random()
        if r < 0.75:
            k = names[int(rng.integers(0, len(names)))]
            return G[k], ("leaf", k)
        if r < 0.9:
            v = float(np.round(rng.uniform(-3, 3), 3))
            return v, ("float", v)
        v = int(rng.integers(-9, 10))
        return v, ("int", v)
    op = ["+", "-", "*", "/", "min", "max", "neg", "abs", "sqrt", "cmp", "where", "cast"][
        int(rng.integers(0, 12))]
    if op in ("neg", "abs", "sqrt", "cast"):
        ge, te = _random_tree(rng, G, h, depth - 1)
        if not isinstance(ge, ga.Expr):  # unary operators need an array operand
            ge, te = G["x32"], ("leaf", "x32")
        if op == "neg":
            return -ge, ("neg", te)
        if op == "abs":
            return abs(ge), ("abs", te)
        if op == "sqrt":
            return ga.sqrt(abs(ge)), ("sqrt", ("abs", te))
        return ge.astype(torch.float64), ("f64", te)
    ga_, ta = _random_tree(rng, G, h, depth - 1)
    gb_, tb = _random_tree(rng, G, h, depth - 1)
    if not isinstance(ga_, ga.Expr) and not isinstance(gb_, ga.Expr):
        ga_, ta = G["x32"], ("leaf", "x32")
    if op == "+":
        return ga_ + gb_, ("+", ta, tb)
    if op == "-":
        return ga_ - gb_, ("-", ta, tb)
    if op == "*":
        return ga_ * gb_, ("*", ta, tb)
    if op == "/":
        if not isinstance(gb_, ga.Expr):
            gb_, tb = G["i32"], ("leaf", "i32")
        return ga_ / (abs(gb_) + 1), ("/", ta, ("+", ("abs", tb), ("int", 1)))
    if op == "min":
        return ga.minimum(ga_, gb_), ("min", ta, tb)
    if op == "max":
        return ga.maximum(ga_, gb_), ("max", ta, tb)
    if op == "cmp":
        return (ga_ < gb_), ("<", ta, tb)
    return ga.where(ga_ > gb_, ga_, gb_), ("where", (">", ta, tb), ta, tb)


def _oracle_tree(t, h, f64):
    """The oracle tuple of a _random_tree record: Python floats are binary64
    scalars when a binary64 array is in the whole tree, else binary32; Python
    ints are int32."""
    if t[0] == "leaf":
        return h[t[1]]
    if t[0] == "float":
        return np.float64(t[1]) if f64 else np.float32(t[1])
    if t[0] == "int":
        return np.int32(t[1])
    return (t[0],) + tuple(_oracle_tree(c, h, f64) for c in t[1:])


def _all_finite(tree):
    """True if every floating value the oracle computes on the way to tree's
    result is finite (no overflow to infinity, no NaN from an integer that
    wrapped to INT_MIN under sqrt(abs(.))): such trees are redrawn, since the
    ordering of NaN under min / max / where is not what the test checks."""
    if not isinstance(tree, tuple):
        return True
    if not all(_all_finite(c) for c in tree[1:]):
        return False
    v = np.asarray(ox.eval_typed(tree))
    return v.dtype.kind != "f" or bool(np.all(np.isfinite(v)))


def _has_f64(t):
    return t == ("leaf", "x64") or (t[0] not in ("leaf", "float", "int") and
                                    any(_has_f64(c) for c in t[1:]))


def test_random_mixed_type_trees():
    """60 random trees of depth up to 4 over every array type and Python scalars,
    each compiled into one kernel and compared with the typed oracle: the result
    type, and every element (integers exactly; floating values exactly, +0 and -0
    counting as equal)."""
    n = 4099
    host, G = _data(n)
    host = dict(host, i32=np.clip(host["i32"], -99, 99).astype(np.int32),
                i64=np.clip(host["i64"], -99, 99).astype(np.int64))
    G = dict(G, i32=ga.GArray(torch.from_numpy(host["i32"]).cuda()),
             i64=ga.GArray(torch.from_numpy(host["i64"]).cuda()))
    rng = np.random.default_rng(98)
    done = 0
    while done < 60:
        expr, rec = _random_tree(rng, G, host, 4)
        if not isinstance(expr, ga.Expr) or isinstance(expr, ga.GArray):
            continue
        tree = _oracle_tree(rec, host, _has_f64(rec))
        if not _all_finite(tree):
            continue
        want = np.asarray(ox.eval_typed(tree))
        got = ga.evaluate(expr).tensor.cpu().numpy()
        assert got.dtype.type == want.dtype.type, (rec, got.dtype, want.dtype)
        assert np.array_equal(got, want), (rec, np.flatnonzero(got != want)[:4])
        done += 1
