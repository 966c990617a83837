"""ORACLE -- test infrastructure only: array expressions (Sec. 3.2.3-3.2.4).

An expression is a nested tuple: (op, operand, ...) with operands that are
expressions, numpy arrays (binary32 / bfloat16-valued binary32 / int32 arrays,
equal lengths) or numpy scalars.  Operators as in the library's fused
expressions: + - * / min max, neg abs sqrt exp exp2 log log2 sin cos tanh.

* `eval_f32(e)`: binary32 evaluation, each operation rounded once, in source
  order (numpy's IEEE binary32 arithmetic; sqrt is correctly rounded).  This is
  the exact result of a binary32 program without contraction, for trees of
  correctly rounded operations only (+ - * / sqrt neg abs min max).
* `eval_bound(e)`: (v, err): v is the expression evaluated in binary64 on the
  exact operand values, err a first-order bound on |z - v| for ANY binary32
  evaluation z of the same tree whose basic operations round to nearest and
  whose math functions are within the maximum errors CUDA documents for its
  single-precision functions (expf, exp2f, sinf, cosf, tanhf: 2 ulp; logf,
  log2f: 1 ulp; sqrtf: correctly rounded).  One ulp of y is at most
  2^-23 |y| = 2u|y| (u = 2^-24), so k ulp <= 2ku|y|.
* `eval_int(e)`: int32 arithmetic with two's-complement wrap (numpy int32).
* `eval_typed(e)`: the mixed-type evaluation of the library's expression
  typing (int32 < int64 < float32 < float64, true division, float64 math of
  integers, int32 comparisons, wrap-around), one rounding per operation in the
  operation's own type; the rules are written out at its definition.

Propagation, for operands with exact values a, b and error bounds ea, eb:
  a +- b : ea + eb + u(|v| + ea + eb)
  a * b  : p = |a|eb + |b|ea + ea eb;          p + u(|v| + p)
  a / b  : p = (ea + |v| eb) / (|b| - eb);     p + u(|v| + p)     (|b| > eb)
  neg, abs : ea;   min, max : max(ea, eb)
  sqrt a : p = sqrt(a + ea) - sqrt(max(a - ea, 0));             p + u(|v| + p)
  exp a  : p = |v|(e^ea - 1);                                    p + 4u(|v| + p)
  exp2 a : p = |v|(2^ea - 1);                                    p + 4u(|v| + p)
  log a  : p = ln(a / (a - ea));                                 p + 2u(|v| + p)
  log2 a : p = log2(a / (a - ea));                               p + 2u(|v| + p)
  sin, cos, tanh a : p = ea (derivatives bounded by 1);          p + 4u(|v| + p)
Leaves have error 0 (their binary64 values are the stored values).
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -24

_F32 = {
    "+": lambda a, b: a + b, "-": lambda a, b: a - b, "*": lambda a, b: a * b,
    "/": lambda a, b: a / b, "min": np.minimum, "max": np.maximum,
    "neg": lambda a: -a, "abs": np.abs, "sqrt": np.sqrt,
}


def _leaf32(x):
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float32
        return x
    return np.float32(x)


def eval_f32(e):
    """Binary32, one rounding per operation, source order."""
    if not isinstance(e, tuple):
        return _leaf32(e)
    op, *args = e
    if op not in _F32:
        raise ValueError("eval_f32 covers correctly rounded operations only, not %r" % op)
    vals = [eval_f32(a) for a in args]
    with np.errstate(all="ignore"):
        r = _F32[op](*vals)
    return np.asarray(r, dtype=np.float32) if isinstance(r, np.ndarray) else np.float32(r)


def _r_add(a, ea, b, eb, sign):
    v = a + sign * b
    return v, ea + eb + U * (np.abs(v) + ea + eb)


def _r_mul(a, ea, b, eb):
    v = a * b
    p = np.abs(a) * eb + np.abs(b) * ea + ea * eb
    return v, p + U * (np.abs(v) + p)


def _r_div(a, ea, b, eb):
    v = a / b
    if np.any(np.abs(b) <= eb):
        raise ValueError("divisor interval contains zero")
    p = (ea + np.abs(v) * eb) / (np.abs(b) - eb)
    return v, p + U * (np.abs(v) + p)


def _r_func(f, k_ulp, prop):
    def rule(a, ea):
        v = f(a)
        p = prop(a, ea, v)
        return v, p + 2 * k_ulp * U * (np.abs(v) + p)
    return rule


def _sqrt_prop(a, ea, v):
    if np.any(a < 0):
        raise ValueError("sqrt of a negative value")
    return np.sqrt(a + ea) - np.sqrt(np.maximum(a - ea, 0.0))


def _log_prop(base):
    def prop(a, ea, v):
        if np.any(a - ea <= 0):
            raise ValueError("log argument interval reaches zero")
        return np.log(a / (a - ea)) / base
    return prop


# Rules: name -> (arity, function of (a, ea[, b, eb]) -> (v, err)).  Exposed so
# tests can check that a planted mistake in one rule is caught.
RULES = {
    "+": (2, lambda a, ea, b, eb: _r_add(a, ea, b, eb, 1.0)),
    "-": (2, lambda a, ea, b, eb: _r_add(a, ea, b, eb, -1.0)),
    "*": (2, _r_mul),
    "/": (2, _r_div),
    "min": (2, lambda a, ea, b, eb: (np.minimum(a, b), np.maximum(ea, eb))),
    "max": (2, lambda a, ea, b, eb: (np.maximum(a, b), np.maximum(ea, eb))),
    "neg": (1, lambda a, ea: (-a, ea)),
    "abs": (1, lambda a, ea: (np.abs(a), ea)),
    "sqrt": (1, _r_func(np.sqrt, 0.5, _sqrt_prop)),
    "exp": (1, _r_func(np.exp, 2, lambda a, ea, v: np.abs(v) * np.expm1(ea))),
    "exp2": (1, _r_func(np.exp2, 2, lambda a, ea, v: np.abs(v) * np.expm1(ea * np.log(2.0)))),
    "log": (1, _r_func(np.log, 1, _log_prop(1.0))),
    "log2": (1, _r_func(np.log2, 1, _log_prop(np.log(2.0)))),
    "sin": (1, _r_func(np.sin, 2, lambda a, ea, v: ea)),
    "cos": (1, _r_func(np.cos, 2, lambda a, ea, v: ea)),
    "tanh": (1, _r_func(np.tanh, 2, lambda a, ea, v: ea)),
}


def eval_bound(e):
    """(binary64 value, first-order bound on any binary32 evaluation's error)."""
    if not isinstance(e, tuple):
        if isinstance(e, np.ndarray):
            v = e.astype(np.float64)
        else:
            v = np.float64(np.float32(e))  # scalar arguments are passed as binary32
        return v, np.zeros_like(v)
    op, *args = e
    arity, rule = RULES[op]
    assert len(args) == arity, op
    flat = []
    for a in args:
        flat.extend(eval_bound(a))
    with np.errstate(all="ignore"):
        return rule(*flat)


_INT = {
    "+": lambda a, b: a + b, "-": lambda a, b: a - b, "*": lambda a, b: a * b,
    "neg": lambda a: -a, "abs": np.abs, "min": np.minimum, "max": np.maximum,
}


def eval_int(e):
    """int32 evaluation with two's-complement wrap-around."""
    if not isinstance(e, tuple):
        return np.asarray(e, dtype=np.int32) if isinstance(e, np.ndarray) else np.int32(e)
    op, *args = e
    vals = [eval_int(a) for a in args]
    with np.errstate(over="ignore"):
        r = _INT[op](*vals)
    return np.asarray(r).astype(np.int32)


# ------------------------------------------------------------------ typed evaluation
# The typing of fused array expressions (C-style, on four types ordered
# int32 < int64 < float32 < float64): bfloat16 and binary16 arrays are read as
# binary32, so they enter here as float32 arrays holding their values; scalar
# arguments carry their own type (numpy scalars: np.float32, np.float64,
# np.int32, np.int64).  A binary operation converts both operands to the higher
# of their types and rounds once in it; true division and the math functions of
# an integer type compute in float64; comparisons give int32 1 or 0; integer
# + - * wrap around in two's complement; the casts f32 f64 i32 i64 convert
# (a float to an integer truncates toward zero).

TYPE_ORDER = (np.int32, np.int64, np.float32, np.float64)
_CMP = {"<": np.less, "<=": np.less_equal, ">": np.greater, ">=": np.greater_equal,
        "==": np.equal, "!=": np.not_equal}
_CASTS = {"f32": np.float32, "f64": np.float64, "i32": np.int32, "i64": np.int64}


def type_of(v):
    t = np.asarray(v).dtype.type
    if t not in TYPE_ORDER:
        raise TypeError("typed operands are int32, int64, float32 or float64, not %r" % t)
    return t


def _is_float(t):
    return t in (np.float32, np.float64)


def result_type(op, types):
    """The type an operation computes in (and returns, but for comparisons)."""
    if op in _CASTS:
        return _CASTS[op]
    if op in ("neg", "abs"):
        return types[0]
    if op == "sqrt":
        return types[0] if _is_float(types[0]) else np.float64
    if op == "where":
        types = types[1:]
    t = max(types, key=TYPE_ORDER.index)
    if op == "/" and not _is_float(t):
        return np.float64  # true division
    return t


def _apply(op, t, vals):
    a = [np.asarray(v).astype(t) for v in vals]
    with np.errstate(all="ignore"):
        if op in _CASTS:
            return np.asarray(vals[0]).astype(t)
        if op == "neg":
            return -a[0]
        if op == "abs":
            return np.abs(a[0])
        if op == "sqrt":
            return np.sqrt(a[0])
        if op == "+":
            return a[0] + a[1]
        if op == "-":
            return a[0] - a[1]
        if op == "*":
            return a[0] * a[1]
        if op == "/":
            return a[0] / a[1]
        if op in ("min", "max"):
            if _is_float(t):
                return (np.fmin if op == "min" else np.fmax)(a[0], a[1])
            return (np.minimum if op == "min" else np.maximum)(a[0], a[1])
        if op in _CMP:
            return _CMP[op](a[0], a[1]).astype(np.int32)
    raise ValueError("eval_typed: unknown operator %r" % op)


def eval_typed(e):
    """Evaluate a tree under the typing above: each operation converts its
    operands to its type and rounds once there, in source order."""
    if not isinstance(e, tuple):
        type_of(e)
        return e
    op, *args = e
    vals = [eval_typed(a) for a in args]
    if op == "where":
        t = result_type(op, [type_of(v) for v in vals])
        c = np.asarray(vals[0])
        return np.where(c != 0, np.asarray(vals[1]).astype(t), np.asarray(vals[2]).astype(t))
    t = result_type(op, [type_of(v) for v in vals])
    r = _apply(op, t, vals)
    return np.asarray(r).astype(np.int32 if op in _CMP else t)
