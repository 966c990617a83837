"""Pins for the array-expression oracle (oracle/expr.py), against exact rational
arithmetic, mpmath, closed forms and an independently pinned oracle function;
and a check that planted mistakes in its propagation rules are caught."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import expr as ox

U = 2.0 ** -24


def rn32(q: Fraction) -> float:
    """Round a rational to the nearest binary32 (ties to even), exactly (normal range)."""
    if q == 0:
        return 0.0
    s = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    m = q / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    lo = m.numerator // m.denominator
    rem = m - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return float(s * lo * Fraction(2) ** (e - 23))


def _exact(e, i):
    """Exact rational value of a tree of + - * / at element i, rounding each
    operation to binary32 exactly (what one correctly rounded evaluation gives)."""
    if not isinstance(e, tuple):
        return Fraction(float(e[i] if isinstance(e, np.ndarray) else np.float32(e)))
    op, a, b = e
    x, y = _exact(a, i), _exact(b, i)
    r = {"+": x + y, "-": x - y, "*": x * y, "/": x / y}[op]
    return Fraction(rn32(r))


def _rand_tree(rng, leaves, depth):
    if depth == 0:
        return leaves[rng.integers(len(leaves))]
    op = ["+", "-", "*", "/"][rng.integers(4)]
    return (op, _rand_tree(rng, leaves, depth - 1), _rand_tree(rng, leaves, rng.integers(depth)))


def test_rn32_matches_numpy():
    rng = np.random.default_rng(50)
    for v in rng.standard_normal(300) * 10.0 ** rng.integers(-5, 5, 300):
        assert rn32(Fraction(float(v))) == float(np.float32(v))


def test_eval_f32_is_one_rounding_per_operation():
    rng = np.random.default_rng(51)
    n = 40
    xs = [(rng.uniform(0.5, 2.0, n) * rng.choice([-1, 1], n)).astype(np.float32) for _ in range(3)]
    leaves = xs + [np.float32(2.5), np.float32(-0.75)]
    checked = 0
    for _ in range(40):
        t = _rand_tree(rng, leaves, 4)
        if not isinstance(t, tuple):
            continue
        z = np.broadcast_to(ox.eval_f32(t), (n,))
        for i in range(n):
            try:
                want = _exact(t, i)
            except ZeroDivisionError:  # a difference of equal leaves as a divisor
                continue
            if not np.isfinite(z[i]) or not 2.0 ** -100 < abs(float(want)) < 2.0 ** 100:
                continue
            assert float(z[i]) == float(want)
            checked += 1
    assert checked > 500


def test_eval_f32_sqrt_correctly_rounded():
    x = np.random.default_rng(52).uniform(0.01, 100, 500).astype(np.float32)
    r = ox.eval_f32(("sqrt", x))
    for xi, ri in zip(x, r):
        lo = Fraction(float(np.nextafter(ri, np.float32(0))))
        hi = Fraction(float(np.nextafter(ri, np.float32(np.inf))))
        mid_lo, mid_hi = (lo + Fraction(float(ri))) / 2, (hi + Fraction(float(ri))) / 2
        assert mid_lo ** 2 <= Fraction(float(xi)) <= mid_hi ** 2


def test_bound_closed_forms_for_single_operations():
    a = np.array([1.5, -3.0, 1000.0], np.float32)
    b = np.array([2.0, 0.25, -7.0], np.float32)
    av, bv = a.astype(np.float64), b.astype(np.float64)
    for op, v in (("+", av + bv), ("-", av - bv), ("*", av * bv), ("/", av / bv)):
        r, e = ox.eval_bound((op, a, b))
        assert np.array_equal(r, v) and np.array_equal(e, U * np.abs(v))
    r, e = ox.eval_bound(("exp", b))
    assert np.allclose(e, 4 * U * np.exp(bv), rtol=1e-15, atol=0)
    r, e = ox.eval_bound(("log", np.abs(a)))
    assert np.allclose(e, 2 * U * np.abs(np.log(np.abs(av))), rtol=1e-15, atol=0)
    r, e = ox.eval_bound(("sqrt", np.abs(a)))
    assert np.allclose(e, U * np.sqrt(np.abs(av)), rtol=1e-15, atol=0)
    r, e = ox.eval_bound(("neg", ("+", a, b)))
    assert np.array_equal(e, U * np.abs(av + bv))


def test_bound_values_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(53)
    n = 60
    x = rng.uniform(-2, 2, n).astype(np.float32)
    y = rng.uniform(-2, 2, n).astype(np.float32)
    w = rng.uniform(0.5, 3, n).astype(np.float32)
    t = ("+", ("*", x, ("exp", ("neg", ("*", y, y)))),
         ("-", ("tanh", ("sin", x)), ("log", ("+", w, ("cos", y)))))
    v, _ = ox.eval_bound(t)
    for i in range(n):
        X, Y, W = (mpmath.mpf(float(q[i])) for q in (x, y, w))
        ref = X * mpmath.exp(-(Y * Y)) + (mpmath.tanh(mpmath.sin(X)) - mpmath.log(W + mpmath.cos(Y)))
        assert abs(float(ref) - v[i]) <= 1e-14 * (1 + abs(float(ref)))


def _cr_eval(e, i, mp):
    """Correctly rounded binary32 evaluation (every node: exact math, one RN32)."""
    if not isinstance(e, tuple):
        return mp.mpf(float(e[i] if isinstance(e, np.ndarray) else np.float32(e)))
    op, *args = e
    a = [_cr_eval(q, i, mp) for q in args]
    f = {"+": lambda p, q: p + q, "-": lambda p, q: p - q, "*": lambda p, q: p * q,
         "/": lambda p, q: p / q, "neg": lambda p: -p, "sqrt": mp.sqrt, "exp": mp.exp,
         "log": mp.log, "sin": mp.sin, "cos": mp.cos, "tanh": mp.tanh,
         "exp2": lambda p: mp.power(2, p), "log2": lambda p: mp.log(p, 2)}[op]
    r = f(*a)
    return mp.mpf(float(np.float32(float(r))))


def test_bound_covers_a_binary32_evaluation():
    """Every bound holds for the correctly rounded evaluation (a legitimate binary32
    evaluation) on inputs chosen to make operand errors large."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(54)
    n = 80
    big = rng.uniform(500, 1000, n).astype(np.float32)
    x = rng.uniform(-2, 2, n).astype(np.float32)
    y = rng.uniform(0.1, 1, n).astype(np.float32)
    third = np.float32(1 / 3)
    trees = [
        ("*", big, ("*", x, third)),
        ("*", ("*", x, third), big),
        ("/", ("*", big, third), ("+", y, third)),
        ("sin", ("*", big, third)),
        ("exp", ("*", x, ("*", third, np.float32(7)))),
        ("log", ("+", ("*", y, third), np.float32(0.5))),
        ("sqrt", ("*", ("+", y, third), big)),
        ("tanh", ("-", ("*", big, third), ("*", big, np.float32(0.3333)))),
        # a divisor with a large relative error (cancellation)
        ("/", x, ("-", ("*", big, third), ("*", big, np.float32(0.3333)))),
    ]
    for t in trees:
        v, e = ox.eval_bound(t)
        for i in range(n):
            z = float(_cr_eval(t, i, mpmath))
            assert abs(z - v[i]) <= e[i] * (1 + 1e-9), (t[0], i, z, v[i], e[i])


def test_gauss_sin_agrees_with_the_map_oracle():
    rng = np.random.default_rng(55)
    n = 500
    x, y, u, w = (rng.uniform(-2, 2, n).astype(np.float32) for _ in range(4))
    v, _ = ox.eval_bound(("+", ("*", x, ("exp", ("neg", ("*", y, y)))), ("*", ("sin", u), w)))
    _, z64, _, _ = oracle.map_gauss_sin(x, y, u, w)
    assert np.allclose(v, z64, rtol=1e-15, atol=1e-300)


def test_eval_int_wraps():
    a = np.array([2 ** 31 - 1, -(2 ** 31), 5], np.int32)
    b = np.array([1, -1, -7], np.int32)
    assert list(ox.eval_int(("+", a, b))) == [-(2 ** 31), 2 ** 31 - 1, -2]
    assert list(ox.eval_int(("*", a, np.int32(2)))) == [-2, 0, 10]


# planted mistakes in single rules: each must make a pin above fail
_MUTANTS = {
    "mul transposed": ("*", lambda a, ea, b, eb: (a * b, np.abs(a) * ea + np.abs(b) * eb + ea * eb
                                                   + U * np.abs(a * b))),
    "add drops rounding": ("+", lambda a, ea, b, eb: (a + b, ea + eb)),
    "exp one ulp": ("exp", ox._r_func(np.exp, 1, lambda a, ea, v: np.abs(v) * np.expm1(ea))),
    "sin ignores operand error": ("sin", ox._r_func(np.sin, 2, lambda a, ea, v: 0 * ea)),
    "div drops divisor error": ("/", lambda a, ea, b, eb: (a / b, ea / np.abs(b)
                                                           + U * np.abs(a / b))),
}


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_catch_planted_rule_mistakes(name, monkeypatch):
    pytest.importorskip("mpmath")
    op, rule = _MUTANTS[name]
    monkeypatch.setitem(ox.RULES, op, (ox.RULES[op][0], rule))
    failed = False
    for pin in (test_bound_closed_forms_for_single_operations,
                test_bound_covers_a_binary32_evaluation):
        try:
            pin()
        except AssertionError:
            failed = True
    assert failed, "the pins did not catch: " + name



# ------------------------------------------------------------------ typed evaluation
_T = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}


def _exact_value(v):
    return Fraction(int(v)) if np.issubdtype(type(v), np.integer) else Fraction(float(v))


def _round_to(q: Fraction, t):
    """A rational rounded once to type t (integers: exact, then wrapped)."""
    if t is np.float64:
        return float(q)                     # Fraction -> float rounds correctly
    if t is np.float32:
        return rn32(q)
    bits = 32 if t is np.int32 else 64
    assert q.denominator == 1
    w = int(q) % 2 ** bits
    return w - 2 ** bits if w >= 2 ** (bits - 1) else w


def test_typed_result_types_follow_the_c_conversions():
    # int < long long < float < double (C's usual arithmetic conversions for these
    # four types), except that / of integers is true division in double
    names = ["i32", "i64", "f32", "f64"]
    for i, p in enumerate(names):
        for j, q in enumerate(names):
            a, b = np.array([3], _T[p]), np.array([2], _T[q])
            want = _T[names[max(i, j)]]
            for op in ("+", "-", "*", "min", "max"):
                assert ox.eval_typed((op, a, b)).dtype == want, (op, p, q)
            div = want if want in (np.float32, np.float64) else np.float64
            assert ox.eval_typed(("/", a, b)).dtype == div, (p, q)
            assert ox.eval_typed(("<", a, b)).dtype == np.int32
    assert ox.eval_typed(("sqrt", np.array([9], np.int32))).dtype == np.float64
    assert ox.eval_typed(("sqrt", np.array([9], np.float32))).dtype == np.float32
    assert ox.eval_typed(("neg", np.array([9], np.int64))).dtype == np.int64
    assert ox.eval_typed(("where", np.array([1], np.int32), np.array([1], np.float32),
                          np.array([2], np.int64))).dtype == np.float32


def test_typed_hand_values():
    i = np.array([7, -7, 2 ** 31 - 1, -(2 ** 31)], np.int32)
    two = np.int32(2)
    assert ox.eval_typed(("/", i, two)).tolist() == [3.5, -3.5, 1073741823.5, -1073741824.0]
    assert ox.eval_typed(("+", i, np.int32(1))).tolist() == [8, -6, -(2 ** 31), -(2 ** 31) + 1]
    assert ox.eval_typed(("abs", i)).tolist() == [7, 7, 2 ** 31 - 1, -(2 ** 31)]  # wraps
    assert ox.eval_typed(("sqrt", np.array([16, 2], np.int64))).tolist() == [4.0, 2.0 ** 0.5]
    assert ox.eval_typed((">", np.array([1.5, 0.5], np.float32), np.int32(1))).tolist() == [1, 0]
    # 2^24 + 1 has no binary32 value: int32 + float32 rounds the integer first
    assert ox.eval_typed(("+", np.array([2 ** 24 + 1], np.int32), np.float32(0.0))).tolist() == [
        float(2 ** 24)]
    assert ox.eval_typed(("i32", np.array([-2.7, 2.7], np.float64))).tolist() == [-2, 2]
    c = np.array([0, 3], np.int32)
    assert ox.eval_typed(("where", c, np.array([1.25, 1.25], np.float64),
                          np.array([9, 9], np.int64))).tolist() == [9.0, 1.25]


def test_typed_operations_against_rationals():
    """Each + - * / min max on random operands of every type pair equals the exact
    rational result rounded once to the operation's type (integers: wrapped)."""
    rng = np.random.default_rng(57)
    draw = {
        "i32": lambda k: rng.integers(-(2 ** 31), 2 ** 31, k).astype(np.int32),
        "i64": lambda k: rng.integers(-(2 ** 62), 2 ** 62, k).astype(np.int64),
        "f32": lambda k: (rng.uniform(-4, 4, k) * 2.0 ** rng.integers(-20, 20, k)).astype(
            np.float32),
        "f64": lambda k: rng.uniform(-4, 4, k) * 2.0 ** rng.integers(-40, 40, k),
    }
    ops = {"+": lambda a, b: a + b, "-": lambda a, b: a - b, "*": lambda a, b: a * b,
           "/": lambda a, b: a / b, "min": min, "max": max}
    names = list(_T)
    for p in names:
        for q in names:
            a, b = draw[p](40), draw[q](40)
            for op, f in ops.items():
                got = ox.eval_typed((op, a, b))
                t = got.dtype.type
                for k in range(40):
                    if op == "/" and b[k] == 0:
                        continue
                    x, y = _exact_value(a[k]), _exact_value(b[k])
                    if t in (np.float32, np.float64):
                        # operands convert to t first (one rounding each), then one more
                        x, y = Fraction(_round_to(x, t)), Fraction(_round_to(y, t))
                        want = _round_to(f(x, y), t)
                    else:
                        want = _round_to(f(x, y), t)
                    assert float(got[k]) == float(want) if t in (np.float32, np.float64) else \
                        int(got[k]) == want, (op, p, q, k, a[k], b[k], got[k], want)


_TYPED_MUTANTS = {
    "integer division floors": ("result_type", lambda op, types: (
        max(types, key=ox.TYPE_ORDER.index) if op not in ox._CASTS and op not in (
            "neg", "abs", "sqrt", "where") else _ORIG_RESULT_TYPE(op, types))),
    "int64 with float32 widens to float64": ("result_type", lambda op, types: (
        np.float64 if np.int64 in types and np.float32 in types else _ORIG_RESULT_TYPE(op, types))),
    "sqrt of an integer in float32": ("result_type", lambda op, types: (
        np.float32 if op == "sqrt" and types[0] in (np.int32, np.int64) else
        _ORIG_RESULT_TYPE(op, types))),
    "float min propagates the first operand": ("_apply", lambda op, t, vals: (
        np.asarray(vals[0]).astype(t) if op == "min" else _ORIG_APPLY(op, t, vals))),
}
_ORIG_RESULT_TYPE = ox.result_type
_ORIG_APPLY = ox._apply


@pytest.mark.parametrize("name", sorted(_TYPED_MUTANTS))
def test_typed_pins_catch_planted_mistakes(name, monkeypatch):
    fn, bad = _TYPED_MUTANTS[name]
    monkeypatch.setattr(ox, fn, bad)
    failed = False
    for pin in (test_typed_result_types_follow_the_c_conversions, test_typed_hand_values,
                test_typed_operations_against_rationals):
        try:
            pin()
        except (AssertionError, ZeroDivisionError):
            failed = True
    assert failed, "the pins did not catch: " + name
