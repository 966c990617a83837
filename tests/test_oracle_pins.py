"""Pins for the CPU oracle: each oracle function is checked against something
other than itself -- closed forms, exact rational arithmetic (fractions),
correctly rounded library sums (math.fsum), arbitrary-precision evaluation
(mpmath), library rounding (numpy / torch CPU conversions), brute force and
invariants -- chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1304_5553_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = int(v)
    return out


def _fr(v):
    return Fraction(float(v))


# ----------------------------------------------------------------- rounding

def test_round_bf16_hand_cases():
    for line in open(os.path.join(GOLD, "bf16_rounding_cases.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        src, want = line.split()
        d = float.fromhex(src)
        w = float("inf") if want == "inf" else float.fromhex(want)
        assert oracle.round_bf16(d) == w, (src, want, oracle.round_bf16(d))
        assert oracle.round_bf16(-d) == -w


def test_round_bf16_matches_torch_on_binary32_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_bf16(float(v)) for v in x])
    assert np.array_equal(got, want)


def test_round_f32_ties_and_numpy():
    assert oracle.round_f32(1 + 2.0 ** -24) == 1.0
    assert oracle.round_f32(1 + 3 * 2.0 ** -24) == 1 + 2.0 ** -22
    rng = np.random.default_rng(2)
    d = rng.standard_normal(5000) * 1e3
    assert np.array_equal(np.array([oracle.round_f32(v) for v in d]), d.astype(np.float32))


# ----------------------------------------------------------------- maps

def _neighbours_f32(z):
    z = np.float32(z)
    return float(np.nextafter(z, np.float32(-np.inf))), float(np.nextafter(z, np.float32(np.inf)))


def _is_nearest(exact: Fraction, z: float, lo: float, hi: float) -> bool:
    """z is a nearest representable value of `exact` given its neighbours."""
    zf = Fraction(z)
    return (Fraction(lo) + zf) / 2 <= exact <= (zf + Fraction(hi)) / 2


def test_map_scale_listing1():
    # Listing 1 / Listing 2: doubling is exact
    x = np.random.default_rng(3).standard_normal((4, 4)).astype(np.float32).ravel()
    z, z64 = oracle.map_scale(2, x)
    assert np.array_equal(z, x * np.float32(2))
    assert np.array_equal(z64, 2.0 * x.astype(np.float64))


def test_map_add_listing4_bit_exact():
    # Listing 4 asserts norm(c - (a+b)) == 0 against numpy's binary32 add
    n = 16 * 32 * 33
    rng = np.random.default_rng(4)
    a = rng.standard_normal(n).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    z, _ = oracle.map_add(a, b)
    assert np.linalg.norm(z - (a + b)) == 0


@pytest.mark.parametrize("out_bf16", [False, True])
def test_map_lin_comb_exact_rational(out_bf16):
    n = 3000
    x = inputs.uniform_f32(11, 0, n, -2.0, 2.0)
    y = inputs.uniform_f32(11, 1, n, -2.0, 2.0)
    if out_bf16:
        x, y = inputs.to_bf16_values(x), inputs.to_bf16_values(y)
    a, b = 2.5, -0.75
    z, z64, tab = oracle.map_lin_comb(a, x, b, y, out_bf16=out_bf16)
    for i in range(n):
        ex = Fraction(a) * _fr(x[i]) + Fraction(b) * _fr(y[i])
        # binary64 value: within half an ulp of binary64
        assert abs(_fr(z64[i]) - ex) <= Fraction(abs(float(ex))) * Fraction(1, 2 ** 53) + Fraction(1, 2 ** 1074)
        assert tab[i] == abs(a * float(x[i])) + abs(b * float(y[i]))
        if out_bf16:
            bits = np.array([z[i]], np.float32).view(np.uint32)[0]
            assert bits & 0xFFFF == 0  # a bfloat16 value
            lo = np.array([bits - 0x10000], np.uint32).view(np.float32)[0] if z[i] != 0 else -2.0 ** -133
            hi = np.array([bits + 0x10000], np.uint32).view(np.float32)[0] if z[i] != 0 else 2.0 ** -133
            if z[i] < 0:
                lo, hi = hi, lo
            assert _is_nearest(ex, float(z[i]), float(lo), float(hi)), i
        else:
            lo, hi = _neighbours_f32(z[i])
            assert _is_nearest(ex, float(z[i]), lo, hi), i


def test_map_lin_comb_listing3a_int_scalars():
    # Listing 3a passes the Python ints 5 and 6 for float parameters
    x = np.arange(50, dtype=np.float32) * np.float32(0.25)
    y = np.arange(50, dtype=np.float32)[::-1].copy()
    z, _, _ = oracle.map_lin_comb(5, x, 6, y)
    assert np.array_equal(z, (5 * x.astype(np.float64) + 6 * y.astype(np.float64)).astype(np.float32))
    # hand value at i = 0: 5*0 + 6*49 = 294
    assert z[0] == 294.0 and z[49] == 5 * 49 * 0.25


@pytest.mark.parametrize("out_bf16", [False, True])
def test_map_lin_comb_f32ops_rounds_each_op(out_bf16):
    # each binary32 operation is the correctly rounded exact result (checked with
    # fractions), applied in source order; numpy's binary32 arithmetic agrees
    n = 2000
    x = inputs.uniform_f32(16, 0, n, -2.0, 2.0)
    y = inputs.uniform_f32(16, 1, n, -2.0, 2.0)
    a, b = np.float32(2.5), np.float32(-0.75)
    z = oracle.map_lin_comb_f32ops(a, x, b, y, out_bf16=out_bf16)
    ref = (a * x + b * y).astype(np.float32)
    if out_bf16:
        ref = inputs.to_bf16_values(ref)
    assert np.array_equal(z, ref)
    for i in range(0, n, 37):
        p = Fraction(float(a)) * _fr(x[i])
        lo, hi = _neighbours_f32(np.float32(a) * x[i])
        assert _is_nearest(p, float(np.float32(a) * x[i]), lo, hi)
    # differs from the binary64-then-round reference somewhere (cancellation)
    z64r, _, _ = oracle.map_lin_comb(2.5, x, -0.75, y)
    if not out_bf16:
        assert not np.array_equal(z, z64r)


def test_map_gauss_sin_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    n = 400
    x = inputs.uniform_f32(12, 0, n, -2.0, 2.0)
    y = inputs.uniform_f32(12, 1, n, -2.0, 2.0)
    u = inputs.uniform_f32(12, 2, n, -2.0, 2.0)
    w = inputs.uniform_f32(12, 3, n, -2.0, 2.0)
    z, z64, t1, t2 = oracle.map_gauss_sin(x, y, u, w)
    for i in range(n):
        X, Y, U, W = (mpmath.mpf(float(v)) for v in (x[i], y[i], u[i], w[i]))
        T1 = X * mpmath.exp(-Y * Y)
        T2 = mpmath.sin(U) * W
        assert abs(float(T1) - t1[i]) <= 4e-16 * abs(float(T1)) + 1e-300
        assert abs(float(T2) - t2[i]) <= 4e-16 * abs(float(T2)) + 1e-300
        assert abs(float(T1 + T2) - z64[i]) <= 4e-16 * (abs(float(T1)) + abs(float(T2)))
    assert np.array_equal(z, z64.astype(np.float32))
    # the sampled variant agrees with the full one
    idx = np.array([0, 7, n - 1, 123], np.int64)
    s64, s1, s2 = oracle.map_gauss_sin_at(idx, x, y, u, w)
    assert np.array_equal(s64, z64[idx]) and np.array_equal(s1, t1[idx])


def test_map_gauss_sin_special_points():
    one = np.ones(1, np.float32)
    zero = np.zeros(1, np.float32)
    # y = 0, u = 0: z = x
    z, z64, _, _ = oracle.map_gauss_sin(one * 3, zero, zero, one * 5)
    assert z64[0] == 3.0
    # x = 0: z = sin(u) w ; sin is odd, so u -> -u flips the sign
    _, a, _, _ = oracle.map_gauss_sin(zero, one, one * 0.5, one * 2)
    _, b, _, _ = oracle.map_gauss_sin(zero, one, -one * 0.5, one * 2)
    assert a[0] == -b[0] and abs(a[0] - 2 * math.sin(0.5)) < 1e-15
    # w = 0: z = x exp(-y^2), even in y
    _, c, _, _ = oracle.map_gauss_sin(one * 2, one * 1.5, one, zero)
    _, d, _, _ = oracle.map_gauss_sin(one * 2, -one * 1.5, one, zero)
    assert c[0] == d[0] and abs(c[0] - 2 * math.exp(-2.25)) < 1e-15


# ----------------------------------------------------------------- superaccumulator

def _adversarial_doubles(rng, n):
    a = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
    a[: n // 4] = -a[n // 4: 2 * (n // 4)]  # exact cancellation pairs
    a = np.concatenate([a, [1e300, 1.0, -1e300, 2.0 ** -1074, -(2.0 ** -1060)]])
    rng.shuffle(a)
    return a


def test_superacc_matches_fsum_and_fractions():
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(1, 400))
        t = _adversarial_doubles(rng, n)
        exact = sum((Fraction(float(v)) for v in t), Fraction(0))
        want = float(exact)  # Fraction -> float rounds correctly
        assert oracle.exact_sum_f64(t) == want
        assert math.fsum(t) == want
    assert oracle.exact_sum_f64(np.zeros(0)) == 0.0
    assert oracle.exact_sum_f64(np.array([1.0, 2.0 ** -60, -1.0])) == 2.0 ** -60
    # ties inside the final rounding: 1 + 2^-53 is a tie -> 1; plus a sticky bit -> up
    assert oracle.exact_sum_f64(np.array([1.0, 2.0 ** -53])) == 1.0
    assert oracle.exact_sum_f64(np.array([1.0, 2.0 ** -53, 2.0 ** -100])) == 1.0 + 2.0 ** -52
    assert oracle.exact_sum_f64(np.array([-1.0, -(2.0 ** -53), -(2.0 ** -100)])) == -(1.0 + 2.0 ** -52)


# ----------------------------------------------------------------- FP sums / dots

def test_listing3b_dot_closed_form():
    g = _golden_kv("listing3b_dot_arange400.txt")
    x = np.arange(g["n"], dtype=np.float32)
    s, ab = oracle.dot_f32(x, x)
    assert s == g["exact"] and ab == g["exact"]
    assert g["exact"] == (g["n"] - 1) * g["n"] * (2 * g["n"] - 1) // 6
    # the golden serial binary32 value is what a one-accumulator loop gives
    acc = np.float32(0)
    for v in x * x:
        acc = np.float32(acc + v)
    assert int(acc) == g["serial_f32"]
    assert abs(g["serial_f32"] - g["exact"]) > 8 * 2.0 ** -24 * g["exact"]


def test_sum_and_dot_vs_exact():
    rng = np.random.default_rng(6)
    for trial in range(20):
        n = int(rng.integers(0, 3000))
        x = (rng.standard_normal(n) * np.exp(3 * rng.standard_normal(n))).astype(np.float32)
        y = rng.uniform(-1, 1, n).astype(np.float32)
        s, ab = oracle.sum_f32(x)
        ex = sum((Fraction(float(v)) for v in x), Fraction(0))
        exa = sum((abs(Fraction(float(v))) for v in x), Fraction(0))
        assert abs(Fraction(s) - ex) <= Fraction(abs(float(ex))) / 2 ** 52 + n * exa / 2 ** 104
        assert abs(Fraction(ab) - exa) <= exa / 2 ** 52
        assert oracle.exact_sum_f32(x) == float(ex)
        d, dab = oracle.dot_f32(x, y)
        exd = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))
        exda = sum((abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(x, y)), Fraction(0))
        assert abs(Fraction(d) - exd) <= Fraction(abs(float(exd))) / 2 ** 52 + n * exda / 2 ** 104
        assert oracle.exact_dot_f32(x, y) == float(exd)
        # operand order does not matter; a transposed operand would
        assert oracle.dot_f32(y, x)[0] == d


def test_sum_closed_forms_and_invariants():
    for n in (0, 1, 2, 3, 999, 1000, 4097):
        x = np.arange(n, dtype=np.float32)
        assert oracle.sum_f32(x)[0] == n * (n - 1) // 2
        alt = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
        assert oracle.sum_f32(alt)[0] == (n % 2)
        c = np.full(n, 0.375, np.float32)
        d = np.full(n, -6.0, np.float32)
        assert oracle.dot_f32(c, d)[0] == -2.25 * n
        assert oracle.dot_f32(alt, c)[0] == 0.375 * (n % 2)
    x = inputs.lognormal_signed_f32(7, 0, 100000)
    assert oracle.sum_f32(x)[0] + oracle.sum_f32(-x)[0] == 0.0
    perm = np.random.default_rng(8).permutation(x.size)
    assert abs(oracle.sum_f32(x[perm])[0] - oracle.exact_sum_f32(x)) <= 2.0 ** -52 * oracle.sum_f32(np.abs(x))[0]


def test_dot_segments_match_slices():
    lens = inputs.segment_lengths(nseg=50, seed=9, max_log2=10)
    off = np.concatenate([[0], np.cumsum(lens)])
    x = inputs.uniform_f32(9, 1, int(off[-1]))
    y = inputs.uniform_f32(9, 2, int(off[-1]))
    v, ab = oracle.dot_segments_f32(off, x, y)
    for s in range(50):
        a, b = off[s], off[s + 1]
        assert v[s] == oracle.dot_f32(x[a:b], y[a:b])[0]
        assert v[s] == pytest.approx(math.fsum((x[a:b].astype(np.float64) * y[a:b]).tolist()), rel=1e-15, abs=1e-300)
        assert ab[s] == oracle.dot_f32(x[a:b], y[a:b])[1]


# ----------------------------------------------------------------- integer / order reductions

def test_int_sums_exact():
    x = inputs.int_uniform_i32(13, 0, 100000)
    assert oracle.sum_i32_i64(x) == int(sum(int(v) for v in x))
    n = 70000
    assert oracle.sum_i32_i64(np.arange(n, dtype=np.int32)) == n * (n - 1) // 2
    big = np.full(5, 2 ** 31 - 1, np.int32)
    assert oracle.sum_i32_i64(big) == 5 * (2 ** 31 - 1)
    y = inputs.int_uniform_i32(13, 1, 1000)
    assert oracle.dot_i32_i64(x[:1000], y) == sum(int(a) * int(b) for a, b in zip(x[:1000], y))
    assert oracle.sum_i32_i64(np.zeros(0, np.int32)) == 0


def test_max_min_argmin_argmax():
    rng = np.random.default_rng(14)
    for n in (1, 2, 5, 100, 4099):
        x = rng.integers(-5, 5, n).astype(np.float32)  # many ties
        assert oracle.max_f32(x) == max(x.tolist()) and oracle.min_f32(x) == min(x.tolist())
        v, i = oracle.argmin_f32(x)
        assert i == int(np.argmin(x)) and v == x.min()  # numpy: first occurrence
        v, i = oracle.argmax_f32(x)
        assert i == int(np.argmax(x)) and v == x.max()
        assert oracle.argmin_f32(-x)[1] == int(np.argmax(x))
    # neutral for n = 0
    assert oracle.argmin_f32(np.zeros(0, np.float32)) == (float("inf"), 2 ** 63 - 1)
    assert oracle.argmax_f32(np.zeros(0, np.float32)) == (float("-inf"), 2 ** 63 - 1)
    # infinities are values like any other: the first one wins
    assert oracle.argmin_f32(np.full(3, np.inf, np.float32)) == (float("inf"), 0)
    assert oracle.max_f32(np.zeros(0, np.float32)) == float("-inf")
    # minima only at the last index; all equal -> index 0
    x = np.ones(1000, np.float32)
    x[-1] = 0
    assert oracle.argmin_f32(x)[1] == 999
    assert oracle.argmin_f32(np.ones(77, np.float32))[1] == 0


def test_argmin_recipe_first_chosen_index():
    n = 100000
    x = inputs.argmin_with_minima(15, n)
    pos = inputs.index_sample(15, 1, n // 100, n)
    v, i = oracle.argmin_f32(x)
    assert v == np.float32(-2.5) and i == int(pos.min())


# ----------------------------------------------------------------- scans (Sec. 3.2.6)

def test_scan_sum_against_library_and_exact():
    rng = np.random.default_rng(20)
    xi = rng.integers(-1000, 1000, 5000).astype(np.float32)  # exact in binary64
    incl, ab = oracle.scan_sum_f32(xi)
    assert np.array_equal(incl, np.cumsum(xi.astype(np.int64)).astype(np.float64))
    assert np.array_equal(ab, np.cumsum(np.abs(xi.astype(np.int64))).astype(np.float64))
    x = (rng.standard_normal(600) * np.exp(3 * rng.standard_normal(600))).astype(np.float32)
    incl, ab = oracle.scan_sum_f32(x)
    run = Fraction(0)
    for i in range(x.size):
        run += Fraction(float(x[i]))
        assert abs(Fraction(incl[i]) - run) <= Fraction(abs(float(run))) / 2 ** 52 + \
            (i + 1) * Fraction(ab[i]) / 2 ** 100
    # the last prefix is the reduction
    assert incl[-1] == oracle.sum_f32(x)[0]
    # a prefix that cancels a term 2^100 times larger: exact only with the compensation
    incl, ab = oracle.scan_sum_f32(np.array([2.0 ** 100, 1.0, -2.0 ** 100, 0.5], np.float32))
    assert list(incl) == [2.0 ** 100, 2.0 ** 100, 1.0, 1.5]
    assert list(ab) == [2.0 ** 100, 2.0 ** 100, 2.0 ** 101, 2.0 ** 101]
    assert oracle.scan_sum_f32(np.zeros(0, np.float32))[0].size == 0


def test_scan_int_inclusive_exclusive():
    x = inputs.int_uniform_i32(21, 0, 10000)
    inc = oracle.scan_sum_i32_i64(x)
    exc = oracle.scan_sum_i32_i64(x, exclusive=True)
    assert np.array_equal(inc, np.cumsum(x.astype(np.int64)))
    assert exc[0] == 0 and np.array_equal(exc[1:], inc[:-1])
    n = 3000
    assert np.array_equal(oracle.scan_sum_i32_i64(np.arange(n, dtype=np.int32)),
                          np.arange(n, dtype=np.int64) * (np.arange(n) + 1) // 2)


def test_scan_max_against_library():
    x = np.random.default_rng(22).standard_normal(4000).astype(np.float32)
    assert np.array_equal(oracle.scan_max_f32(x), np.maximum.accumulate(x))
    assert oracle.scan_max_f32(np.array([np.float32(-np.inf)]))[0] == -np.inf


def test_scan_affine_composition():
    """Prefix compositions of v -> a v + b (mod 2^32): the composed map applied
    to a point equals iterating the maps one by one; a = 1 reduces to prefix
    sums of b and b = 0 to prefix products of a."""
    rng = np.random.default_rng(23)
    n = 3000
    a = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    out = oracle.scan_affine_u32(a, b)
    A, B = (out >> np.uint64(32)).astype(np.uint64), (out & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    for v0 in (0, 1, 0x9E3779B9, 2 ** 32 - 1):
        v = v0
        for i in range(n):
            v = (int(a[i]) * v + int(b[i])) % 2 ** 32
            assert (int(A[i]) * v0 + int(B[i])) % 2 ** 32 == v
    ones = np.ones(n, np.uint32)
    out = oracle.scan_affine_u32(ones, b)
    assert np.all(out >> np.uint64(32) == 1)
    assert np.array_equal(out & np.uint64(0xFFFFFFFF), np.cumsum(b.astype(np.uint64)) % 2 ** 32)
    out = oracle.scan_affine_u32(a, np.zeros(n, np.uint32))
    assert np.all(out & np.uint64(0xFFFFFFFF) == 0)
    assert np.array_equal(out >> np.uint64(32), np.array(_cumprod_mod32(a), np.uint64))


def _cumprod_mod32(a):
    r, p = [], 1
    for v in a:
        p = p * int(v) % 2 ** 32
        r.append(p)
    return r

