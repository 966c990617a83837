"""Pins of ``oracle/storage.py`` (binary16, binary64 and integer storage of the
argument spec, Sec. 3.1 type strings; map Sec. 3.2.4, map-reduce Sec. 3.2.5).

Nothing here re-calls the oracle's own arithmetic: the expected values come
from exact rational arithmetic rounded by ``_round`` below (round to nearest,
ties to even, written from the IEEE 754 definition of a binary format with p
significand bits and exponent range [emin, emax]), from the binary16 format's
boundary values, from closed forms, and from Python's unbounded integers.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import storage

F16 = (11, -14, 15)
F32 = (24, -126, 127)
F64 = (53, -1022, 1023)
INF = float("inf")


def _round(q, fmt):
    """Round the rational q to the binary format fmt = (p, emin, emax), ties to even;
    overflow gives +-inf."""
    p, emin, emax = fmt
    q = Fraction(q)
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, emin)  # below the normal range the quantum stays 2^(emin - p + 1)
    quantum = Fraction(2) ** (e - p + 1)
    m = a / quantum
    k = m.numerator // m.denominator
    rem = m - k
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and k % 2 == 1):
        k += 1
    r = k * quantum
    if r >= Fraction(2) ** (emax + 1):
        return sign * INF
    return sign * r


def _f(q):
    return float(q) if not isinstance(q, float) else q


# --- the round-to-nearest reference itself, on the formats' defining values ----------

def test_round_reference_on_format_boundaries():
    # binary16: largest finite (2 - 2^-10) 2^15, overflow threshold 65520, smallest
    # subnormal 2^-24; binary32 and binary64 largest finite values
    assert _round(65504, F16) == 65504
    assert _round(Fraction(65519), F16) == 65504
    assert _round(65520, F16) == INF
    assert _round(Fraction(1, 2 ** 24), F16) == Fraction(1, 2 ** 24)
    assert _round(Fraction(1, 2 ** 25), F16) == 0                       # tie -> even (0)
    assert _round(Fraction(3, 2 ** 25), F16) == Fraction(1, 2 ** 23)     # tie -> even (2 quanta)
    assert _round(1 + Fraction(1, 2 ** 11), F16) == 1                     # tie -> even
    assert _round(1 + Fraction(3, 2 ** 11), F16) == 1 + Fraction(1, 2 ** 9)
    assert _f(_round((2 - Fraction(1, 2 ** 23)) * Fraction(2) ** 127, F32)) == float(np.finfo(np.float32).max)
    assert _f(_round((2 - Fraction(1, 2 ** 52)) * Fraction(2) ** 1023, F64)) == float(np.finfo(np.float64).max)
    assert _f(_round(Fraction(1, 3), F64)) == 1 / 3


# --- binary16 rounding ----------------------------------------------------------------

def test_round_f16_boundary_values():
    v = np.array([65504, 65519.996, 65520, -65520, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -25,
                  1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 0.1], np.float32)
    want = [65504, 65504, INF, -INF, 2.0 ** -24, 0.0, 2.0 ** -23, 1.0, 1 + 2.0 ** -9,
            _f(_round(Fraction(float(np.float32(0.1))), F16))]
    got = storage.round_f16(v).astype(np.float64)
    assert got.tolist() == want


def test_round_f16_random_against_rationals():
    rng = np.random.default_rng(11)
    # magnitudes from deep subnormal to past the overflow threshold
    v = (rng.uniform(-1, 1, 3000) * 2.0 ** rng.uniform(-27, 17, 3000)).astype(np.float32)
    got = storage.round_f16(v).astype(np.float64)
    want = [_f(_round(Fraction(float(t)), F16)) for t in v]
    assert got.tolist() == want


# --- maps --------------------------------------------------------------------------------

def _f16_values(rng, n, lo, hi):
    return rng.uniform(lo, hi, n).astype(np.float16)


@pytest.mark.parametrize("a,b", [(2.5, -0.75), (0.1, 3.3)])
def test_lin_comb_f16_against_rationals(a, b):
    rng = np.random.default_rng(12)
    x = _f16_values(rng, 1500, -2, 2)
    y = _f16_values(rng, 1500, -2, 2)
    a32, b32 = float(np.float32(a)), float(np.float32(b))
    got = storage.lin_comb_f16(a, x, b, y).astype(np.float64)
    for k in range(len(x)):
        ax = _round(Fraction(a32) * Fraction(float(x[k])), F32)
        by = _round(Fraction(b32) * Fraction(float(y[k])), F32)
        z = _round(_round(ax + by, F32), F16)
        assert got[k] == _f(z), k


def test_lin_comb_f64_against_rationals():
    rng = np.random.default_rng(13)
    n = 1500
    x = rng.uniform(-2, 2, n) * 2.0 ** rng.integers(-30, 30, n)
    y = rng.uniform(-2, 2, n)
    a, b = 2.5, -0.7
    y[::3] = a * x[::3] / 0.7  # heavy cancellation in every third element
    got = storage.lin_comb_f64(a, x, b, y)
    for k in range(n):
        ax = _round(Fraction(a) * Fraction(float(x[k])), F64)
        by = _round(Fraction(b) * Fraction(float(y[k])), F64)
        assert got[k] == _f(_round(ax + by, F64)), k


@pytest.mark.parametrize("bits", [32, 64])
def test_lin_comb_int_wraps_like_twos_complement(bits):
    rng = np.random.default_rng(14)
    lim = 2 ** (bits - 1)
    dt = np.int32 if bits == 32 else np.int64
    x = rng.integers(-lim, lim, 2000, dtype=dt)
    y = rng.integers(-lim, lim, 2000, dtype=dt)
    a, b = 3, -7
    got = storage.lin_comb_int(a, x, b, y, bits)
    for k in range(len(x)):
        v = (a * int(x[k]) + b * int(y[k])) % (2 ** bits)
        if v >= lim:
            v -= 2 ** bits
        assert int(got[k]) == v, k


def test_mixed_promotion_against_rationals():
    rng = np.random.default_rng(15)
    x = _f16_values(rng, 1500, -2, 2)
    y = rng.uniform(-1, 1, 1500) * 2.0 ** rng.integers(-40, 10, 1500)
    got = storage.add_f16_f64_to_f32(x, y).astype(np.float64)
    for k in range(len(x)):
        s = _round(Fraction(float(x[k])) + Fraction(float(y[k])), F64)
        assert got[k] == _f(_round(s, F32)), k


# --- sums ----------------------------------------------------------------------------------

def test_sum_exact_closed_form_and_sign():
    n = 100001
    t = np.arange(n, dtype=np.float64)
    s, ab = storage.sum_exact(t)
    assert s == n * (n - 1) // 2 and ab == s
    s2, _ = storage.sum_exact(-t)
    assert s2 == -s


def test_sum_exact_against_rationals():
    rng = np.random.default_rng(16)
    t = rng.uniform(-1, 1, 2000) * 2.0 ** rng.integers(-60, 60, 2000)
    s, ab = storage.sum_exact(t)
    exact = sum(Fraction(float(v)) for v in t)
    assert s == _f(_round(exact, F64))
    assert ab == _f(_round(sum(abs(Fraction(float(v))) for v in t), F64))


def test_dot_exact_f16_against_rationals():
    rng = np.random.default_rng(17)
    x = _f16_values(rng, 2000, -2, 2)
    y = _f16_values(rng, 2000, -2, 2)
    s, ab = storage.dot_exact_f16(x, y)
    exact = sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(x, y))
    assert s == _f(_round(exact, F64))
    absum = sum(abs(Fraction(float(p)) * Fraction(float(q))) for p, q in zip(x, y))
    assert ab == _f(_round(absum, F64))


def test_sum_int_closed_form():
    n = 70001
    assert storage.sum_int(np.arange(n, dtype=np.int64)) == n * (n - 1) // 2
    big = np.full(5, 2 ** 62, np.int64)
    assert storage.sum_int(big) == 5 * 2 ** 62  # no wrap-around


def test_extrema_brute_force():
    rng = np.random.default_rng(18)
    for n in (1, 2, 7, 300):
        x = rng.integers(-50, 50, n)
        assert storage.max_value(x, -10 ** 9) == sorted(x.tolist())[-1]
        assert storage.min_value(x, 10 ** 9) == sorted(x.tolist())[0]
        d = rng.uniform(-1, 1, n)
        assert storage.min_value(d, float("inf")) == sorted(d.tolist())[0]
    # the neutral value comes back for no elements; it does not win a tie
    assert storage.max_value(np.array([], np.int32), -7) == -7
    assert storage.min_value(np.array([5, 5]), 5) == 5


def test_map_u8_add_index_hand_values():
    # worked by hand: 200 + ((2^32 + 5) >> 20 = 4096 -> low byte 0) = 200;
    # 250 + 10 = 260 -> 4; 255 + ((2^31 + 3 * 2^20) >> 20 = 2051 -> 3) = 258 -> 2
    got = storage.map_u8_add_index([200, 250, 255], [2 ** 32 + 5, 10 << 20, 2 ** 31 + 3 * 2 ** 20], 20)
    assert got.tolist() == [200, 4, 2]
    # brute force against Python integers on indices around 2^31 and 2^32
    rng = np.random.default_rng(19)
    idx = np.concatenate([np.arange(2 ** 31 - 3000, 2 ** 31 + 3000),
                          np.arange(2 ** 32 - 3000, 2 ** 32 + 3000)])
    x = rng.integers(0, 256, idx.size)
    got = storage.map_u8_add_index(x, idx, 20)
    assert all(int(g) == (int(a) + ((int(i) >> 20) % 256)) % 256 for g, a, i in zip(got, x, idx))


def test_scan_sum_int_brute_force_and_closed_form():
    # prefix sums of 1..n: k(k+1)/2; exclusive: (k-1)k/2
    n = 1000
    inc = storage.scan_sum_int(np.arange(1, n + 1))
    exc = storage.scan_sum_int(np.arange(1, n + 1), exclusive=True)
    k = np.arange(1, n + 1)
    assert inc.tolist() == (k * (k + 1) // 2).tolist()
    assert exc.tolist() == ((k - 1) * k // 2).tolist()
    # brute force against Python integers on signed values near 2^40
    rng = np.random.default_rng(23)
    x = rng.integers(-(2 ** 40), 2 ** 40, 3001)
    for ex in (False, True):
        got = storage.scan_sum_int(x, exclusive=ex).tolist()
        want = [sum(int(v) for v in x[: i + (0 if ex else 1)]) for i in range(0, 3001, 97)]
        assert got[::97] == want
    assert storage.scan_sum_int([]).size == 0
    with pytest.raises(ValueError):
        storage.scan_sum_int(np.full(4, 2 ** 61))


def test_scan_count_nonzero_hand_values():
    assert storage.scan_count_nonzero([0, 3, 0, 0, 255, 1]).tolist() == [0, 0, 1, 1, 1, 2]
    assert storage.scan_count_nonzero([0, 3, 0, 0, 255, 1], exclusive=False).tolist() == [
        0, 1, 1, 1, 2, 3]


def test_scan_max_brute_force():
    # worked by hand, with a tie and the neutral element kept until a larger value
    got = storage.scan_max([-5.0, -7.0, 2.0, 2.0, 1.5, 3.25], -np.inf).tolist()
    assert got == [-5.0, -5.0, 2.0, 2.0, 2.0, 3.25]
    assert storage.scan_max([-1.0], 0.0).tolist() == [0.0]
    rng = np.random.default_rng(29)
    x = rng.standard_normal(2000).astype(np.float16)
    got = storage.scan_max(x, -np.inf)
    assert all(got[i] == max(float(v) for v in x[: i + 1]) for i in range(0, 2000, 37))


# planted mistakes in the storage oracle: each must make one of the pins above fail
def _f16_in_binary64(a, x16, b, y16):
    x = np.asarray(x16, np.float16).astype(np.float64)
    y = np.asarray(y16, np.float16).astype(np.float64)
    return (a * x + b * y).astype(np.float16)


def _f16_truncating(v):
    # round toward zero instead of to nearest even
    v = np.asarray(v, np.float64)
    with np.errstate(over="ignore"):
        r = v.astype(np.float16).astype(np.float64)
    over = np.abs(r) > np.abs(v)
    r[over] = np.nextafter(r[over].astype(np.float16), np.float16(0)).astype(np.float64)
    return r.astype(np.float16)


_MUTANTS = {
    "binary16 map computed in binary64": ("lin_comb_f16", _f16_in_binary64),
    "binary16 store truncates": ("round_f16", _f16_truncating),
    "binary64 map sign": ("lin_comb_f64", lambda a, x, b, y: np.float64(a) * np.asarray(x)
                          - np.float64(b) * np.asarray(y)),
    "binary64 map contracted": ("lin_comb_f64", lambda a, x, b, y: (
        np.longdouble(a) * np.asarray(x, np.longdouble)
        + np.longdouble(b) * np.asarray(y, np.longdouble)).astype(np.float64)),
    "integer map saturates": ("lin_comb_int", lambda a, x, b, y, bits: np.clip(
        a * np.asarray(x, np.float64) + b * np.asarray(y, np.float64),
        -2.0 ** (bits - 1), 2.0 ** (bits - 1) - 1).astype({32: np.int32, 64: np.int64}[bits])),
    "promotion to binary32 first": ("add_f16_f64_to_f32", lambda x16, y64: (
        np.asarray(x16, np.float16).astype(np.float32) + np.asarray(y64).astype(np.float32))),
    "sum drops the last term": ("sum_exact", lambda t: (
        math.fsum(np.asarray(t, np.float64).ravel()[:-1].tolist()),
        math.fsum(np.abs(np.asarray(t, np.float64)).ravel().tolist()))),
    "u8 map without the index": ("map_u8_add_index", lambda x, idx, shift: (
        np.asarray(x, np.int64) & 255).astype(np.uint8)),
    "min keeps the first element": ("min_value", lambda x, empty: (
        np.asarray(x).ravel().tolist() or [empty])[0]),
    "scan: exclusive taken as inclusive": ("scan_sum_int", lambda x, exclusive=False: np.cumsum(
        np.asarray(x).ravel().astype(np.int64))),
    "scan: prefix one element late": ("scan_sum_int", lambda x, exclusive=False: (
        lambda inc: np.concatenate([[0, 0], inc[:-2]]) if exclusive else np.concatenate(
            [[0], inc[:-1]]))(np.cumsum(np.asarray(x).ravel().astype(np.int64)))),
    "scan max ignores the neutral": ("scan_max", lambda x, neutral: np.maximum.accumulate(
        np.asarray(x, np.float64).ravel())),
    "count counts zeros": ("scan_count_nonzero", lambda x, exclusive=True: storage.scan_sum_int(
        np.asarray(x).ravel() == 0, exclusive)),
}

_PINS = [test_round_f16_boundary_values, test_round_f16_random_against_rationals,
         lambda: test_lin_comb_f16_against_rationals(0.1, 3.3),
         test_lin_comb_f64_against_rationals,
         lambda: test_lin_comb_int_wraps_like_twos_complement(32),
         test_mixed_promotion_against_rationals, test_sum_exact_closed_form_and_sign,
         test_sum_exact_against_rationals, test_map_u8_add_index_hand_values,
         test_extrema_brute_force, test_scan_sum_int_brute_force_and_closed_form,
         test_scan_count_nonzero_hand_values, test_scan_max_brute_force]


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_catch_planted_mistakes(name, monkeypatch):
    fn, bad = _MUTANTS[name]
    monkeypatch.setattr(storage, fn, bad)
    failed = False
    for pin in _PINS:
        try:
            pin()
        except AssertionError:
            failed = True
    assert failed, "the pins did not catch: " + name
