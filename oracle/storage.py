"""ORACLE -- test infrastructure only: the map and map-reduce of Sec. 3.2.4 and
Sec. 3.2.5 over the storage types of the argument spec that the binary32 /
bfloat16 functions of ``oracle.c`` do not cover (the C type strings of Sec. 3.1:
binary16 ``__half``, binary64 ``double``, ``int`` and ``long long``).

Each function is the plain definition written out with numpy's IEEE
arithmetic: C evaluation of the statement in source order, one rounding per
operation (no contraction), a binary16 store rounding the binary32 value once
to nearest even, integer arithmetic in two's complement.  Sums are exact
(``math.fsum`` of values whose products are exact in binary64), so the tests
judge any association order of the GPU's tree against them.

Only ``tests/`` may import this module; it imports nothing from the library.
Pinned by ``tests/test_oracle_storage_pins.py`` (exact rationals with a
rounding written from the IEEE 754 definition, the binary16 format's own
boundary values, closed forms and big-integer wrap-around).
"""
from __future__ import annotations

import math

import numpy as np


def round_f16(v):
    """binary32 (or binary64) values -> binary16, round to nearest, ties to even."""
    with np.errstate(over="ignore"):
        return np.asarray(v).astype(np.float16)


def lin_comb_f16(a, x16, b, y16):
    """z = a*x + b*y with binary16 x, y, binary32 scalars a, b: x and y widen
    exactly to binary32, RN32(RN32(a x) + RN32(b y)), then one rounding to binary16."""
    x = np.asarray(x16, np.float16).astype(np.float32)
    y = np.asarray(y16, np.float16).astype(np.float32)
    with np.errstate(all="ignore"):
        z32 = np.float32(a) * x + np.float32(b) * y
    return z32.astype(np.float16)


def lin_comb_f64(a, x, b, y):
    """z = RN64(RN64(a x) + RN64(b y)): binary64 source order, no contraction."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    with np.errstate(all="ignore"):
        return np.float64(a) * x + np.float64(b) * y


def lin_comb_int(a, x, b, y, bits):
    """z = a*x + b*y in two's-complement integers of the given width (wrap-around)."""
    dt = {32: np.int32, 64: np.int64}[bits]
    x = np.asarray(x, dt)
    y = np.asarray(y, dt)
    with np.errstate(over="ignore"):
        return (dt(a) * x + dt(b) * y).astype(dt)


def add_f16_f64_to_f32(x16, y64):
    """z = x + y with binary16 x, binary64 y and a binary32 z (C promotion: x
    widens exactly to binary64, the sum rounds in binary64, the store to binary32)."""
    s = np.asarray(x16, np.float16).astype(np.float64) + np.asarray(y64, np.float64)
    return s.astype(np.float32)


def sum_exact(t):
    """(S, sum |t|): the exact sum of binary64 values rounded once (fsum), and the
    absolute sum the tolerances scale with."""
    t = np.asarray(t, np.float64).ravel()
    return math.fsum(t.tolist()), math.fsum(np.abs(t).tolist())


def dot_exact_f16(x16, y16):
    """(S, sum |x y|) for binary16 vectors: every product of two binary16 values is
    exact in binary64 (22 significant bits), so fsum gives the exact dot product
    rounded once."""
    p = np.asarray(x16, np.float16).astype(np.float64) * np.asarray(y16, np.float16).astype(
        np.float64)
    return sum_exact(p)


def sum_int(x):
    """Exact integer sum (Python integers; no wrap)."""
    return int(sum(int(v) for v in np.asarray(x).ravel().tolist()))


def max_value(x, empty):
    """Largest element by the C comparison a > b (``empty`` for no elements)."""
    r = empty
    for v in np.asarray(x).ravel().tolist():
        if v > r:
            r = v
    return r


def min_value(x, empty):
    """Smallest element by the C comparison a < b (``empty`` for no elements)."""
    r = empty
    for v in np.asarray(x).ravel().tolist():
        if v < r:
            r = v
    return r


def map_u8_add_index(x, idx, shift):
    """z[i] = x[i] + (unsigned char)(i >> shift) stored to unsigned char, at the
    indices idx (64-bit): C promotes both operands to int, the store keeps the
    low 8 bits."""
    x = np.asarray(x, np.int64)
    idx = np.asarray(idx, np.int64)
    return ((x + ((idx >> shift) & 255)) & 255).astype(np.uint8)


# ------------------------------------------------------------------ scans
# Parallel prefix scans (Sec. 3.2.6) over these storage types, by their plain
# definitions: out[i] combines x[0], ..., x[i] (inclusive) or x[0], ..., x[i-1]
# (exclusive, the neutral element at i = 0) in index order.

def scan_sum_int(x, exclusive=False):
    """Prefix sums of integer values, exact.  The inputs are kept small enough
    (n * max|x| < 2^62) that no prefix leaves int64, so the running sum in
    int64 is the exact one; larger inputs are refused."""
    x = np.asarray(x).ravel().astype(np.int64)
    if x.size and int(np.abs(x).max()) * x.size >= 2 ** 62:
        raise ValueError("prefix sums could leave int64")
    inc = np.cumsum(x, dtype=np.int64)
    if not exclusive:
        return inc
    out = np.zeros_like(inc)
    out[1:] = inc[:-1]
    return out


def scan_count_nonzero(x, exclusive=True):
    """Prefix counts of the nonzero elements (the output offsets of a stream
    compaction when exclusive)."""
    return scan_sum_int(np.asarray(x).ravel() != 0, exclusive)


def scan_max(x, neutral):
    """Prefix maxima by the C rule acc = acc > v ? acc : v, starting from
    ``neutral``, in index order (values widened exactly to binary64)."""
    out = np.empty(np.asarray(x).size, np.float64)
    acc = float(neutral)
    for k, v in enumerate(np.asarray(x).ravel().astype(np.float64).tolist()):
        acc = acc if acc > v else v
        out[k] = acc
    return out
