"""ORACLE -- test infrastructure only.

ctypes binding of ``oracle.c``: the plain single-threaded CPU statement of what
the map / map-reduce path computes (Sec. 3.2.4 and Sec. 3.2.5 of Klockner et al.,
"GPU Scripting and Code Generation with PyCUDA"), in binary64.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library (``paper_1304_5553_gb300``) never
does, and this package imports nothing from the library.

Every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_DIR, "_build")
_SRC = os.path.join(_DIR, "oracle.c")
LIB_PATH = os.path.join(_BUILD, "liboracle.so")


def build_cmd():
    return [os.environ.get("CC", "gcc"), "-O2", "-std=gnu11", "-ffp-contract=off",
            "-fno-fast-math", "-fPIC", "-shared", "-o", LIB_PATH, _SRC, "-lm"]


def build(force=False):
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or \
            os.path.getmtime(LIB_PATH) < os.path.getmtime(_SRC):
        p = subprocess.run(build_cmd(), capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + p.stderr)
    return LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        # ORACLE_LIB: load another build of oracle.c instead (the mutation test
        # uses it to check that the pins catch planted mistakes)
        path = os.environ.get("ORACLE_LIB")
        if not path:
            build()
            path = LIB_PATH
        lib = ctypes.CDLL(path)
        i64, f64, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        sig = {
            "orc_round_bf16": (f64, [f64]),
            "orc_round_f32": (ctypes.c_float, [f64]),
            "orc_map_scale": (None, [i64, f64, vp, vp, vp]),
            "orc_map_add": (None, [i64, vp, vp, vp, vp]),
            "orc_map_lin_comb": (None, [i64, f64, vp, f64, vp, ctypes.c_int, vp, vp, vp]),
            "orc_map_lin_comb_f32ops": (None, [i64, ctypes.c_float, vp, ctypes.c_float, vp,
                                               ctypes.c_int, vp]),
            "orc_map_gauss_sin": (None, [i64, vp, vp, vp, vp, vp, vp, vp, vp]),
            "orc_map_gauss_sin_at": (None, [i64, vp, vp, vp, vp, vp, vp, vp, vp]),
            "orc_sum_f32": (f64, [i64, vp, vp]),
            "orc_dot_f32": (f64, [i64, vp, vp, vp]),
            "orc_dot_segments_f32": (None, [i64, vp, vp, vp, vp, vp]),
            "orc_sum_i32_i64": (i64, [i64, vp]),
            "orc_dot_i32_i64": (i64, [i64, vp, vp]),
            "orc_max_f32": (ctypes.c_float, [i64, vp]),
            "orc_min_f32": (ctypes.c_float, [i64, vp]),
            "orc_argmin_f32": (None, [i64, vp, vp, vp]),
            "orc_argmax_f32": (None, [i64, vp, vp, vp]),
            "orc_scan_sum_f32": (None, [i64, vp, vp, vp]),
            "orc_scan_sum_i32_i64": (None, [i64, vp, ctypes.c_int, vp]),
            "orc_scan_max_f32": (None, [i64, vp, vp]),
            "orc_scan_affine_u32": (None, [i64, vp, vp, vp]),
            "orc_exact_sum_f64": (f64, [i64, vp]),
            "orc_exact_dot_f32": (f64, [i64, vp, vp]),
            "orc_exact_sum_f32": (f64, [i64, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data


# ------------------------------------------------------------------ rounding

def round_bf16(d: float) -> float:
    """binary64 -> nearest bfloat16, ties to even (one rounding)."""
    return float(_load().orc_round_bf16(float(d)))


def round_f32(d: float) -> float:
    return float(_load().orc_round_f32(float(d)))


# ------------------------------------------------------------------ maps

def map_scale(s, x):
    """Listing 1/2: z = s*x.  Returns (z binary32, z binary64)."""
    x = _f32(x)
    z, z64 = np.empty_like(x), np.empty(x.size, np.float64)
    _load().orc_map_scale(x.size, float(s), _ptr(x), _ptr(z), _ptr(z64))
    return z, z64


def map_add(x, y):
    """Listing 4: z = x + y.  Returns (z binary32, z binary64)."""
    x, y = _f32(x), _f32(y)
    assert x.size == y.size
    z, z64 = np.empty_like(x), np.empty(x.size, np.float64)
    _load().orc_map_add(x.size, _ptr(x), _ptr(y), _ptr(z), _ptr(z64))
    return z, z64


def map_lin_comb(a, x, b, y, out_bf16=False):
    """Listing 3a: z = a*x + b*y.  Returns (z, z64, |a x| + |b y|); z holds the
    binary32 or bfloat16 (as binary32 values) storage result."""
    x, y = _f32(x), _f32(y)
    assert x.size == y.size
    z = np.empty_like(x)
    z64, tab = np.empty(x.size, np.float64), np.empty(x.size, np.float64)
    _load().orc_map_lin_comb(x.size, float(a), _ptr(x), float(b), _ptr(y), int(out_bf16),
                             _ptr(z), _ptr(z64), _ptr(tab))
    return z, z64, tab


def map_lin_comb_f32ops(a, x, b, y, out_bf16=False):
    """Listing 3a evaluated as binary32 C source (each operation rounded, no
    contraction); bfloat16 output rounds the binary32 value on the store."""
    x, y = _f32(x), _f32(y)
    assert x.size == y.size
    z = np.empty_like(x)
    _load().orc_map_lin_comb_f32ops(x.size, float(a), _ptr(x), float(b), _ptr(y), int(out_bf16),
                                    _ptr(z))
    return z


def map_gauss_sin(x, y, u, w):
    """z = x*exp(-y*y) + sin(u)*w.  Returns (z, z64, t1, t2) with the binary64
    addends t1 = x exp(-y^2), t2 = sin(u) w."""
    x, y, u, w = _f32(x), _f32(y), _f32(u), _f32(w)
    n = x.size
    assert y.size == n and u.size == n and w.size == n
    z = np.empty_like(x)
    z64, t1, t2 = (np.empty(n, np.float64) for _ in range(3))
    _load().orc_map_gauss_sin(n, _ptr(x), _ptr(y), _ptr(u), _ptr(w), _ptr(z), _ptr(z64),
                              _ptr(t1), _ptr(t2))
    return z, z64, t1, t2


def map_gauss_sin_at(idx, x, y, u, w):
    """The four-input map at the given indices only: (z64, t1, t2)."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.size
    z64, t1, t2 = (np.empty(k, np.float64) for _ in range(3))
    _load().orc_map_gauss_sin_at(k, _ptr(idx), _ptr(_f32(x)), _ptr(_f32(y)), _ptr(_f32(u)),
                                 _ptr(_f32(w)), _ptr(z64), _ptr(t1), _ptr(t2))
    return z64, t1, t2


# ------------------------------------------------------------------ reductions

def sum_f32(x):
    """(sum x in binary64 (compensated), sum |x|)."""
    x = _f32(x)
    a = ctypes.c_double()
    s = _load().orc_sum_f32(x.size, _ptr(x), ctypes.addressof(a))
    return s, a.value


def dot_f32(x, y):
    """Listing 3b: (sum x*y in binary64 (compensated), sum |x*y|)."""
    x, y = _f32(x), _f32(y)
    assert x.size == y.size
    a = ctypes.c_double()
    s = _load().orc_dot_f32(x.size, _ptr(x), _ptr(y), ctypes.addressof(a))
    return s, a.value


def dot_segments_f32(offsets, x, y):
    """Per-segment dot products; returns (values, sum |terms| per segment)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = off.size - 1
    x, y = _f32(x), _f32(y)
    assert off[-1] <= x.size and off[-1] <= y.size
    out, ab = np.empty(nseg, np.float64), np.empty(nseg, np.float64)
    _load().orc_dot_segments_f32(nseg, _ptr(off), _ptr(x), _ptr(y), _ptr(out), _ptr(ab))
    return out, ab


def sum_i32_i64(x):
    x = np.ascontiguousarray(x, dtype=np.int32)
    return int(_load().orc_sum_i32_i64(x.size, _ptr(x)))


def dot_i32_i64(x, y):
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    return int(_load().orc_dot_i32_i64(x.size, _ptr(x), _ptr(y)))


def max_f32(x):
    x = _f32(x)
    return float(_load().orc_max_f32(x.size, _ptr(x)))


def min_f32(x):
    x = _f32(x)
    return float(_load().orc_min_f32(x.size, _ptr(x)))


def argmin_f32(x):
    x = _f32(x)
    v, i = ctypes.c_float(), ctypes.c_int64()
    _load().orc_argmin_f32(x.size, _ptr(x), ctypes.addressof(v), ctypes.addressof(i))
    return float(v.value), int(i.value)


def argmax_f32(x):
    x = _f32(x)
    v, i = ctypes.c_float(), ctypes.c_int64()
    _load().orc_argmax_f32(x.size, _ptr(x), ctypes.addressof(v), ctypes.addressof(i))
    return float(v.value), int(i.value)


# ------------------------------------------------------------------ scans

def scan_sum_f32(x):
    """Inclusive prefix sums in binary64 (compensated) and prefix sums of |x|."""
    x = _f32(x)
    incl, ab = np.empty(x.size, np.float64), np.empty(x.size, np.float64)
    _load().orc_scan_sum_f32(x.size, _ptr(x), _ptr(incl), _ptr(ab))
    return incl, ab


def scan_sum_i32_i64(x, exclusive=False):
    x = np.ascontiguousarray(x, dtype=np.int32)
    out = np.empty(x.size, np.int64)
    _load().orc_scan_sum_i32_i64(x.size, _ptr(x), int(exclusive), _ptr(out))
    return out


def scan_max_f32(x):
    x = _f32(x)
    out = np.empty_like(x)
    _load().orc_scan_max_f32(x.size, _ptr(x), _ptr(out))
    return out


def scan_affine_u32(a, b):
    """Prefix compositions of v -> a[k] v + b[k] mod 2^32, packed A << 32 | B."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    assert a.size == b.size
    out = np.empty(a.size, np.uint64)
    _load().orc_scan_affine_u32(a.size, _ptr(a), _ptr(b), _ptr(out))
    return out


def exact_sum_f64(t):
    t = np.ascontiguousarray(t, dtype=np.float64)
    return float(_load().orc_exact_sum_f64(t.size, _ptr(t)))


def exact_sum_f32(x):
    x = _f32(x)
    return float(_load().orc_exact_sum_f32(x.size, _ptr(x)))


def exact_dot_f32(x, y):
    x, y = _f32(x), _f32(y)
    return float(_load().orc_exact_dot_f32(x.size, _ptr(x), _ptr(y)))


# ------------------------------------------------------------------ sharded reductions
# A map-reduce over [0, n) cut into contiguous shards.  Sec. 3.2.5 defines the
# reduction by an associative reduce operation whose neutral element is an
# identity, so the reduction of the whole range equals the operation applied,
# in shard order, to the reductions of the shards.  A shard's partial is the
# reductions above applied to the shard's own elements, with indices shifted by
# the shard's first global index i0; combine_partials folds them in order.

SHARD_KINDS = ("sum_i32_i64", "max_f32", "argmin_f32", "argmax_f32", "sum_f32", "dot_f32")
_NO_INDEX = 2 ** 63 - 1  # index of the argmin / argmax neutral element


def shard_partial(kind, arrays, i0):
    """Partial of one shard: `arrays` hold the shard's elements, the first of
    which is element i0 of the whole range.  sum_i32_i64: int; max_f32: float;
    argmin_f32 / argmax_f32: (value, global index); sum_f32 / dot_f32: (binary64
    sum, sum of |terms|)."""
    if kind == "sum_i32_i64":
        return sum_i32_i64(arrays[0])
    if kind == "max_f32":
        return max_f32(arrays[0])
    if kind in ("argmin_f32", "argmax_f32"):
        v, i = (argmin_f32 if kind == "argmin_f32" else argmax_f32)(arrays[0])
        return v, (i if i == _NO_INDEX else i0 + i)
    if kind == "sum_f32":
        return sum_f32(arrays[0])
    if kind == "dot_f32":
        return dot_f32(arrays[0], arrays[1])
    raise ValueError(kind)


def combine_partials(kind, parts):
    """Fold the shards' partials in shard order with the reduction's own
    operation (an empty list gives the neutral element)."""
    import math
    if kind == "sum_i32_i64":
        return sum(parts)
    if kind == "max_f32":
        m = -math.inf
        for p in parts:
            if p > m:
                m = p
        return m
    if kind in ("argmin_f32", "argmax_f32"):
        sign = 1.0 if kind == "argmin_f32" else -1.0
        best = (sign * math.inf, _NO_INDEX)
        for v, i in parts:
            if sign * v < sign * best[0] or (v == best[0] and i < best[1]):
                best = (v, i)
        return best
    if kind in ("sum_f32", "dot_f32"):
        return math.fsum(p[0] for p in parts), sum(p[1] for p in parts)
    raise ValueError(kind)
