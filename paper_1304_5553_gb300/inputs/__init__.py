"""Seeded synthetic inputs for the map / map-reduce workloads.

This module only draws input values; it holds none of the method's arithmetic.
Every value is a pure function of (seed, stream, index) -- see ``gen.c`` for the
exact definitions -- so the tests, the oracle checks and the benchmark all see
the same bits for the same recipe, and any slice can be regenerated alone.

Recipes used by the workloads (seed, stream):
  * uniform[-1,1) / uniform[-2,2): 24-bit draws, exact in binary32
  * lognormal(0, 3) with a random sign
  * int32 uniform on [-2^20, 2^20]
  * bf16 storage: the binary32 draw rounded to bfloat16 (round to nearest
    even, done by torch's CPU conversion)
  * binary16 storage: the binary32 draw rounded to binary16 (round to nearest
    even, numpy's conversion)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .. import buildlib

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = buildlib.gen_lib_path()
        if not os.path.exists(path):
            buildlib.build_gen()
        lib = ctypes.CDLL(path)
        u64, i64, f64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        vp = ctypes.c_void_p
        lib.pycgen_bits.restype = u64
        lib.pycgen_bits.argtypes = [u64, u64, u64]
        lib.pycgen_splitmix64_next.restype = u64
        lib.pycgen_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
        lib.pycgen_uniform_f32.argtypes = [u64, u64, u64, i64, f64, f64, vp, i32]
        lib.pycgen_lognormal_signed_f32.argtypes = [u64, u64, u64, i64, f64, vp, i32]
        lib.pycgen_int_uniform_i32.argtypes = [u64, u64, u64, i64, i64, i64, vp, i32]
        lib.pycgen_index_sample.argtypes = [u64, u64, u64, i64, i64, vp]
        lib.pycgen_loguniform_i64.argtypes = [u64, u64, u64, i64, f64, f64, i64, i64, vp]
        lib.pycgen_exponential_f64.argtypes = [u64, u64, u64, i64, f64, vp]
        lib.pycgen_unit_f64.argtypes = [u64, u64, u64, i64, vp]
        for fn in ("pycgen_uniform_f32", "pycgen_lognormal_signed_f32",
                   "pycgen_int_uniform_i32", "pycgen_index_sample",
                   "pycgen_loguniform_i64", "pycgen_exponential_f64", "pycgen_unit_f64"):
            getattr(lib, fn).restype = None
        _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def bits(seed: int, stream: int, i: int) -> int:
    return int(_load().pycgen_bits(seed, stream, i))


def splitmix64_sequence(state: int, count: int) -> list[int]:
    """The classic sequential SplitMix64 sequence from ``state`` (pins mix64)."""
    s = ctypes.c_uint64(state)
    return [int(_load().pycgen_splitmix64_next(ctypes.byref(s))) for _ in range(count)]


def uniform_f32(seed, stream, n, lo=-1.0, hi=1.0, offset=0, out=None) -> np.ndarray:
    out = np.empty(n, np.float32) if out is None else out
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == n
    _load().pycgen_uniform_f32(seed, stream, offset, n, lo, hi, out.ctypes.data, _threads())
    return out


def lognormal_signed_f32(seed, stream, n, sigma=3.0, offset=0, out=None) -> np.ndarray:
    out = np.empty(n, np.float32) if out is None else out
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == n
    _load().pycgen_lognormal_signed_f32(seed, stream, offset, n, sigma, out.ctypes.data,
                                        _threads())
    return out


def int_uniform_i32(seed, stream, n, lo=-(1 << 20), hi=(1 << 20), offset=0, out=None):
    out = np.empty(n, np.int32) if out is None else out
    assert out.dtype == np.int32 and out.flags.c_contiguous and out.size == n
    _load().pycgen_int_uniform_i32(seed, stream, offset, n, lo, hi, out.ctypes.data,
                                   _threads())
    return out


def index_sample(seed, stream, k, n_range, offset=0) -> np.ndarray:
    out = np.empty(k, np.int64)
    _load().pycgen_index_sample(seed, stream, offset, k, n_range, out.ctypes.data)
    return out


def loguniform_i64(seed, stream, n, lg_lo, lg_span, vmin, vmax, offset=0) -> np.ndarray:
    out = np.empty(n, np.int64)
    _load().pycgen_loguniform_i64(seed, stream, offset, n, lg_lo, lg_span, vmin, vmax,
                                  out.ctypes.data)
    return out


def exponential_f64(seed, stream, n, rate, offset=0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().pycgen_exponential_f64(seed, stream, offset, n, rate, out.ctypes.data)
    return out


def unit_f64(seed, stream, n, offset=0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().pycgen_unit_f64(seed, stream, offset, n, out.ctypes.data)
    return out


def to_bf16_values(x: np.ndarray) -> np.ndarray:
    """binary32 draws rounded to bfloat16 (torch CPU conversion, round to nearest
    even) and returned as the exactly representable binary32 values."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy()


def to_f16_values(x: np.ndarray) -> np.ndarray:
    """binary32 draws rounded to binary16 (numpy's conversion, round to nearest
    even), returned as a float16 array."""
    with np.errstate(over="ignore"):
        return np.ascontiguousarray(x, dtype=np.float32).astype(np.float16)


# ------------------------------------------------------------------ recipes
# Named workload recipes (seed, stream) shared by tests and the benchmark.

def segment_lengths(nseg=20000, seed=3, stream=0, max_log2=20) -> np.ndarray:
    """Segment lengths log-uniform in [1, 2^max_log2]: floor(2^(max_log2*U))."""
    return loguniform_i64(seed, stream, nseg, 0.0, float(max_log2), 1, 1 << max_log2)


def argmin_with_minima(seed, n, frac=0.01, minimum=-2.5, stream_vals=0, stream_pos=1):
    """uniform[-2,2) values with floor(frac*n) positions (sampled with replacement)
    overwritten by ``minimum``; the expected argmin is the smallest chosen index."""
    x = uniform_f32(seed, stream_vals, n, -2.0, 2.0)
    k = int(n * frac)
    if k > 0:
        pos = index_sample(seed, stream_pos, k, n)
        x[pos] = np.float32(minimum)
    return x


# ------------------------------------------------------------------ sparse matrices

def poisson2d(nx, ny, dtype=np.float32):
    """CSR of the 5-point Laplacian on an nx x ny grid (Dirichlet boundary):
    4 on the diagonal, -1 for each grid neighbour; rows in grid order
    (row = iy * nx + ix).  Returns (rowptr int64, col int32, val)."""
    n = nx * ny
    iy, ix = np.divmod(np.arange(n, dtype=np.int64), nx)
    cols, vals = [], []
    for dx, dy, v in ((0, -1, -1.0), (-1, 0, -1.0), (0, 0, 4.0), (1, 0, -1.0), (0, 1, -1.0)):
        ok = (ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
        cols.append(np.where(ok, (iy + dy) * nx + ix + dx, -1))
        vals.append(np.full(n, v))
    c = np.stack(cols, 1)
    v = np.stack(vals, 1)
    keep = c >= 0
    counts = keep.sum(1)
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return rowptr, c[keep].astype(np.int32), v[keep].astype(dtype)


def random_spd(n, seed, max_degree=1000, empty_every=0, dtype=np.float64):
    """A seeded symmetric, strictly diagonally dominant (so positive definite)
    CSR matrix: row i draws log-uniform in [1, max_degree] partners j (both a_ij
    and a_ji are set, values uniform in [-1, 0)), the diagonal is the row's sum
    of |off-diagonal| + 1.  With empty_every = k, every k-th row and column are
    left empty (not SPD then; for products only).  Returns (rowptr, col, val)."""
    rng = np.random.default_rng(seed)
    deg = np.floor(2.0 ** (rng.random(n) * np.log2(max_degree))).astype(np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    cols = rng.integers(0, n, rows.size)
    vals = -rng.random(rows.size)
    r = np.concatenate([rows, cols])
    c = np.concatenate([cols, rows])
    v = np.concatenate([vals, vals])
    off = r != c
    r, c, v = r[off], c[off], v[off]
    if empty_every:
        live = (r % empty_every != 0) & (c % empty_every != 0)
        r, c, v = r[live], c[live], v[live]
    key = r * n + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    uniq, first = np.unique(key, return_index=True)
    v = np.add.reduceat(v, first)           # merge duplicate draws of one entry
    r, c = np.divmod(uniq, n)
    diag = np.bincount(r, weights=np.abs(v), minlength=n) + 1.0
    di = np.arange(n, dtype=np.int64)
    if empty_every:
        keepd = di % empty_every != 0
        di, diag = di[keepd], diag[keepd]
    R = np.concatenate([r, di])
    C = np.concatenate([c, di])
    V = np.concatenate([v, diag[di] if not empty_every else diag])
    order = np.lexsort((C, R))
    R, C, V = R[order], C[order], V[order]
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(R, minlength=n))]).astype(np.int64)
    return rowptr, C.astype(np.int32), V.astype(dtype)
