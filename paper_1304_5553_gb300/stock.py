"""Stock specifications of the standard map / map-reduce workloads.

Each entry is an argument spec plus statement (map) or result type, neutral
element, reduce and map expressions (map-reduce), exactly as a user would
write them for ``pyc_map_create`` / ``pyc_reduce_create``:

  lin_comb_*   z[i] = a*x[i] + b*y[i]                       (Listing 3a)
  gauss_sin    z[i] = x[i]*exp(-y[i]*y[i]) + sin(u[i])*w[i]  (four inputs)
  dot_*        sum x[i]*y[i], neutral 0                      (Listing 3b)
  sum_*        plain and compensated binary32 sums, int32 -> int64 sum
  max / argmin binary32 maximum; (value, first index) minimum
"""
from __future__ import annotations

import threading
from concurrent.futures import ThreadPoolExecutor

from . import pyc

MAPS = {
    "lin_comb_f32": ("float a, float *x, float b, float *y, float *z", "z[i] = a*x[i] + b*y[i]"),
    "lin_comb_bf16": ("float a, __nv_bfloat16 *x, float b, __nv_bfloat16 *y, __nv_bfloat16 *z",
                      "z[i] = a*x[i] + b*y[i]"),
    "lin_comb_i32": ("int a, int *x, int b, int *y, int *z", "z[i] = a*x[i] + b*y[i]"),
    "gauss_sin_f32": ("float *x, float *y, float *u, float *w, float *z",
                      "z[i] = x[i]*exp(-y[i]*y[i]) + sin(u[i])*w[i]"),
    "scale2_f32": ("float *a", "a[i] *= 2"),
    "add_f32": ("float *tgt, float *op1, float *op2", "tgt[i] = op1[i] + op2[i]"),
    "copy_f32": ("float *src, float *dst", "dst[i] = src[i]"),
}

# name: (result dtype, neutral, reduce expression, map expression, argspec, options)
REDUCES = {
    "dot_f32": (pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y", {}),
    "dot_bf16": (pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "__nv_bfloat16 *x, __nv_bfloat16 *y", {}),
    "dot_i32_i64": (pyc.PYC_I64, "0", "a+b", "(long long)x[i]*y[i]", "int *x, int *y", {}),
    "sum_f32": (pyc.PYC_F32, "0", "a+b", "x[i]", "float *x", {}),
    "sum_f32_comp": (pyc.PYC_F32, "0", "a+b", "x[i]", "float *x", {"compensated": 1}),
    "sum_i32_i64": (pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "int *x", {}),
    "max_f32": (pyc.PYC_F32, "-INFINITY", "a > b ? a : b", "x[i]", "float *x", {}),
    "argmin_f32": (pyc.PYC_ARGMIN_F32, None, None, "x[i]", "float *x", {}),
    "argmax_f32": (pyc.PYC_ARGMAX_F32, None, None, "x[i]", "float *x", {}),
}

# name: (value dtype, neutral, scan expression, input expression, output statement, argspec)
SCANS = {
    "cumsum_f32": (pyc.PYC_F32, "0", "a+b", "x[i]", "y[i] = item", "float *x, float *y"),
    "cumsum_excl_i32_i64": (pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "y[i] = prev_item",
                            "int *x, long long *y"),
    # fmaxf: one instruction where a compare-and-select takes two, and a scan applies
    # its operation about three times per element (NaN elements are skipped)
    "cummax_f32": (pyc.PYC_F32, "-INFINITY", "fmaxf(a, b)", "x[i]", "y[i] = item",
                   "float *x, float *y"),
    # composition of v -> ca[i] v + cb[i] (mod 2^32), packed A << 32 | B: not commutative
    "affine_u32": (pyc.PYC_U64, "1ull << 32",
                   "((unsigned long long)((unsigned)(a >> 32) * (unsigned)(b >> 32)) << 32)"
                   " | (unsigned)((unsigned)(b >> 32) * (unsigned)a + (unsigned)b)",
                   "((unsigned long long)ca[i] << 32) | cb[i]", "y[i] = item",
                   "unsigned *ca, unsigned *cb, unsigned long long *y"),
}

_handles = {}
_lock = threading.Lock()


def create(name, **opts):
    """Handle for a stock spec (created once per process and option set)."""
    key = (name, tuple(sorted(opts.items())))
    with _lock:
        if key in _handles:
            return _handles[key]
    if name in MAPS:
        spec, stmt = MAPS[name]
        h = pyc.pyc_map_create(spec, stmt, name, opts or None)
    elif name in SCANS:
        dt, neu, red, inp, out, spec = SCANS[name]
        h = pyc.pyc_scan_create(dt, neu, red, inp, out, spec, opts or None)
    else:
        dt, neu, red, mexpr, spec, o = REDUCES[name]
        o = dict(o, **opts)
        h = pyc.pyc_reduce_create(dt, neu, red, mexpr, spec, o or None)
    with _lock:
        _handles.setdefault(key, h)
        return _handles[key]


def compile_all(names=None, threads=8):
    """Create (and so compile or load from cache) the stock specs in parallel:
    NVRTC runs outside the GIL, one program per thread."""
    names = list(names or (list(MAPS) + list(REDUCES) + list(SCANS)))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(create, names))
    return names
