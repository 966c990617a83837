"""Python binding of the pyc C ABI (``include/pyc.h``).

Argument marshalling only: every entry point keeps the C name and forwards to
``libpyc.so``; all work runs in the library and its generated kernels.  Device
pointers are ints (e.g. ``tensor.data_ptr()``) and streams are raw handles
(e.g. ``torch.cuda.current_stream().cuda_stream``).

The paper-style front ends ``ElementwiseKernel`` and ``ReductionKernel`` (Sec.
3.2.4 and 3.2.5) take torch tensors and Python scalars and marshal them in the
declared order.  If the native library is missing, importing this module
raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import struct

from . import buildlib

PYC_OK, PYC_E_PARSE, PYC_E_COMPILE, PYC_E_ARG, PYC_E_CUDA, PYC_E_NOMEM, PYC_E_BUSY, \
    PYC_E_TIMEOUT, PYC_E_INTERNAL, PYC_E_NOTFOUND = range(10)
STATUS_NAMES = {0: "PYC_OK", 1: "PYC_E_PARSE", 2: "PYC_E_COMPILE", 3: "PYC_E_ARG",
                4: "PYC_E_CUDA", 5: "PYC_E_NOMEM", 6: "PYC_E_BUSY", 7: "PYC_E_TIMEOUT",
                8: "PYC_E_INTERNAL", 9: "PYC_E_NOTFOUND"}

PYC_F32, PYC_F64, PYC_BF16, PYC_F16, PYC_I32, PYC_I64, PYC_ARGMIN_F32, PYC_ARGMAX_F32, \
    PYC_U8, PYC_I8, PYC_U32, PYC_U64, PYC_I16, PYC_U16 = range(14)

# struct-module codes for packing scalars of each dtype (bf16/half packed as raw bits)
_SCALAR_FMT = {PYC_F32: "f", PYC_F64: "d", PYC_I32: "i", PYC_I64: "q", PYC_U8: "B",
               PYC_I8: "b", PYC_U32: "I", PYC_U64: "Q", PYC_I16: "h", PYC_U16: "H",
               PYC_BF16: "H", PYC_F16: "e"}


class PycError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.message = message


class pyc_opts(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("vec_bytes", ctypes.c_int),
                ("items_per_thread", ctypes.c_int), ("compensated", ctypes.c_int),
                ("fmad", ctypes.c_int), ("preamble", ctypes.c_char_p),
                ("debug_bounds", ctypes.c_int)]


class pyc_param_info(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("is_pointer", ctypes.c_int),
                ("dtype", ctypes.c_int), ("elem_bytes", ctypes.c_int),
                ("scalar_offset", ctypes.c_int), ("pointer_slot", ctypes.c_int),
                ("read", ctypes.c_int), ("written", ctypes.c_int), ("lifted", ctypes.c_int)]


class pyc_argf32(ctypes.Structure):
    _fields_ = [("v", ctypes.c_float), ("pad", ctypes.c_int32), ("i", ctypes.c_int64)]


PYC_REQ_MAP, PYC_REQ_REDUCE = 0, 1
PYC_REPLAY_SERVER, PYC_REPLAY_DIRECT = 0, 1


class pyc_server_cfg(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("num_streams", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("max_inflight", ctypes.c_int), ("max_queue", ctypes.c_int)]


class pyc_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("pad", ctypes.c_int), ("handle", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("ptrs", ctypes.POINTER(ctypes.c_void_p)),
                ("scalars", ctypes.c_void_p), ("deadline_us", ctypes.c_int64)]


HOST_EXEC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(pyc_request),
                                ctypes.c_void_p)


class pyc_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("batch_size", ctypes.c_int), ("d_out", ctypes.c_void_p),
                ("value", ctypes.c_ubyte * 16), ("t_submit_ns", ctypes.c_int64),
                ("t_admit_ns", ctypes.c_int64), ("t_launch_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class pyc_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "batches",
                                              "admitted_bytes", "peak_admitted_bytes", "queued",
                                              "arena_in_use")]


class pyc_pool_cfg(ctypes.Structure):
    _fields_ = [("max_bytes", ctypes.c_int64), ("max_retained", ctypes.c_int64)]


class pyc_pool_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("live_bytes", "live_blocks", "retained_bytes",
                                              "retained_blocks", "system_bytes", "hits",
                                              "misses", "system_allocs", "system_frees")]


PYC_POOL_DEVICE, PYC_POOL_PINNED, PYC_POOL_HOST = 0, 1, 2


class pyc_cg_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("residual", ctypes.c_double),
                ("converged", ctypes.c_int), ("pad", ctypes.c_int)]

# every symbol include/pyc.h declares (checked by the tests)
EXPORTED = [
    "pyc_last_error", "pyc_version",
    "pyc_map_create", "pyc_map_launch", "pyc_map_num_params", "pyc_map_param",
    "pyc_map_scalar_bytes", "pyc_map_source", "pyc_map_autotune", "pyc_map_destroy",
    "pyc_reduce_create", "pyc_reduce_launch", "pyc_reduce_batched", "pyc_reduce_num_params",
    "pyc_reduce_param", "pyc_reduce_scalar_bytes", "pyc_reduce_out_bytes", "pyc_reduce_source",
    "pyc_reduce_autotune", "pyc_reduce_destroy", "pyc_cache_stats", "pyc_reduce_launch_static",
    "pyc_reduce_static_scratch", "pyc_reduce_shard", "pyc_reduce_combine",
    "pyc_map_check_bounds", "pyc_reduce_check_bounds", "pyc_test_inject",
    "pyc_server_create", "pyc_server_create_host", "pyc_server_submit", "pyc_server_poll",
    "pyc_server_release",
    "pyc_server_get_stats", "pyc_server_destroy", "pyc_server_replay", "pyc_map_launch_host",
    "pyc_map_config", "pyc_reduce_config", "pyc_reduce_batched_autotune",
    "pyc_reduce_batched_config", "pyc_reduce_batched_plan",
    "pyc_scan_create", "pyc_scan_launch", "pyc_scan_num_params", "pyc_scan_param",
    "pyc_scan_scalar_bytes", "pyc_scan_source", "pyc_scan_autotune", "pyc_scan_config", "pyc_scan_destroy",
    "pyc_scan_sync", "pyc_scan_launch_test", "pyc_expr_map_create", "pyc_expr_reduce_create",
    "pyc_expr_type", "pyc_pool_block_size", "pyc_pool_create", "pyc_pool_alloc", "pyc_pool_free",
    "pyc_pool_trim", "pyc_pool_get_stats", "pyc_pool_destroy",
    "pyc_csr_create", "pyc_csr_width", "pyc_csr_set_width", "pyc_spmv", "pyc_spmv_autotune", "pyc_cg_solve",
    "pyc_csr_destroy",
]

_lib = None


def default_cache_dir():
    return os.path.join(buildlib.REPO_DIR, ".pyc_kcache")


def load(build_if_missing=True):
    """Load libpyc.so (building it in-tree if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = buildlib.pyc_lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError("libpyc.so is not built: run __graft_entry__.build()")
        buildlib.build_all()
    os.environ.setdefault("PYC_CACHE_DIR", default_cache_dir())
    lib = ctypes.CDLL(path)
    vp, i64, i32, cp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_char_p
    st = ctypes.c_int
    sig = {
        "pyc_last_error": (cp, []),
        "pyc_version": (cp, []),
        "pyc_map_create": (st, [cp, cp, cp, ctypes.POINTER(pyc_opts), ctypes.POINTER(vp)]),
        "pyc_map_launch": (st, [vp, i64, ctypes.POINTER(vp), vp, vp]),
        "pyc_map_launch_host": (st, [vp, i64, ctypes.POINTER(vp), vp]),
        "pyc_map_config": (st, [vp, i64] + [ctypes.POINTER(i32)] * 3),
        "pyc_reduce_config": (st, [vp, i64] + [ctypes.POINTER(i32)] * 3),
        "pyc_reduce_batched_config": (st, [vp] + [ctypes.POINTER(i32)] * 4),
        "pyc_reduce_batched_plan": (st, [vp, i64, vp, ctypes.POINTER(vp), vp, vp, vp, i64,
                                         ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "pyc_scan_config": (st, [vp, i64] + [ctypes.POINTER(i32)] * 3),
        "pyc_map_num_params": (i32, [vp]),
        "pyc_map_param": (st, [vp, i32, ctypes.POINTER(pyc_param_info)]),
        "pyc_map_scalar_bytes": (i32, [vp]),
        "pyc_map_source": (cp, [vp]),
        "pyc_map_autotune": (st, [vp, i64, vp]),
        "pyc_map_destroy": (None, [vp]),
        "pyc_reduce_create": (st, [i32, cp, cp, cp, cp, ctypes.POINTER(pyc_opts),
                                   ctypes.POINTER(vp)]),
        "pyc_reduce_launch": (st, [vp, i64, ctypes.POINTER(vp), vp, vp, vp]),
        "pyc_reduce_batched": (st, [vp, i64, ctypes.POINTER(i64), ctypes.POINTER(vp), vp, vp,
                                    vp]),
        "pyc_reduce_launch_static": (st, [vp, i64, ctypes.POINTER(vp), vp, vp, vp]),
        "pyc_reduce_static_scratch": (st, [ctypes.POINTER(vp), ctypes.POINTER(i64)]),
        "pyc_reduce_shard": (st, [vp, i64, i64, i64, ctypes.POINTER(vp), vp, vp, vp]),
        "pyc_reduce_combine": (st, [vp, i64, vp, vp, vp]),
        "pyc_map_check_bounds": (st, [vp]),
        "pyc_test_inject": (st, [i32, i64]),
        "pyc_reduce_check_bounds": (st, [vp]),
        "pyc_scan_create": (st, [i32, cp, cp, cp, cp, cp, ctypes.POINTER(pyc_opts),
                                 ctypes.POINTER(vp)]),
        "pyc_scan_launch": (st, [vp, i64, ctypes.POINTER(vp), vp, vp]),
        "pyc_scan_sync": (st, [vp, vp]),
        "pyc_expr_map_create": (st, [cp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), i32,
                                     ctypes.POINTER(pyc_opts), ctypes.POINTER(vp)]),
        "pyc_expr_reduce_create": (st, [cp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), i32,
                                        cp, ctypes.POINTER(pyc_opts), ctypes.POINTER(vp)]),
        "pyc_expr_type": (st, [cp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i32)]),
        "pyc_pool_block_size": (i64, [i64]),
        "pyc_pool_create": (st, [i32, ctypes.POINTER(pyc_pool_cfg), ctypes.POINTER(vp)]),
        "pyc_pool_alloc": (st, [vp, i64, vp, ctypes.POINTER(vp)]),
        "pyc_pool_free": (st, [vp, vp, vp]),
        "pyc_pool_trim": (st, [vp]),
        "pyc_pool_get_stats": (st, [vp, ctypes.POINTER(pyc_pool_stats)]),
        "pyc_pool_destroy": (None, [vp]),
        "pyc_csr_create": (st, [i64, i64, i64, vp, vp, vp, i32, ctypes.POINTER(vp)]),
        "pyc_csr_width": (st, [vp, ctypes.POINTER(i32)]),
        "pyc_csr_set_width": (st, [vp, i32]),
        "pyc_spmv": (st, [vp, vp, vp, vp]),
        "pyc_spmv_autotune": (st, [vp, vp, vp, vp]),
        "pyc_cg_solve": (st, [vp, vp, vp, ctypes.c_double, i64, vp, ctypes.POINTER(pyc_cg_info)]),
        "pyc_csr_destroy": (None, [vp]),
        "pyc_scan_launch_test": (st, [vp, i64, ctypes.POINTER(vp), vp, vp, i64, i64]),
        "pyc_scan_num_params": (i32, [vp]),
        "pyc_scan_param": (st, [vp, i32, ctypes.POINTER(pyc_param_info)]),
        "pyc_scan_scalar_bytes": (i32, [vp]),
        "pyc_scan_source": (cp, [vp]),
        "pyc_scan_autotune": (st, [vp, i64, vp]),
        "pyc_scan_destroy": (None, [vp]),
        "pyc_reduce_batched_autotune": (st, [vp, i64, ctypes.POINTER(i64), ctypes.POINTER(vp), vp,
                                             vp, vp]),
        "pyc_reduce_num_params": (i32, [vp]),
        "pyc_reduce_param": (st, [vp, i32, ctypes.POINTER(pyc_param_info)]),
        "pyc_reduce_scalar_bytes": (i32, [vp]),
        "pyc_reduce_out_bytes": (i32, [vp]),
        "pyc_reduce_source": (cp, [vp]),
        "pyc_reduce_autotune": (st, [vp, i64, vp]),
        "pyc_reduce_destroy": (None, [vp]),
        "pyc_cache_stats": (None, [ctypes.POINTER(i64)] * 3),
        "pyc_server_create": (st, [ctypes.POINTER(pyc_server_cfg), ctypes.POINTER(vp)]),
        "pyc_server_create_host": (st, [ctypes.POINTER(pyc_server_cfg), HOST_EXEC_FN, vp,
                                        ctypes.POINTER(vp)]),
        "pyc_server_submit": (st, [vp, ctypes.POINTER(pyc_request), ctypes.POINTER(ctypes.c_uint64)]),
        "pyc_server_poll": (st, [vp, ctypes.c_uint64, ctypes.POINTER(pyc_result), i64]),
        "pyc_server_release": (st, [vp, ctypes.c_uint64]),
        "pyc_server_get_stats": (st, [vp, ctypes.POINTER(pyc_server_stats)]),
        "pyc_server_destroy": (None, [vp]),
        "pyc_server_replay": (st, [vp, i64, ctypes.POINTER(pyc_request), ctypes.POINTER(i64),
                                   ctypes.c_int, ctypes.POINTER(pyc_result)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != PYC_OK:
        raise PycError(status, load().pyc_last_error().decode(errors="replace"))


def _enc(s):
    return None if s is None else s.encode()


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, pyc_opts):
        return ctypes.byref(opts)
    o = pyc_opts()
    for k, v in dict(opts).items():
        if k == "preamble":
            v = _enc(v)
        setattr(o, k, v)
    # keep the preamble bytes alive for the call
    return ctypes.byref(o)


def _ptr_array(ptrs):
    ptrs = list(ptrs or [])
    arr = (ctypes.c_void_p * max(1, len(ptrs)))(*[int(p) if p else None for p in ptrs])
    return arr


def _stream(stream):
    return None if not stream else ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------ C-named calls

def pyc_last_error() -> str:
    return load().pyc_last_error().decode(errors="replace")


def pyc_version() -> str:
    return load().pyc_version().decode()


def pyc_map_create(argspec, stmt, name=None, opts=None):
    h = ctypes.c_void_p()
    _check(load().pyc_map_create(_enc(argspec), _enc(stmt), _enc(name), _opts(opts),
                                 ctypes.byref(h)))
    return h


def pyc_map_launch(h, n, ptrs, scalars=None, stream=None):
    _check(load().pyc_map_launch(h, int(n), _ptr_array(ptrs), scalars, _stream(stream)))


def pyc_map_launch_host(h, n, host_ptrs, scalars=None):
    """Map over host arrays (addresses of page-locked or pageable host memory)."""
    _check(load().pyc_map_launch_host(h, int(n), _ptr_array(host_ptrs), scalars))


def pyc_map_destroy(h):
    load().pyc_map_destroy(h)


def pyc_map_source(h) -> str:
    return load().pyc_map_source(h).decode()


def pyc_map_autotune(h, n, stream=None):
    _check(load().pyc_map_autotune(h, int(n), _stream(stream)))


def pyc_reduce_create(out_dtype, neutral, reduce_expr, map_expr, argspec, opts=None):
    h = ctypes.c_void_p()
    _check(load().pyc_reduce_create(int(out_dtype), _enc(neutral), _enc(reduce_expr),
                                    _enc(map_expr), _enc(argspec), _opts(opts), ctypes.byref(h)))
    return h


def pyc_reduce_launch(h, n, ptrs, scalars, d_out, stream=None):
    _check(load().pyc_reduce_launch(h, int(n), _ptr_array(ptrs), scalars, d_out,
                                    _stream(stream)))


def pyc_reduce_launch_static(h, n, ptrs, scalars, d_out, stream=None):
    """pyc_reduce_launch without any device allocation (static scratch area)."""
    _check(load().pyc_reduce_launch_static(h, int(n), _ptr_array(ptrs), scalars, d_out,
                                           _stream(stream)))


PYC_RECORD_BYTES = 16


def pyc_reduce_shard(h, n_total, i0, n, ptrs, scalars, d_rec, stream=None):
    """Fold shard [i0, i0 + n) of [0, n_total) into a 16-byte record at d_rec."""
    _check(load().pyc_reduce_shard(h, int(n_total), int(i0), int(n), _ptr_array(ptrs), scalars,
                                   d_rec, _stream(stream)))


def pyc_reduce_combine(h, k, d_recs, d_out, stream=None):
    """Fold k consecutive 16-byte records into the result at d_out."""
    _check(load().pyc_reduce_combine(h, int(k), d_recs, d_out, _stream(stream)))


PYC_INJECT_ALLOC, PYC_INJECT_COMPILE, PYC_INJECT_STALL_MS, PYC_INJECT_ADMIT = 0, 1, 2, 3


def pyc_test_inject(what, value):
    """Test hook: make the next `value` allocations / compilations fail, or the
    next scheduler wake-up sleep `value` ms (value 0 clears)."""
    _check(load().pyc_test_inject(int(what), int(value)))


def pyc_map_check_bounds(h):
    """Raise PycError(PYC_E_INTERNAL) if the checked map recorded a violation."""
    _check(load().pyc_map_check_bounds(h))


def pyc_reduce_check_bounds(h):
    """Raise PycError(PYC_E_INTERNAL) if the checked map-reduce recorded a violation."""
    _check(load().pyc_reduce_check_bounds(h))


def pyc_reduce_static_scratch():
    """(device address, bytes) of pyc_reduce_launch_static's scratch area in the
    current context; the first query in a context looks the address up there."""
    a, b = ctypes.c_void_p(), ctypes.c_int64()
    _check(load().pyc_reduce_static_scratch(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def pyc_reduce_batched(h, nseg, seg_offsets, ptrs, scalars, d_out, stream=None):
    import numpy as np
    off = np.ascontiguousarray(seg_offsets, dtype=np.int64)
    if off.size != int(nseg) + 1:
        raise ValueError("seg_offsets must hold nseg + 1 entries")
    _check(load().pyc_reduce_batched(h, int(nseg),
                                     off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     _ptr_array(ptrs), scalars, d_out, _stream(stream)))


def pyc_scan_create(dtype, neutral, scan_expr, input_expr, output_stmt, argspec, opts=None):
    h = ctypes.c_void_p()
    _check(load().pyc_scan_create(int(dtype), _enc(neutral), _enc(scan_expr), _enc(input_expr),
                                  _enc(output_stmt), _enc(argspec), _opts(opts), ctypes.byref(h)))
    return h


def pyc_scan_launch(h, n, ptrs, scalars=None, stream=None):
    _check(load().pyc_scan_launch(h, int(n), _ptr_array(ptrs), scalars, _stream(stream)))


def pyc_expr_map_create(expr, arg_dtypes, arg_is_array, out_dtype, opts=None):
    n = len(arg_dtypes)
    dt = (ctypes.c_int * max(n, 1))(*[int(d) for d in arg_dtypes])
    ia = (ctypes.c_int * max(n, 1))(*[int(bool(a)) for a in arg_is_array])
    h = ctypes.c_void_p()
    _check(load().pyc_expr_map_create(_enc(expr), n, dt, ia, int(out_dtype), _opts(opts),
                                      ctypes.byref(h)))
    return h


def pyc_expr_reduce_create(expr, arg_dtypes, arg_is_array, out_dtype, reduce="sum", opts=None):
    n = len(arg_dtypes)
    dt = (ctypes.c_int * max(n, 1))(*[int(d) for d in arg_dtypes])
    ia = (ctypes.c_int * max(n, 1))(*[int(bool(a)) for a in arg_is_array])
    h = ctypes.c_void_p()
    _check(load().pyc_expr_reduce_create(_enc(expr), n, dt, ia, int(out_dtype), _enc(reduce),
                                         _opts(opts), ctypes.byref(h)))
    return h


def pyc_expr_type(expr, arg_dtypes, arg_is_array):
    n = len(arg_dtypes)
    dt = (ctypes.c_int * max(n, 1))(*[int(d) for d in arg_dtypes])
    ia = (ctypes.c_int * max(n, 1))(*[int(bool(a)) for a in arg_is_array])
    r = ctypes.c_int()
    _check(load().pyc_expr_type(_enc(expr), n, dt, ia, ctypes.byref(r)))
    return r.value


def pyc_pool_block_size(nbytes):
    return int(load().pyc_pool_block_size(int(nbytes)))


def pyc_pool_create(kind=PYC_POOL_DEVICE, max_bytes=0, max_retained=0):
    cfg = pyc_pool_cfg(int(max_bytes), int(max_retained))
    h = ctypes.c_void_p()
    _check(load().pyc_pool_create(int(kind), ctypes.byref(cfg), ctypes.byref(h)))
    _destroyed_pools.discard(h.value)
    return h


def pyc_pool_alloc(p, nbytes, stream=None):
    q = ctypes.c_void_p()
    _check(load().pyc_pool_alloc(p, int(nbytes), _stream(stream), ctypes.byref(q)))
    return q.value


def pyc_pool_free(p, ptr, stream=None):
    _check(load().pyc_pool_free(p, ptr, _stream(stream)))


def pyc_pool_trim(p):
    _check(load().pyc_pool_trim(p))


def pyc_pool_get_stats(p):
    st = pyc_pool_stats()
    _check(load().pyc_pool_get_stats(p, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in pyc_pool_stats._fields_}


_destroyed_pools = set()


def pyc_pool_destroy(p):
    _destroyed_pools.add(p.value if hasattr(p, "value") else p)
    load().pyc_pool_destroy(p)


class _PoolBlock:
    """A device pool block exposed through __cuda_array_interface__; torch keeps
    this object alive as long as a tensor made from it, and its deletion returns
    the block to the pool with the stream current at that time."""

    def __init__(self, pool, n, dtype, stream):
        import torch
        self._torch = torch
        self._pool = pool
        self._dt = dtype
        nbytes = max(n, 1) * torch.empty(0, dtype=dtype).element_size()
        self._ptr = pyc_pool_alloc(pool, nbytes, stream)
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": torch.empty(0, dtype=dtype).numpy().dtype.str
            if dtype != torch.bfloat16 else "<V2", "data": (self._ptr, False),
            "version": 2}

    def __del__(self):
        ptr, self._ptr = getattr(self, "_ptr", None), None
        pool = getattr(self, "_pool", None)
        if not ptr or _lib is None or pool is None:
            return
        key = pool.value if hasattr(pool, "value") else pool
        if key in _destroyed_pools:  # destroy already returned the memory
            return
        try:
            s = self._torch.cuda.current_stream().cuda_stream
            pyc_pool_free(pool, ptr, s)
        except Exception:  # interpreter shutdown, or a pool handle reused since
            pass


def pool_empty(pool, n, dtype, stream=None):
    """A 1-D CUDA tensor of n elements backed by a block of a device pool; the
    block goes back to the pool when the tensor is deleted."""
    import torch
    if dtype == torch.bfloat16:  # the interface has no bfloat16 type string
        return pool_empty(pool, n, torch.int16, stream).view(torch.bfloat16)
    blk = _PoolBlock(pool, n, dtype, stream)
    return torch.as_tensor(blk, device="cuda")


def pyc_csr_create(nrows, ncols, nnz, rowptr, colidx, vals, vt=PYC_F32):
    h = ctypes.c_void_p()
    _check(load().pyc_csr_create(int(nrows), int(ncols), int(nnz), rowptr, colidx, vals, int(vt),
                                 ctypes.byref(h)))
    return h


def pyc_csr_width(a):
    w = ctypes.c_int()
    _check(load().pyc_csr_width(a, ctypes.byref(w)))
    return w.value


def pyc_csr_set_width(a, width):
    _check(load().pyc_csr_set_width(a, int(width)))


def pyc_spmv(a, x, y, stream=None):
    _check(load().pyc_spmv(a, x, y, _stream(stream)))


def pyc_spmv_autotune(a, x, y, stream=None):
    _check(load().pyc_spmv_autotune(a, x, y, _stream(stream)))


def pyc_cg_solve(a, b, x, rtol=1e-6, maxit=1000, stream=None):
    info = pyc_cg_info()
    _check(load().pyc_cg_solve(a, b, x, float(rtol), int(maxit), _stream(stream),
                               ctypes.byref(info)))
    return {"iterations": info.iterations, "residual": info.residual,
            "converged": bool(info.converged)}


def pyc_csr_destroy(a):
    load().pyc_csr_destroy(a)


def pyc_scan_sync(h, stream=None):
    """Synchronize `stream`; PycError(PYC_E_TIMEOUT) if a scan launch gave up a wait."""
    _check(load().pyc_scan_sync(h, _stream(stream)))


def pyc_scan_launch_test(h, n, ptrs, scalars=None, stream=None, stall_tile=-1,
                         spin_limit=1 << 20):
    _check(load().pyc_scan_launch_test(h, int(n), _ptr_array(ptrs), scalars, _stream(stream),
                                       int(stall_tile), int(spin_limit)))


def pyc_scan_autotune(h, n, stream=None):
    _check(load().pyc_scan_autotune(h, int(n), _stream(stream)))


def pyc_scan_source(h) -> str:
    return load().pyc_scan_source(h).decode()


def pyc_scan_destroy(h):
    load().pyc_scan_destroy(h)


def pyc_reduce_batched_autotune(h, nseg, seg_offsets, ptrs, scalars, d_out, stream=None):
    import numpy as np
    off = np.ascontiguousarray(seg_offsets, dtype=np.int64)
    if off.size != int(nseg) + 1:
        raise ValueError("seg_offsets must hold nseg + 1 entries")
    _check(load().pyc_reduce_batched_autotune(h, int(nseg),
                                              off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              _ptr_array(ptrs), scalars, d_out, _stream(stream)))


def pyc_reduce_destroy(h):
    load().pyc_reduce_destroy(h)


def pyc_reduce_source(h) -> str:
    return load().pyc_reduce_source(h).decode()


def pyc_reduce_out_bytes(h) -> int:
    return load().pyc_reduce_out_bytes(h)


def pyc_reduce_autotune(h, n, stream=None):
    _check(load().pyc_reduce_autotune(h, int(n), _stream(stream)))


def launch_config(h, n, reduce=False):
    """(vec_bytes, unroll, block) a launch of n elements would use."""
    v, u, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    fn = getattr(load(), "pyc_%s_config" % _kind(reduce))
    _check(fn(h, int(n), ctypes.byref(v), ctypes.byref(u), ctypes.byref(b)))
    return v.value, u.value, b.value


def batched_plan(h, seg_offsets, ptrs, scalars=None):
    """Host-side work plan of pyc_reduce_batched: (task_info (nseg x 6 int64:
    segment, n, head, chunk, nchunks, slot0), items (k x 4 int32: task, chunk,
    count, 0), partial slots)."""
    import numpy as np
    off = np.ascontiguousarray(seg_offsets, dtype=np.int64)
    nseg = off.size - 1
    lib = load()
    n_items, n_slots = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.pyc_reduce_batched_plan(h, nseg, off.ctypes.data, _ptr_array(ptrs), scalars,
                                       None, None, 0, ctypes.byref(n_items),
                                       ctypes.byref(n_slots)))
    info = np.zeros((max(nseg, 0), 6), np.int64)
    items = np.zeros((n_items.value, 4), np.int32)
    _check(lib.pyc_reduce_batched_plan(h, nseg, off.ctypes.data, _ptr_array(ptrs), scalars,
                                       info.ctypes.data, items.ctypes.data, n_items.value,
                                       ctypes.byref(n_items), ctypes.byref(n_slots)))
    return info, items, n_slots.value


def batched_config(h):
    """(vec_bytes, unroll, block) of the handle's batched launches."""
    return batched_config_full(h)[:3]


def batched_config_full(h):
    """(vec_bytes, unroll, block, reg_cap) of the handle's batched launches;
    reg_cap 0 = the regular build, else the register cap of the lean build."""
    v, u, b, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().pyc_reduce_batched_config(h, ctypes.byref(v), ctypes.byref(u), ctypes.byref(b),
                                            ctypes.byref(r)))
    return v.value, u.value, b.value, r.value


def batched_config_name(h):
    """The batched configuration as text, e.g. vec16_u2_b128_r80."""
    v, u, b, r = batched_config_full(h)
    return "vec%d_u%d_b%d" % (v, u, b) + ("_r%d" % r if r else "")


def pyc_cache_stats():
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    load().pyc_cache_stats(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return {"compiled": a.value, "disk_hits": b.value, "mem_hits": c.value}


def _kind(reduce):
    """'map', 'reduce' or 'scan' from the `reduce` argument (False, True or 'scan')."""
    return "scan" if reduce == "scan" else ("reduce" if reduce else "map")


def params(h, reduce=False):
    """Declared parameters as dicts (name, is_pointer, dtype, ... ); reduce is
    False (map), True (map-reduce) or 'scan'."""
    lib = load()
    k = _kind(reduce)
    num = getattr(lib, "pyc_%s_num_params" % k)(h)
    get = getattr(lib, "pyc_%s_param" % k)
    out = []
    for k in range(num):
        info = pyc_param_info()
        _check(get(h, k, ctypes.byref(info)))
        out.append({f: getattr(info, f) for f, _ in pyc_param_info._fields_})
        out[-1]["name"] = out[-1]["name"].decode()
    return out


def pack_scalars(h, values, reduce=False):
    """Pack scalar values in declaration order into the layout the handle expects
    (Python ints/floats are converted to the declared C type, as in Listing 3a)."""
    lib = load()
    size = getattr(lib, "pyc_%s_scalar_bytes" % _kind(reduce))(h)
    buf = ctypes.create_string_buffer(max(size, 1))
    scal = [p for p in params(h, reduce) if not p["is_pointer"]]
    if len(scal) != len(values):
        raise ValueError("expected %d scalars, got %d" % (len(scal), len(values)))
    for p, v in zip(scal, values):
        if p["dtype"] == PYC_BF16:
            import torch
            bits = torch.tensor([float(v)], dtype=torch.float32).to(torch.bfloat16).view(
                torch.int16).item() & 0xFFFF
            struct.pack_into("H", buf, p["scalar_offset"], bits)
        else:
            fmt = _SCALAR_FMT[p["dtype"]]
            struct.pack_into(fmt, buf, p["scalar_offset"],
                             float(v) if fmt in "fde" else int(v))
    return buf


# ------------------------------------------------------------------ serving

def pyc_server_create(mem_budget_bytes, arena_bytes=0, num_streams=0, max_batch=0,
                      max_inflight=0, max_queue=0):
    cfg = pyc_server_cfg(int(mem_budget_bytes), int(arena_bytes), num_streams, max_batch,
                         max_inflight, max_queue)
    h = ctypes.c_void_p()
    _check(load().pyc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


_host_servers = {}  # server handle -> its executor callback (kept alive while it runs)


def pyc_server_create_host(exec_fn, mem_budget_bytes, arena_bytes=0, num_streams=0,
                           max_batch=0, max_inflight=0, max_queue=0):
    """A serving loop whose batches run on the host (test hook, no GPU needed):
    exec_fn(req, value) is called once per request on the executor thread with
    req a pyc_request (ptrs: the arrays, server outputs filled in) and value the
    address of the result bytes of a map-reduce; it returns a status (0 = OK).  An
    exception raised by exec_fn fails that request with PYC_E_INTERNAL."""
    def call(user, req, value):
        try:
            return int(exec_fn(req.contents, value))
        except Exception:  # an executor that raised fails its request
            return PYC_E_INTERNAL

    cb = HOST_EXEC_FN(call)
    cfg = pyc_server_cfg(int(mem_budget_bytes), int(arena_bytes), num_streams, max_batch,
                         max_inflight, max_queue)
    h = ctypes.c_void_p()
    _check(load().pyc_server_create_host(ctypes.byref(cfg), cb, None, ctypes.byref(h)))
    _host_servers[h.value] = cb
    return h


def make_request(kind, handle, n, ptrs, scalars=None, deadline_us=0):
    """A pyc_request plus the buffers it points to (keep the tuple alive)."""
    arr = _ptr_array(ptrs)
    req = pyc_request(kind, 0, handle.value if isinstance(handle, ctypes.c_void_p) else handle,
                      int(n), ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)),
                      ctypes.cast(scalars, ctypes.c_void_p) if scalars is not None else None,
                      int(deadline_us))
    return req, arr, scalars


def pyc_server_submit(s, req):
    rid = ctypes.c_uint64()
    r = req[0] if isinstance(req, tuple) else req
    _check(load().pyc_server_submit(s, ctypes.byref(r), ctypes.byref(rid)))
    return rid.value


def pyc_server_poll(s, rid, timeout_us=0):
    """pyc_result, or None while the request is still running."""
    res = pyc_result()
    st = load().pyc_server_poll(s, rid, ctypes.byref(res), int(timeout_us))
    if st == PYC_E_TIMEOUT:
        return None
    _check(st)
    return res


def pyc_server_release(s, rid):
    _check(load().pyc_server_release(s, rid))


def pyc_server_get_stats(s):
    st = pyc_server_stats()
    _check(load().pyc_server_get_stats(s, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in pyc_server_stats._fields_}


def pyc_server_destroy(s):
    load().pyc_server_destroy(s)
    _host_servers.pop(s.value if isinstance(s, ctypes.c_void_p) else s, None)


class RequestTable:
    """A contiguous array of pyc_request (for pyc_server_replay) with every
    request's pointer list and scalars in two shared buffers."""

    def __init__(self, nreq, max_ptrs=4, scalar_bytes=16):
        self.n = nreq
        self.reqs = (pyc_request * nreq)()
        self.ptrs = (ctypes.c_void_p * (nreq * max_ptrs))()
        self.scal = ctypes.create_string_buffer(nreq * scalar_bytes)
        self.max_ptrs, self.sb = max_ptrs, scalar_bytes

    def set(self, k, kind, handle, n, ptrs, scalar_bytes=b""):
        base = k * self.max_ptrs
        for j, p in enumerate(ptrs):
            self.ptrs[base + j] = int(p) if p else None
        r = self.reqs[k]
        r.kind, r.handle, r.n, r.deadline_us = kind, handle.value, int(n), 0
        r.ptrs = ctypes.cast(ctypes.byref(self.ptrs, base * ctypes.sizeof(ctypes.c_void_p)),
                             ctypes.POINTER(ctypes.c_void_p))
        if scalar_bytes:
            off = k * self.sb
            ctypes.memmove(ctypes.addressof(self.scal) + off, scalar_bytes, len(scalar_bytes))
            r.scalars = ctypes.addressof(self.scal) + off
        else:
            r.scalars = None


def pyc_server_replay(s, table, arrival_ns=None, mode=PYC_REPLAY_SERVER):
    """Replay a RequestTable; returns the pyc_result array."""
    import numpy as np
    res = (pyc_result * table.n)()
    arr = None
    if arrival_ns is not None:
        arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        assert arr.size == table.n
    _check(load().pyc_server_replay(
        s, table.n, table.reqs, None if arr is None else arr.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int64)), mode, res))
    return res


# ------------------------------------------------------------------ paper-style front ends

_TORCH_DT = None


def _torch_dtype(d):
    import torch
    return {PYC_F32: torch.float32, PYC_F64: torch.float64, PYC_BF16: torch.bfloat16,
            PYC_F16: torch.float16, PYC_I32: torch.int32, PYC_I64: torch.int64,
            PYC_U8: torch.uint8, PYC_I8: torch.int8, PYC_I16: torch.int16,
            PYC_U32: torch.uint32, PYC_U64: torch.uint64, PYC_U16: torch.uint16}[d]


class _Front:
    _reduce = False

    def _marshal(self, args):
        import torch
        ps = self._params
        if len(args) != len(ps):
            raise TypeError("expected %d arguments, got %d" % (len(ps), len(args)))
        ptrs, scal, n = [], [], None
        for p, a in zip(ps, args):
            if p["is_pointer"]:
                if not isinstance(a, torch.Tensor) or not a.is_cuda:
                    raise TypeError("argument %r must be a CUDA tensor" % p["name"])
                if not a.is_contiguous():
                    raise ValueError("argument %r must be contiguous" % p["name"])
                if a.dtype != _torch_dtype(p["dtype"]):
                    raise TypeError("argument %r has dtype %s, spec says %s"
                                    % (p["name"], a.dtype, _torch_dtype(p["dtype"])))
                if n is None:
                    n = a.numel()
                elif a.numel() != n:  # all arrays have the same length (Sec. 3.2.4)
                    raise ValueError("all array arguments must have the same length")
                ptrs.append(a.data_ptr())
            else:
                scal.append(a)
        return ptrs, pack_scalars(self._h, scal, self._reduce), (n or 0)


class ElementwiseKernel(_Front):
    """z = ElementwiseKernel("float a, float *x, float b, float *y, float *z",
    "z[i] = a*x[i] + b*y[i]"); z(5, x, 6, y, out) -- Listing 3a."""

    def __init__(self, arguments, operation, name="kernel", **opts):
        self._h = pyc_map_create(arguments, operation, name, opts or None)
        self._params = params(self._h)

    def __call__(self, *args, stream=None, n=None):
        import torch
        ptrs, sc, nn = self._marshal(args)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        pyc_map_launch(self._h, nn if n is None else n, ptrs, sc, s)

    def autotune(self, n, stream=None):
        pyc_map_autotune(self._h, n, stream)

    @property
    def source(self):
        return pyc_map_source(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            pyc_map_destroy(self._h)


class ReductionKernel(_Front):
    """ReductionKernel(PYC_F32, neutral="0", reduce_expr="a+b", map_expr="x[i]*y[i]",
    arguments="float *x, float *y") -- Listing 3b.  Calling it returns a one-element
    device tensor: the result stays on the GPU (Sec. 3.2.5)."""
    _reduce = True

    def __init__(self, dtype_out, neutral, reduce_expr, map_expr=None, arguments=None, **opts):
        self._h = pyc_reduce_create(dtype_out, neutral, reduce_expr, map_expr, arguments,
                                    opts or None)
        self._params = params(self._h, True)
        self._out_dtype = dtype_out

    def _out(self, count=1):
        import torch
        if self._out_dtype in (PYC_ARGMIN_F32, PYC_ARGMAX_F32):
            return torch.empty((count, 2), dtype=torch.int64, device="cuda")
        return torch.empty(count, dtype=_torch_dtype(self._out_dtype), device="cuda")

    def __call__(self, *args, out=None, stream=None, n=None):
        import torch
        ptrs, sc, nn = self._marshal(args)
        out = self._out() if out is None else out
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        pyc_reduce_launch(self._h, nn if n is None else n, ptrs, sc, out.data_ptr(), s)
        return out

    def batched(self, seg_offsets, *args, out=None, stream=None):
        import torch
        ptrs, sc, _ = self._marshal(args)
        nseg = len(seg_offsets) - 1
        out = self._out(nseg) if out is None else out
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        pyc_reduce_batched(self._h, nseg, seg_offsets, ptrs, sc, out.data_ptr(), s)
        return out

    def autotune(self, n, stream=None):
        pyc_reduce_autotune(self._h, n, stream)

    @property
    def source(self):
        return pyc_reduce_source(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            pyc_reduce_destroy(self._h)


def argf32_from_tensor(t):
    """Decode ARGMIN/ARGMAX results stored as int64 pairs: returns (values, indices)."""
    import torch
    t = t.reshape(-1, 2).contiguous()
    words = t.view(torch.int32).reshape(-1, 4)  # little endian: word 0 is the value
    return words[:, 0].contiguous().view(torch.float32), t[:, 1]
