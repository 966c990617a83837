"""GPUArray-style arithmetic on device arrays, fused into one kernel per expression.

Sec. 3.2.3 gives GPUArray numpy-like operators, and Sec. 3.2.4 notes that
evaluating nested expressions with them makes a temporary per intermediate
result.  Here operators on `GArray` build an expression tree instead;
`evaluate` (or `GArray.assign`) compiles the whole tree into ONE map kernel
through `pyc_expr_map_create` (prefix text, cached per expression shape and
types) and launches it, and `sum` / `max` / `min` / `dot` compile it into one
map-reduce.  `evaluate_eager` runs the tree node by node, one kernel and one
temporary per node, as operator-at-a-time GPUArray arithmetic does; it is the
unfused baseline.

    x, y = GArray(tx), GArray(ty)
    z = evaluate(x * exp(-y * y) + sin(u) * w)          # one kernel
    s = sum(x * y)                                       # one map-reduce

`set_pool` makes outputs and temporaries come from a device memory pool
(Sec. 3.2.6: pools integrate with GPUArray, whose operators allocate and free
arrays of recurring sizes).

Python scalars become scalar kernel arguments (no recompilation when their
value changes): binary64 if an F64 array appears in the expression, else
binary32; integers int32 (int64 if they do not fit).
"""
from __future__ import annotations

import threading

from . import pyc

_DT = None


def _dtypes():
    global _DT
    if _DT is None:
        import torch
        _DT = {torch.float32: pyc.PYC_F32, torch.float64: pyc.PYC_F64,
               torch.bfloat16: pyc.PYC_BF16, torch.float16: pyc.PYC_F16,
               torch.int32: pyc.PYC_I32, torch.int64: pyc.PYC_I64}
    return _DT


class Expr:
    """A node: operator name and operands (Expr, GArray or Python numbers)."""
    __slots__ = ("op", "args")
    __array_priority__ = 100

    def __init__(self, op, *args):
        self.op = op
        self.args = args

    # arithmetic builds nodes
    def __add__(self, o): return Expr("+", self, o)
    def __radd__(self, o): return Expr("+", o, self)
    def __sub__(self, o): return Expr("-", self, o)
    def __rsub__(self, o): return Expr("-", o, self)
    def __mul__(self, o): return Expr("*", self, o)
    def __rmul__(self, o): return Expr("*", o, self)
    def __truediv__(self, o): return Expr("/", self, o)
    def __rtruediv__(self, o): return Expr("/", o, self)
    def __pow__(self, o): return Expr("pow", self, o)
    def __rpow__(self, o): return Expr("pow", o, self)
    def __neg__(self): return Expr("neg", self)
    def __abs__(self): return Expr("abs", self)
    def __lt__(self, o): return Expr("<", self, o)
    def __le__(self, o): return Expr("<=", self, o)
    def __gt__(self, o): return Expr(">", self, o)
    def __ge__(self, o): return Expr(">=", self, o)
    def eq(self, o): return Expr("==", self, o)
    def ne(self, o): return Expr("!=", self, o)
    def astype(self, dtype):
        if not _CAST:
            _init_casts()
        if dtype not in _CAST:
            raise TypeError("astype takes torch.float32, float64, int32 or int64, not %s" % dtype)
        return Expr(_CAST[dtype], self)


class GArray(Expr):
    """A 1-D contiguous CUDA tensor as an expression leaf (`.tensor` is the data)."""
    __slots__ = ("tensor",)

    def __init__(self, tensor):
        import torch
        if not isinstance(tensor, torch.Tensor) or not tensor.is_cuda:
            raise TypeError("GArray needs a CUDA tensor")
        if tensor.dim() != 1 or not tensor.is_contiguous():
            raise ValueError("GArray needs a contiguous 1-D tensor")
        if tensor.dtype not in _dtypes():
            raise TypeError("unsupported dtype %s" % tensor.dtype)
        Expr.__init__(self, "leaf")
        self.tensor = tensor

    @property
    def dtype(self):
        return _dtypes()[self.tensor.dtype]

    def __len__(self):
        return self.tensor.numel()

    def assign(self, expr, stream=None):
        """self[:] = expr, fused (the output may be one of the operands: in place)."""
        evaluate(expr, out=self, stream=stream)
        return self


def _unary(name):
    def f(x):
        return Expr(name, x)
    f.__name__ = name
    f.__doc__ = "Element-wise %s (CUDA's math function for the operand type)." % name
    return f


exp, exp2, log, log2 = _unary("exp"), _unary("exp2"), _unary("log"), _unary("log2")
sin, cos, tan, tanh = _unary("sin"), _unary("cos"), _unary("tan"), _unary("tanh")
sqrt, rsqrt, floor, ceil = _unary("sqrt"), _unary("rsqrt"), _unary("floor"), _unary("ceil")
fabs = _unary("abs")


def minimum(a, b): return Expr("min", a, b)
def maximum(a, b): return Expr("max", a, b)
def where(c, a, b): return Expr("where", c, a, b)


_CAST = {}


def _init_casts():
    import torch
    _CAST.update({torch.float32: "f32", torch.float64: "f64", torch.int32: "i32",
                  torch.int64: "i64"})


# ------------------------------------------------------------------ compilation

class _Lowered:
    """The prefix text of a tree and its arguments (arrays by identity, scalars)."""

    def __init__(self, root):
        self.arrays = []       # GArray leaves in slot order (deduplicated)
        self.array_slot = {}   # id(tensor) -> slot
        self.args = []         # (dtype, is_array, value)
        self.has_f64 = False
        self._scan(root)
        self.text = self._text(root)

    def _scan(self, e):
        if isinstance(e, GArray):
            if e.dtype == pyc.PYC_F64:
                self.has_f64 = True
        elif isinstance(e, Expr):
            for a in e.args:
                self._scan(a)

    def _text(self, e):
        if isinstance(e, GArray):
            key = id(e.tensor)
            if key not in self.array_slot:
                self.array_slot[key] = len(self.args)
                self.args.append((e.dtype, True, e))
                self.arrays.append(e)
            return "$%d" % self.array_slot[key]
        if isinstance(e, Expr):
            return "(" + e.op + " " + " ".join(self._text(a) for a in e.args) + ")"
        if isinstance(e, bool):
            e = int(e)
        if isinstance(e, int):
            dt = pyc.PYC_I32 if -2 ** 31 <= e < 2 ** 31 else pyc.PYC_I64
        elif isinstance(e, float):
            dt = pyc.PYC_F64 if self.has_f64 else pyc.PYC_F32
        else:
            import torch
            if isinstance(e, torch.Tensor) and e.is_cuda:
                return self._text(GArray(e.reshape(-1)) if e.dim() != 1 else GArray(e))
            raise TypeError("unsupported operand %r" % (e,))
        self.args.append((dt, False, e))
        return "%%%d" % (len(self.args) - 1)

    @property
    def key(self):
        return (self.text, tuple((d, a) for d, a, _ in self.args))

    def n(self):
        if not self.arrays:
            raise ValueError("an expression needs at least one array")
        n = len(self.arrays[0])
        for a in self.arrays:
            if len(a) != n:  # equal lengths (Sec. 3.2.4)
                raise ValueError("all arrays of an expression must have the same length")
        return n

    def result_dtype(self):
        """The expression's type under the library's rules (for a default output)."""
        return pyc.pyc_expr_type(self.text, [d for d, _, _ in self.args],
                                 [a for _, a, _ in self.args])


_cache = {}
_lock = threading.Lock()
_pool = [None]


def set_pool(pool):
    """Allocate expression outputs (and the temporaries of evaluate_eager) from a
    device memory pool (pyc_pool_create(PYC_POOL_DEVICE)); None: torch's allocator."""
    _pool[0] = pool


def _empty(n, dtype, device, stream):
    import torch
    if _pool[0] is not None:
        return pyc.pool_empty(_pool[0], n, dtype, stream)
    return torch.empty(n, dtype=dtype, device=device)


def _map_handle(low, out_dtype):
    key = ("map", low.key, out_dtype)
    with _lock:
        h = _cache.get(key)
    if h is None:
        h = pyc.pyc_expr_map_create(low.text, [d for d, _, _ in low.args],
                                    [a for _, a, _ in low.args], out_dtype)
        with _lock:
            h = _cache.setdefault(key, h)
    return h


def _reduce_handle(low, out_dtype, reduce):
    key = ("reduce", low.key, out_dtype, reduce)
    with _lock:
        h = _cache.get(key)
    if h is None:
        h = pyc.pyc_expr_reduce_create(low.text, [d for d, _, _ in low.args],
                                       [a for _, a, _ in low.args], out_dtype, reduce)
        with _lock:
            h = _cache.setdefault(key, h)
    return h


def _stream(stream):
    import torch
    return stream if stream is not None else torch.cuda.current_stream().cuda_stream


def _launch_args(low, h, reduce):
    scal = [v for _, a, v in low.args if not a]
    ptrs = [g.tensor.data_ptr() for g in low.arrays]
    return ptrs, pyc.pack_scalars(h, scal, reduce)


def evaluate(expr, out=None, dtype=None, stream=None):
    """Evaluate `expr` in one kernel; returns the output GArray (new unless given)."""
    import torch
    if not _CAST:
        _init_casts()
    if not isinstance(expr, Expr):
        raise TypeError("evaluate needs an expression")
    low = _Lowered(expr)
    n = low.n()
    if out is None:
        od = dtype if dtype is not None else low.result_dtype()
        out = GArray(_empty(n, pyc._torch_dtype(od), low.arrays[0].tensor.device, stream))
    elif not isinstance(out, GArray):
        out = GArray(out)
    if len(out) != n:
        raise ValueError("output length differs from the operands'")
    h = _map_handle(low, out.dtype)
    ptrs, sc = _launch_args(low, h, False)
    pyc.pyc_map_launch(h, n, ptrs + [out.tensor.data_ptr()], sc, _stream(stream))
    return out


def autotune(expr, out_dtype=None, stream=None):
    """Time the launch variants of the kernel `evaluate(expr)` uses, at its n, and
    keep the fastest (persisted by the tuning cache)."""
    if not _CAST:
        _init_casts()
    low = _Lowered(expr)
    od = out_dtype if out_dtype is not None else low.result_dtype()
    pyc.pyc_map_autotune(_map_handle(low, od), low.n(), _stream(stream))


def _reduce(expr, reduce, dtype, stream):
    import torch
    if not _CAST:
        _init_casts()
    if not isinstance(expr, Expr):
        raise TypeError("a reduction needs an expression or a GArray")
    low = _Lowered(expr)
    n = low.n()
    rd = low.result_dtype()
    if dtype is None:
        dtype = pyc.PYC_I64 if rd in (pyc.PYC_I32, pyc.PYC_I64) and reduce == "sum" else rd
    h = _reduce_handle(low, dtype, reduce)
    ptrs, sc = _launch_args(low, h, True)
    out = torch.empty(1, dtype=pyc._torch_dtype(dtype), device=low.arrays[0].tensor.device)
    pyc.pyc_reduce_launch(h, n, ptrs, sc, out.data_ptr(), _stream(stream))
    return out


def sum(expr, dtype=None, stream=None):  # noqa: A001 -- numpy's name
    """Sum of the expression's elements in one map-reduce (a 1-element device tensor)."""
    return _reduce(expr, "sum", dtype, stream)


def max(expr, dtype=None, stream=None):  # noqa: A001
    return _reduce(expr, "max", dtype, stream)


def min(expr, dtype=None, stream=None):  # noqa: A001
    return _reduce(expr, "min", dtype, stream)


def dot(a, b, dtype=None, stream=None):
    """sum(a*b) in one pass (Listing 3b)."""
    return _reduce(Expr("*", a, b), "sum", dtype, stream)


# ------------------------------------------------------------------ eager (unfused)

def evaluate_eager(expr, stream=None):
    """Operator-at-a-time evaluation: every node is its own kernel writing a new
    temporary array (what Sec. 3.2.4 calls inefficient); returns (result, kernels)."""
    launches = [0]

    def rec(e):
        if isinstance(e, GArray) or not isinstance(e, Expr):
            return e
        kids = [rec(a) for a in e.args]
        launches[0] += 1
        return evaluate(Expr(e.op, *kids), stream=stream)

    r = rec(expr)
    if not isinstance(r, GArray):
        raise ValueError("an expression needs at least one array")
    return r, launches[0]
