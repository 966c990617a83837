"""Map and map-reduce parity on the GPU for the storage types of the argument
spec beyond binary32 / bfloat16 (Sec. 3.1 type strings; map Sec. 3.2.4,
map-reduce Sec. 3.2.5): binary16 ``__half``, binary64 ``double``, ``int``,
``long long`` and a statement that mixes them (C promotion), through the C ABI,
against ``oracle/storage.py``.

Maps are bit-exact (each operation rounds once, in source order, no
contraction; a binary16 store rounds the binary32 value once).  Sizes span
several tiles with ragged tails; offsets exercise the scalar head (equal
misalignment) and the element-wise path (unequal misalignment).
"""
import math

import numpy as np
import pytest
import torch

from bounds import U
from oracle import storage
from paper_1304_5553_gb300 import inputs, pyc

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 5, 4099, 70001, (1 << 20) + 3]
U64 = 2.0 ** -53
_handles = {}


def _s():
    return torch.cuda.current_stream().cuda_stream


def _map(spec, stmt):
    key = ("map", spec, stmt)
    if key not in _handles:
        _handles[key] = pyc.pyc_map_create(spec, stmt)
    return _handles[key]


def _red(out, neutral, red, mexpr, spec):
    key = ("red", out, neutral, red, mexpr, spec)
    if key not in _handles:
        _handles[key] = pyc.pyc_reduce_create(out, neutral, red, mexpr, spec)
    return _handles[key]


def _dev(a, off=0):
    """Device copy of the numpy array a starting `off` elements into a larger buffer."""
    t = torch.from_numpy(np.ascontiguousarray(a))
    buf = torch.zeros(t.numel() + 8, dtype=t.dtype, device="cuda")
    v = buf[off:off + t.numel()]
    v.copy_(t.cuda())
    return v


def _f16(seed, stream, n, lo=-2.0, hi=2.0):
    return inputs.to_f16_values(inputs.uniform_f32(seed, stream, n, lo, hi))


def _f64(seed, stream, n, lo=-2.0, hi=2.0):
    return lo + (hi - lo) * inputs.unit_f64(seed, stream, n)


def _run_map(h, n, arrays, out_np_dtype, scalars, offs):
    ins = [_dev(a, o) for a, o in zip(arrays, offs[:-1])]
    zbuf = torch.zeros(n + 8, dtype=out_np_dtype, device="cuda")
    z = zbuf[offs[-1]:offs[-1] + n]
    ptrs = [t.data_ptr() for t in ins] + [z.data_ptr()]
    pyc.pyc_map_launch(h, n, ptrs, pyc.pack_scalars(h, scalars), _s())
    torch.cuda.synchronize()
    return z.cpu().numpy(), zbuf


# ---------------------------------------------------------------------------- maps

@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("offs", [(0, 0, 0), (3, 3, 3), (1, 2, 0)])
def test_half_storage_lin_comb_bit_exact(n, offs):
    h = _map("float a, __half *x, float b, __half *y, __half *z", "z[i] = a*x[i] + b*y[i]")
    x, y = _f16(20, 0, n), _f16(20, 1, n)
    got, zbuf = _run_map(h, n, [x, y], torch.float16, [2.5, -0.75], offs)
    want = storage.lin_comb_f16(2.5, x, -0.75, y)
    assert np.array_equal(got.view(np.uint16), want.view(np.uint16))
    # nothing written outside [0, n) of the output view
    rest = torch.cat([zbuf[:offs[2]], zbuf[offs[2] + n:]])
    assert int(torch.count_nonzero(rest)) == 0


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("offs", [(0, 0, 0), (1, 1, 1), (1, 0, 0)])
def test_double_storage_lin_comb_bit_exact(n, offs):
    h = _map("double a, double *x, double b, double *y, double *z", "z[i] = a*x[i] + b*y[i]")
    x, y = _f64(21, 0, n), _f64(21, 1, n)
    a, b = 2.5, -0.7  # -0.7 is not a short binary fraction: b*y rounds
    got, _ = _run_map(h, n, [x, y], torch.float64, [a, b], offs)
    want = storage.lin_comb_f64(a, x, b, y)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("n", SIZES)
def test_long_long_storage_lin_comb_exact(n):
    h = _map("long long a, long long *x, long long b, long long *y, long long *z",
             "z[i] = a*x[i] + b*y[i]")
    # values up to 2^40 in magnitude: products and the sum stay inside int64
    x = inputs.int_uniform_i32(22, 0, n).astype(np.int64) * (1 << 20) + \
        inputs.int_uniform_i32(22, 1, n)
    y = inputs.int_uniform_i32(22, 2, n).astype(np.int64) * (1 << 20) + \
        inputs.int_uniform_i32(22, 3, n)
    got, _ = _run_map(h, n, [x, y], torch.int64, [3, -7], (0, 1, 0))
    assert np.array_equal(got, storage.lin_comb_int(3, x, -7, y, 64))


@pytest.mark.parametrize("n", SIZES)
def test_int_storage_lin_comb_exact(n):
    h = _map("int a, int *x, int b, int *y, int *z", "z[i] = a*x[i] + b*y[i]")
    x, y = inputs.int_uniform_i32(23, 0, n), inputs.int_uniform_i32(23, 1, n)
    got, _ = _run_map(h, n, [x, y], torch.int32, [3, -7], (2, 2, 2))
    assert np.array_equal(got, storage.lin_comb_int(3, x, -7, y, 32))


@pytest.mark.parametrize("n", [1, 4099, (1 << 20) + 3])
def test_mixed_types_follow_c_promotion(n):
    h = _map("__half *x, double *y, float *z", "z[i] = x[i] + y[i]")
    x = _f16(24, 0, n)
    # y spans many binades so the binary64 sum and the binary32 store both round
    y = _f64(24, 1, n, -1, 1) * np.exp2(inputs.int_uniform_i32(24, 2, n, -40, 10))
    got, _ = _run_map(h, n, [x, y], torch.float32, [], (0, 0, 0))
    want = storage.add_f16_f64_to_f32(x, y)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# ---------------------------------------------------------------------------- reductions

def _reduce(h, n, arrays, out_dtype, offs=None):
    offs = offs or [0] * len(arrays)
    ds = [a if isinstance(a, torch.Tensor) else _dev(a, o) for a, o in zip(arrays, offs)]
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    pyc.pyc_reduce_launch(h, n, [d.data_ptr() for d in ds], None, out.data_ptr(), _s())
    torch.cuda.synchronize()
    raw = out.cpu().numpy().view(np.uint8)
    return {pyc.PYC_F64: lambda: float(raw[:8].view(np.float64)[0]),
            pyc.PYC_F32: lambda: float(raw[:4].view(np.float32)[0]),
            pyc.PYC_F16: lambda: float(raw[:2].view(np.float16)[0]),
            pyc.PYC_I64: lambda: int(raw[:8].view(np.int64)[0]),
            pyc.PYC_I32: lambda: int(raw[:4].view(np.int32)[0])}[out_dtype]()


def _gamma(k, u):
    """gamma_k = k u / (1 - k u): bound on the relative error of any summation
    order of k + 1 terms (recursive or tree), relative to the sum of |terms|."""
    return k * u / (1 - k * u)


@pytest.mark.parametrize("n", SIZES + [5000000])
def test_double_sum_integer_values_exact(n):
    # integer-valued binary64 terms whose partial sums stay below 2^53: every
    # association order gives the exact sum
    h = _red(pyc.PYC_F64, "0", "a+b", "x[i]", "double *x")
    x = inputs.int_uniform_i32(25, 0, n).astype(np.float64)
    assert _reduce(h, n, [x], pyc.PYC_F64, [1]) == storage.sum_int(x.astype(np.int64))


@pytest.mark.parametrize("n", [4099, (1 << 20) + 3, 5000000])
def test_double_sum_within_any_order_bound(n):
    h = _red(pyc.PYC_F64, "0", "a+b", "x[i]", "double *x")
    x = _f64(26, 0, n) * np.exp2(inputs.int_uniform_i32(26, 1, n, -20, 20))
    r = _reduce(h, n, [x], pyc.PYC_F64)
    s, ab = storage.sum_exact(x)
    assert abs(r - s) <= _gamma(n - 1, U64) * ab
    # fixed association order: the sum of -x is exactly the negated sum
    assert _reduce(h, n, [-x], pyc.PYC_F64) == -r


@pytest.mark.parametrize("n", [1, 4099, (1 << 20) + 3])
def test_half_dot_binary32_and_binary16_results(n):
    spec = "__half *x, __half *y"
    x, y = _f16(27, 0, n), _f16(27, 1, n)
    s, ab = storage.dot_exact_f16(x, y)
    # binary32 result: products of binary16 values are exact in binary32, the sum
    # is a plain binary32 reduction (stated tolerance 8 u sum|terms|)
    r32 = _reduce(_red(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", spec), n, [x, y], pyc.PYC_F32)
    assert abs(r32 - s) <= 8 * U * ab
    # binary16 result: binary32 accumulation, then one rounding to binary16
    # (unit roundoff 2^-11)
    r16 = _reduce(_red(pyc.PYC_F16, "0", "a+b", "x[i]*y[i]", spec), n, [x, y], pyc.PYC_F16)
    acc = 8 * U * ab
    assert abs(r16 - s) <= 2.0 ** -11 * (abs(s) + acc) + acc


@pytest.mark.parametrize("n", SIZES)
def test_long_long_sum_and_int_extrema_exact(n):
    # |x| < 2^41, so at most 2^21 terms cannot leave int64
    x = inputs.int_uniform_i32(28, 0, n).astype(np.int64) * (1 << 20) + \
        inputs.int_uniform_i32(28, 1, n)
    hs = _red(pyc.PYC_I64, "0", "a+b", "x[i]", "long long *x")
    assert _reduce(hs, n, [x], pyc.PYC_I64, [1]) == storage.sum_int(x)
    xi = inputs.int_uniform_i32(28, 2, n, -(2 ** 31), 2 ** 31 - 1)
    hmax = _red(pyc.PYC_I32, "-2147483647-1", "a > b ? a : b", "x[i]", "int *x")
    hmin = _red(pyc.PYC_I32, "2147483647", "a < b ? a : b", "x[i]", "int *x")
    assert _reduce(hmax, n, [xi], pyc.PYC_I32) == storage.max_value(xi, -2 ** 31)
    assert _reduce(hmin, n, [xi], pyc.PYC_I32, [3]) == storage.min_value(xi, 2 ** 31 - 1)


@pytest.mark.parametrize("n", [1, 70001, (1 << 20) + 3])
def test_double_min_exact(n):
    h = _red(pyc.PYC_F64, "INFINITY", "a < b ? a : b", "x[i]", "double *x")
    x = _f64(29, 0, n)
    assert _reduce(h, n, [x], pyc.PYC_F64, [1]) == storage.min_value(x, math.inf)
    assert math.isinf(_reduce(h, 0, [x], pyc.PYC_F64))


def test_u8_map_and_sum_beyond_32bit_indices():
    """Maximum sizes: 2^32 + 19 one-byte elements, so element indices pass both the
    int32 and the uint32 range (the formal index i is 64-bit).  x repeats a seeded
    block of 2^20 bytes; the map mixes in bits 20.. of i, so an index that wrapped
    or was truncated anywhere gives a wrong byte."""
    n = (1 << 32) + 19
    blk_n = 1 << 20
    block = inputs.int_uniform_i32(30, 0, blk_n, 0, 255).astype(np.uint8)
    x = torch.from_numpy(block).cuda().repeat(-(-n // blk_n))[:n]
    z = torch.empty(n, dtype=torch.uint8, device="cuda")
    h = _map("unsigned char *x, unsigned char *z", "z[i] = x[i] + (unsigned char)(i >> 20)")
    pyc.pyc_map_launch(h, n, [x.data_ptr(), z.data_ptr()], None, _s())
    torch.cuda.synchronize()
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([
        np.arange(0, 4096), np.arange(n - 8192, n),
        np.arange(2 ** 31 - 4096, 2 ** 31 + 4096), rng.integers(0, n, 16384)])).astype(np.int64)
    got = z[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(got, storage.map_u8_add_index(block[idx % blk_n], idx, 20))
    del z
    # sum of all 2^32 + 19 bytes into int64: whole blocks plus the ragged rest
    hs = _red(pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "unsigned char *x")
    full, rem = divmod(n, blk_n)
    want = full * storage.sum_int(block) + storage.sum_int(block[:rem])
    assert _reduce(hs, n, [x], pyc.PYC_I64) == want
