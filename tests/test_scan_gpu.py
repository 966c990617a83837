"""Parallel prefix scan parity on the GPU through the C ABI (Sec. 3.2.6)."""
import numpy as np
import pytest
import torch

import oracle
from bounds import U
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu


def _s():
    return torch.cuda.current_stream().cuda_stream


def _scan(name, x, n=None, out_dtype=torch.float32, **opts):
    h = stock.create(name, **opts)
    dx = x if isinstance(x, torch.Tensor) else torch.from_numpy(x).cuda()
    n = dx.numel() if n is None else n
    dy = torch.full((dx.numel(),), -7, dtype=out_dtype, device="cuda")
    pyc.pyc_scan_launch(h, n, [dx.data_ptr(), dy.data_ptr()], None, _s())
    torch.cuda.synchronize()
    return dy.cpu().numpy()


def _depth_bound(n):
    """Worst-case depth of the addition tree behind one prefix: rows of a chunk
    scanned one after another (at most n / (152 CTAs x 32 threads x 4 elements)),
    plus the per-thread runs, warp and block trees of both passes (< 256)."""
    return 256 + n // (152 * 32 * 4)


def test_integer_valued_floats_are_exact():
    # every partial sum is an integer below 2^24, so any association is exact:
    # this checks every index and every carry of the scan structure
    rng = np.random.default_rng(30)
    for n in (1, 2, 31, 32, 33, 1000, 4096, 4097, 65537, 1 << 20, (1 << 21) + 11):
        x = rng.integers(-8, 9, n).astype(np.float32)
        y = _scan("cumsum_f32", x)
        assert np.array_equal(y, np.cumsum(x.astype(np.int64)).astype(np.float32)), n


@pytest.mark.parametrize("vec,unroll,block", [(16, 1, 32), (16, 4, 256), (32, 2, 512),
                                              (32, 4, 128), (16, 2, 96)])
def test_every_variant_int_exact(vec, unroll, block):
    o = dict(vec_bytes=vec, items_per_thread=unroll, block=block)
    for n in (0, 1, 5, 1000, 65536 + 3, 1000003):
        x = inputs.int_uniform_i32(31, 0, n)
        y = _scan("cumsum_excl_i32_i64", x, out_dtype=torch.int64, **o)
        assert np.array_equal(y, oracle.scan_sum_i32_i64(x, exclusive=True)), n
        xf = np.random.default_rng(n).integers(-50, 50, n).astype(np.float32)
        assert np.array_equal(_scan("cummax_f32", xf, **o), oracle.scan_max_f32(xf)), n


def test_offsets_and_ragged_sizes():
    """Unaligned starts (scalar heads) and every small size."""
    base = inputs.int_uniform_i32(32, 0, 3000)
    dx = torch.from_numpy(base).cuda()
    h = stock.create("cumsum_excl_i32_i64")
    for off in range(0, 9):
        for n in list(range(0, 70)) + [255, 256, 257, 1025, 2000]:
            dy = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
            pyc.pyc_scan_launch(h, n, [dx.data_ptr() + 4 * off, dy.data_ptr()], None, _s())
            torch.cuda.synchronize()
            y = dy.cpu().numpy()
            assert np.array_equal(y[:n], oracle.scan_sum_i32_i64(base[off:off + n], exclusive=True))
            assert y[n] == -7  # nothing written past n


def test_float_scan_within_bound():
    for n in (100003, 1 << 22):
        x = inputs.uniform_f32(33, 0, n, -1.0, 1.0)
        y = _scan("cumsum_f32", x).astype(np.float64)
        ref, ab = oracle.scan_sum_f32(x)
        assert np.all(np.abs(y - ref) <= _depth_bound(n) * U * ab + 1e-30)


def test_in_place_scan():
    h = pyc.pyc_scan_create(pyc.PYC_F32, "0", "a+b", "x[i]", "x[i] = item", "float *x")
    try:
        n = 300001
        x = np.random.default_rng(34).integers(-4, 5, n).astype(np.float32)
        dx = torch.from_numpy(x.copy()).cuda()
        pyc.pyc_scan_launch(h, n, [dx.data_ptr()], None, _s())
        torch.cuda.synchronize()
        assert np.array_equal(dx.cpu().numpy(), np.cumsum(x.astype(np.int64)).astype(np.float32))
    finally:
        pyc.pyc_scan_destroy(h)


def test_full_size_scan_sampled():
    """n = 2^28 binary32 prefix sums: every 4096th element and the last 4096."""
    n = 1 << 28
    x = inputs.uniform_f32(35, 0, n, -1.0, 1.0)
    y = _scan("cumsum_f32", x)
    ref, ab = oracle.scan_sum_f32(x)
    idx = np.concatenate([np.arange(0, n, 4096), np.arange(n - 4096, n)])
    err = np.abs(y[idx].astype(np.float64) - ref[idx])
    assert np.all(err <= _depth_bound(n) * U * ab[idx])
    xi = inputs.int_uniform_i32(35, 1, n)
    yi = _scan("cumsum_excl_i32_i64", xi, out_dtype=torch.int64)
    assert np.array_equal(yi, oracle.scan_sum_i32_i64(xi, exclusive=True))
    torch.cuda.empty_cache()
