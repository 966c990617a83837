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


def _depth_bound(h, n, elem_bytes=4):
    """Worst-case depth of the addition tree behind one binary32 prefix for the
    launch configuration of n.  Within a tile: a lane's run of E elements, the
    5-level warp fold or scan of a row, at most R = 64*U rows of a warp, the
    warp-prefix scan (<= 5).  Across tiles: an inclusive prefix is an earlier
    one plus the aggregates after it, folded per lane (<= 3), across the warp
    (5), window after window (<= 1 per window) and with its own aggregate (1):
    <= 11 levels per hop, at most tau hops (tau = number of tiles)."""
    vec, unroll, block = pyc.launch_config(h, n, reduce="scan")
    e = vec // elem_bytes
    tau = -(-n // (block * e * unroll)) + 2
    return 11 * tau + 2 * (e + 5 + 64 * unroll + 5) + 10


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
        d = _depth_bound(stock.create("cumsum_f32"), n)
        assert np.all(np.abs(y - ref) <= d * U * ab * (1 + 1e-6) + 1e-30)


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
    """n = 2^28 binary32 prefix sums: every 4096th element and the last 4096;
    int32 -> int64 exclusive sums, every element.  Both in the launch
    configuration the benchmark times (tuned first)."""
    n = 1 << 28
    for name in ("cumsum_f32", "cumsum_excl_i32_i64"):
        pyc.pyc_scan_autotune(stock.create(name), n, _s())
    x = inputs.uniform_f32(35, 0, n, -1.0, 1.0)
    y = _scan("cumsum_f32", x)
    ref, ab = oracle.scan_sum_f32(x)
    idx = np.concatenate([np.arange(0, n, 4096), np.arange(n - 4096, n)])
    err = np.abs(y[idx].astype(np.float64) - ref[idx])
    assert np.all(err <= _depth_bound(stock.create("cumsum_f32"), n) * U * ab[idx] * (1 + 1e-6))
    xi = inputs.int_uniform_i32(35, 1, n)
    yi = _scan("cumsum_excl_i32_i64", xi, out_dtype=torch.int64)
    assert np.array_equal(yi, oracle.scan_sum_i32_i64(xi, exclusive=True))
    torch.cuda.empty_cache()


def test_scan_beyond_2e31_elements():
    """n = 2^31 + 100003: int32 -> int64 exclusive prefix sums whose element
    indices, tile offsets and look-back windows pass 2^31 (8.6 GB in, 17.2 GB
    out).  The input is 1 everywhere except two windows of seeded values in
    [-2^30, 2^30) (one across 2^31, one at the end), so every prefix has a
    closed form: the ones before i plus the windows' elements before i."""
    n = (1 << 31) + 100003
    wins = [((1 << 31) - 70000, (1 << 31) + 70001), (n - 3000, n)]
    x = torch.ones(n, dtype=torch.int32, device="cuda")
    vals, cums = [], []
    for k, (a, b) in enumerate(wins):
        v = inputs.int_uniform_i32(36, k, b - a, -(1 << 30), 1 << 30)
        x[a:b] = torch.from_numpy(v).cuda()
        vals.append(v)
        cums.append(np.concatenate([[0], np.cumsum(v.astype(np.int64))]))
    h = stock.create("cumsum_excl_i32_i64")
    y = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    pyc.pyc_scan_launch(h, n, [x.data_ptr(), y.data_ptr()], None, _s())
    pyc.pyc_scan_sync(h, _s())

    def want(i):
        s = i
        for (a, b), c in zip(wins, cums):
            m = min(max(i - a, 0), b - a)
            s += int(c[m]) - m
        return s

    # each window element by element: the closed form at its start plus the
    # oracle's exclusive prefix of the window
    for (a, b), v in zip(wins, vals):
        ref = want(a) + oracle.scan_sum_i32_i64(v, exclusive=True)
        assert np.array_equal(y[a:b].cpu().numpy(), ref), (a, b)
    idx = np.unique(np.concatenate([
        np.random.default_rng(37).integers(0, n, 4096),
        [0, 1, 2, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, n - 1],
        np.arange((1 << 31) - 70000 - 2048, (1 << 31) - 70000 + 2048)]))
    got = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    bad = [(int(i), int(g), want(int(i))) for g, i in zip(got, idx) if int(g) != want(int(i))]
    assert not bad, bad[:5]
    del x, y
    torch.cuda.empty_cache()


def _affine_inputs(seed, n):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    return a, b


def _u32_dev(a):
    return torch.from_numpy(a.view(np.int32)).cuda()


@pytest.mark.parametrize("vec,unroll,block", [(None, None, None), (16, 1, 32), (32, 4, 512),
                                              (16, 2, 160), (32, 1, 64)])
def test_noncommutative_scan_order(vec, unroll, block):
    """Composition of affine maps: any operand swapped in the warp scans, the
    block step or the look-back fold changes the result."""
    o = {} if vec is None else dict(vec_bytes=vec, items_per_thread=unroll, block=block)
    h = stock.create("affine_u32", **o)
    for n in (1, 2, 33, 4097, 200003, 3 * (1 << 20) + 5):
        a, b = _affine_inputs(n, n)
        da, db = _u32_dev(a), _u32_dev(b)
        dy = torch.zeros(n, dtype=torch.int64, device="cuda")
        pyc.pyc_scan_launch(h, n, [da.data_ptr(), db.data_ptr(), dy.data_ptr()], None, _s())
        pyc.pyc_scan_sync(h, _s())
        assert np.array_equal(dy.cpu().numpy().view(np.uint64), oracle.scan_affine_u32(a, b)), n


def test_noncommutative_scan_misaligned():
    """Arrays that share no vector alignment: every tile takes the ragged path."""
    h = stock.create("affine_u32")
    n = 100000
    a, b = _affine_inputs(7, n + 8)
    da, db = _u32_dev(a), _u32_dev(b)
    for oa, ob in ((1, 0), (0, 3), (2, 2), (3, 1)):
        dy = torch.zeros(n, dtype=torch.int64, device="cuda")
        pyc.pyc_scan_launch(h, n, [da.data_ptr() + 4 * oa, db.data_ptr() + 4 * ob, dy.data_ptr()],
                            None, _s())
        pyc.pyc_scan_sync(h, _s())
        want = oracle.scan_affine_u32(a[oa:oa + n], b[ob:ob + n])
        assert np.array_equal(dy.cpu().numpy().view(np.uint64), want), (oa, ob)


def test_repeated_launches_and_growth():
    """Back-to-back launches reuse the descriptors (a new epoch each); a larger
    n grows the workspace."""
    h = stock.create("cumsum_excl_i32_i64")
    for n in (5000, 5000, 1 << 22, 777, 1 << 24, 1 << 24):
        x = inputs.int_uniform_i32(40, n % 7, n)
        dx = torch.from_numpy(x).cuda()
        dy = torch.empty(n, dtype=torch.int64, device="cuda")
        pyc.pyc_scan_launch(h, n, [dx.data_ptr(), dy.data_ptr()], None, _s())
        pyc.pyc_scan_sync(h, _s())
        assert np.array_equal(dy.cpu().numpy(), oracle.scan_sum_i32_i64(x, exclusive=True)), n


def test_wait_gives_up_and_reports():
    """A tile that publishes nothing: the next tile's wait runs out after
    spin_limit polls, the launch completes, pyc_scan_sync reports
    PYC_E_TIMEOUT, and the next launch on the stream is correct."""
    h = pyc.pyc_scan_create(pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "y[i] = item",
                            "int *x, long long *y", {"vec_bytes": 16, "items_per_thread": 1,
                                                     "block": 128})
    try:
        n = 1 << 20
        x = inputs.int_uniform_i32(41, 0, n)
        dx = torch.from_numpy(x).cuda()
        dy = torch.empty(n, dtype=torch.int64, device="cuda")
        ptrs = [dx.data_ptr(), dy.data_ptr()]
        pyc.pyc_scan_launch_test(h, n, ptrs, None, _s(), stall_tile=1, spin_limit=1 << 12)
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_scan_sync(h, _s())
        assert e.value.status == pyc.PYC_E_TIMEOUT
        pyc.pyc_scan_sync(h, _s())  # the error was cleared
        pyc.pyc_scan_launch(h, n, ptrs, None, _s())
        pyc.pyc_scan_sync(h, _s())
        assert np.array_equal(dy.cpu().numpy(), oracle.scan_sum_i32_i64(x))
    finally:
        pyc.pyc_scan_destroy(h)
