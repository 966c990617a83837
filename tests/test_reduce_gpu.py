"""Map-reduce parity on the GPU through the C ABI (Sec. 3.2.5, Listing 3b):
closed forms, invariants, brute force over sizes and offsets, and the full-size
reductions against the oracle with the stated tolerances."""
import numpy as np
import pytest
import torch

import oracle
from bounds import U, compensated_sum_bound, plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu
I64MAX = 2 ** 63 - 1


def _s():
    return torch.cuda.current_stream().cuda_stream


def _decode(raw, dtype):
    """Result bytes -> Python value (argmin/argmax: (value, index))."""
    if dtype in (pyc.PYC_ARGMIN_F32, pyc.PYC_ARGMAX_F32):
        return float(raw[:4].view(np.float32)[0]), int(raw[8:16].view(np.int64)[0])
    return {pyc.PYC_F32: lambda: float(raw[:4].view(np.float32)[0]),
            pyc.PYC_F64: lambda: float(raw[:8].view(np.float64)[0]),
            pyc.PYC_I64: lambda: int(raw[:8].view(np.int64)[0])}[dtype]()


def _reduce(name, arrays, n=None, **opts):
    h = stock.create(name, **opts)
    ds = [a if isinstance(a, torch.Tensor) else torch.from_numpy(a).cuda() for a in arrays]
    n = ds[0].numel() if n is None else n
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    pyc.pyc_reduce_launch(h, n, [d.data_ptr() for d in ds], None, out.data_ptr(), _s())
    torch.cuda.synchronize()
    return _decode(out.cpu().numpy().view(np.uint8), stock.REDUCES[name][0])


def test_listing3b_dot_arange400():
    a = np.arange(400, dtype=np.float32)
    r = _reduce("dot_f32", [a, a])
    ref, ab = oracle.dot_f32(a, a)
    assert ref == 21253400
    assert abs(r - ref) <= plain_sum_bound(ab)
    # a one-accumulator serial loop misses by 16; short chains + tree do better
    assert abs(r - ref) < 16


def test_listing3b_front_end_result_stays_on_device():
    k = pyc.ReductionKernel(pyc.PYC_F32, neutral="0", reduce_expr="a+b", map_expr="x[i]*y[i]",
                            arguments="float *x, float *y")
    a = torch.arange(400, dtype=torch.float32, device="cuda")
    out = k(a, a)
    assert out.is_cuda and out.numel() == 1
    assert abs(out.item() - 21253400) <= 10


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 32, 33, 255, 256, 4095, 4096, 4097, 70001, 1 << 20,
                               5000000])
def test_closed_forms(n):
    idx = np.arange(n, dtype=np.float32)
    if n < 5000:  # every partial sum is an integer below 2^24: exact in any order
        assert _reduce("sum_f32", [idx]) == n * (n - 1) // 2
    alt = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    assert _reduce("sum_f32", [alt]) == n % 2
    c, d = np.full(n, 0.375, np.float32), np.full(n, -6.0, np.float32)
    if n < (1 << 21):
        assert _reduce("dot_f32", [c, d]) == -2.25 * n
    assert _reduce("dot_f32", [alt, c]) == 0.375 * (n % 2)
    ii = np.arange(n, dtype=np.int32)
    assert _reduce("sum_i32_i64", [ii]) == n * (n - 1) // 2


def test_neutral_for_empty_input():
    z = torch.zeros(4, device="cuda")
    assert _reduce("sum_f32", [z], n=0) == 0.0
    assert _reduce("max_f32", [z], n=0) == float("-inf")
    assert _reduce("argmin_f32", [z], n=0) == (float("inf"), I64MAX)
    assert _reduce("argmax_f32", [z], n=0) == (float("-inf"), I64MAX)
    assert _reduce("sum_f32_comp", [z], n=0) == 0.0


def test_sum_of_x_and_minus_x_cancel():
    x = inputs.lognormal_signed_f32(3, 0, (1 << 22) + 77)
    a, b = _reduce("sum_f32", [x]), _reduce("sum_f32", [-x])
    assert a + b == 0.0
    assert _reduce("sum_f32", [x]) == a  # reproducible


def test_permutation_within_bound_and_exact_for_order_free_ops():
    n = (1 << 21) + 5
    x = inputs.lognormal_signed_f32(4, 0, n)
    p = np.random.default_rng(0).permutation(n)
    ref, ab = oracle.sum_f32(x)
    for arr in (x, x[p]):
        assert abs(_reduce("sum_f32", [arr]) - ref) <= plain_sum_bound(ab)
    assert _reduce("max_f32", [x]) == _reduce("max_f32", [x[p]]) == oracle.max_f32(x)
    xi = inputs.int_uniform_i32(4, 1, n)
    assert _reduce("sum_i32_i64", [xi]) == _reduce("sum_i32_i64", [xi[p]]) == oracle.sum_i32_i64(xi)


def _brute_reduce(name, arr, sizes, offsets, check):
    d = torch.from_numpy(arr).cuda()
    h = stock.create(name)
    ob = pyc.pyc_reduce_out_bytes(h)
    cases = [(o, n) for o in offsets for n in sizes]
    out = torch.zeros(len(cases) * max(ob, 8) // 8 * (2 if ob == 16 else 1) + 2, dtype=torch.int64,
                      device="cuda")
    for k, (o, n) in enumerate(cases):
        pyc.pyc_reduce_launch(h, n, [d.data_ptr() + o * arr.itemsize], None,
                              out.data_ptr() + k * ob, _s())
    torch.cuda.synchronize()
    raw = out.cpu().numpy().view(np.uint8)
    for k, (o, n) in enumerate(cases):
        check(raw[k * ob:(k + 1) * ob], arr[o:o + n])


def test_brute_force_int_sum_exact():
    arr = inputs.int_uniform_i32(5, 0, 1200 + 16)
    sizes = list(range(0, 1101))

    def chk(raw, a):
        assert int(raw.view(np.int64)[0]) == oracle.sum_i32_i64(a)
    _brute_reduce("sum_i32_i64", arr, sizes, list(range(16)), chk)


def test_brute_force_argmin_max_exact():
    arr = np.random.default_rng(5).integers(-8, 8, 1200 + 16).astype(np.float32)  # many ties
    sizes = list(range(1, 1101, 3))

    def chk_arg(raw, a):
        v = float(raw[:4].view(np.float32)[0])
        i = int(raw[8:16].view(np.int64)[0])
        assert (v, i) == oracle.argmin_f32(a)

    def chk_max(raw, a):
        assert float(raw[:4].view(np.float32)[0]) == oracle.max_f32(a)
    _brute_reduce("argmin_f32", arr, sizes, list(range(16)), chk_arg)
    _brute_reduce("max_f32", arr, sizes, [0, 1, 5, 15], chk_max)


def test_brute_force_float_sum_bound():
    arr = inputs.lognormal_signed_f32(6, 0, 1200 + 16)
    sizes = list(range(0, 1101, 5))

    def chk(raw, a):
        ref, ab = oracle.sum_f32(a)
        assert abs(float(raw[:4].view(np.float32)[0]) - ref) <= plain_sum_bound(ab) + 1e-38
    _brute_reduce("sum_f32", arr, sizes, list(range(0, 16, 3)), chk)


@pytest.mark.parametrize("vec,unroll,block", [(16, 1, 32), (16, 2, 64), (16, 4, 512),
                                              (32, 1, 128), (32, 2, 256), (32, 4, 96)])
def test_every_variant(vec, unroll, block):
    o = dict(vec_bytes=vec, items_per_thread=unroll, block=block)
    for n in (0, 1, 100, 4097, 65536 + 3, 1000003):
        x = inputs.lognormal_signed_f32(7, 0, n)
        y = inputs.uniform_f32(7, 1, n)
        ref, ab = oracle.dot_f32(x, y)
        assert abs(_reduce("dot_f32", [x, y], **o) - ref) <= plain_sum_bound(ab)
        xi = inputs.int_uniform_i32(7, 2, n)
        assert _reduce("sum_i32_i64", [xi], **o) == oracle.sum_i32_i64(xi)
        assert _reduce("argmin_f32", [x], **o) == oracle.argmin_f32(x)
        rc = _reduce("sum_f32_comp", [x], **o)
        assert abs(rc - oracle.exact_sum_f32(x)) <= compensated_sum_bound(oracle.exact_sum_f32(x),
                                                                          oracle.sum_f32(x)[1])


def test_dot_small_config():
    """Listing 3b at n = 2^20, uniform[-1,1) from seed 0 (streams 0 and 1), in
    the default and in the tuned configuration the benchmark times."""
    n = 1 << 20
    x = inputs.uniform_f32(0, 0, n, -1.0, 1.0)
    y = inputs.uniform_f32(0, 1, n, -1.0, 1.0)
    ref, ab = oracle.dot_f32(x, y)
    r = _reduce("dot_f32", [x, y])
    assert abs(r - ref) <= plain_sum_bound(ab)
    pyc.pyc_reduce_autotune(stock.create("dot_f32"), n, _s())
    r = _reduce("dot_f32", [x, y])
    assert abs(r - ref) <= plain_sum_bound(ab)
    bx = inputs.to_bf16_values(x)
    by = inputs.to_bf16_values(y)
    dbx = torch.from_numpy(bx).to(torch.bfloat16).cuda()
    dby = torch.from_numpy(by).to(torch.bfloat16).cuda()
    refb, abb = oracle.dot_f32(bx, by)
    assert abs(_reduce("dot_bf16", [dbx, dby]) - refb) <= plain_sum_bound(abb)


def test_full_size_reductions():
    """n = 2^28: plain vs compensated binary32 sums of lognormal(0,3) values with
    random sign, int32 -> int64 sum (bit-exact), max and argmin (bit-exact), each
    in the launch configuration the benchmark times (tuned first)."""
    n = 1 << 28
    for name in ("sum_f32", "sum_f32_comp", "max_f32", "sum_i32_i64", "argmin_f32"):
        pyc.pyc_reduce_autotune(stock.create(name), n, _s())
    x = inputs.lognormal_signed_f32(0, 0, n)
    dx = torch.from_numpy(x).cuda()
    exact = oracle.exact_sum_f32(x)
    ref, ab = oracle.sum_f32(x)
    assert abs(ref - exact) <= 2.0 ** -50 * ab
    rp = _reduce("sum_f32", [dx])
    rc = _reduce("sum_f32_comp", [dx])
    print("sum n=2^28: exact %.9g plain err %.3g (bound %.3g) compensated err %.3g (bound %.3g)"
          % (exact, abs(rp - exact), plain_sum_bound(ab), abs(rc - exact),
             compensated_sum_bound(exact, ab)))
    assert abs(rp - exact) <= plain_sum_bound(ab)
    assert abs(rc - exact) <= compensated_sum_bound(exact, ab)
    assert _reduce("max_f32", [dx]) == oracle.max_f32(x)
    del dx
    xi = inputs.int_uniform_i32(0, 0, n)
    assert _reduce("sum_i32_i64", [xi]) == oracle.sum_i32_i64(xi)
    del xi
    xa = inputs.argmin_with_minima(0, n)
    assert _reduce("argmin_f32", [xa]) == oracle.argmin_f32(xa)
    torch.cuda.empty_cache()


def test_argmin_boundary_positions():
    n = (1 << 24) + 11
    x = inputs.uniform_f32(8, 0, n, -2.0, 2.0)
    last = x.copy()
    last[-1] = -3.0  # only minimum at n-1
    assert _reduce("argmin_f32", [last]) == (-3.0, n - 1)
    tail = x.copy()
    tail[n - 1000:] = -3.0  # all minima in the last CTA's range
    assert _reduce("argmin_f32", [tail]) == (-3.0, n - 1000)
    same = np.full(n, 1.5, np.float32)
    assert _reduce("argmin_f32", [same]) == (1.5, 0)
    assert _reduce("argmax_f32", [same]) == (1.5, 0)


def test_two_streams_use_separate_workspaces():
    n = (1 << 22) + 1
    x = inputs.int_uniform_i32(9, 0, n)
    dx = torch.from_numpy(x).cuda()
    h = stock.create("sum_i32_i64")
    outs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(8)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    torch.cuda.synchronize()
    for k, o in enumerate(outs):
        s = streams[k % 2]
        pyc.pyc_reduce_launch(h, n, [dx.data_ptr()], None, o.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    want = oracle.sum_i32_i64(x)
    assert all(o.item() == want for o in outs)
