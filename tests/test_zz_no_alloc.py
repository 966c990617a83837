"""pyc_reduce_launch_static, the map-reduce launch that allocates nothing.

It serves callers that cannot allocate device memory when they launch (a
fixed memory footprint reserved at start-up, device memory owned by an outside
manager, or a latency budget an allocation would break).  It runs the same
kernel and chunk plan as pyc_reduce_launch with its partials and ticket in a
static scratch area of the library, so its results must match the regular
entry point's; after the first call on the device (the set-up) it must not
change the device's free memory.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
from bounds import compensated_sum_bound, plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 33, 4097, (1 << 20) + 3, 1 << 24]


def _s():
    return torch.cuda.current_stream().cuda_stream


def _outputs(name, arrays, n):
    """(regular result, static result of call 1, static result of call 2) as raw bytes."""
    h = stock.create(name)
    ptrs = [a.data_ptr() for a in arrays]
    outs = [torch.zeros(2, dtype=torch.int64, device="cuda") for _ in range(3)]
    pyc.pyc_reduce_launch(h, n, ptrs, None, outs[0].data_ptr(), _s())
    pyc.pyc_reduce_launch_static(h, n, ptrs, None, outs[1].data_ptr(), _s())
    pyc.pyc_reduce_launch_static(h, n, ptrs, None, outs[2].data_ptr(), _s())
    torch.cuda.synchronize()
    return [o.cpu().numpy().view(np.uint8) for o in outs]


def test_static_launch_matches_regular_on_two_calls():
    nmax = max(SIZES)
    x = inputs.lognormal_signed_f32(21, 0, nmax)
    y = inputs.uniform_f32(21, 1, nmax, -1.0, 1.0)
    xi = inputs.int_uniform_i32(21, 2, nmax)
    dx, dy, dxi = (torch.from_numpy(a).cuda() for a in (x, y, xi))
    for n in SIZES:
        # binary32 dot: both entry points within the plain-sum tolerance of the oracle
        ref, ab = oracle.dot_f32(x[:n], y[:n])
        r = [float(o[:4].view(np.float32)[0]) for o in _outputs("dot_f32", [dx, dy], n)]
        for v in r:
            assert abs(v - ref) <= plain_sum_bound(ab)
        assert abs(r[1] - r[0]) <= plain_sum_bound(ab) and abs(r[2] - r[0]) <= plain_sum_bound(ab)
        # compensated binary32 sum
        ex = oracle.exact_sum_f32(x[:n])
        sab = oracle.sum_f32(x[:n])[1]
        r = [float(o[:4].view(np.float32)[0]) for o in _outputs("sum_f32_comp", [dx], n)]
        for v in r:
            assert abs(v - ex) <= compensated_sum_bound(ex, sab)
        # integer sum and argmin: exact, so the two entry points agree bit for bit
        r = [int(o[:8].view(np.int64)[0]) for o in _outputs("sum_i32_i64", [dxi], n)]
        assert r[0] == r[1] == r[2] == oracle.sum_i32_i64(xi[:n])
        r = [(float(o[:4].view(np.float32)[0]), int(o[8:16].view(np.int64)[0]))
             for o in _outputs("argmin_f32", [dx], n)]
        assert r[0] == r[1] == r[2] == oracle.argmin_f32(x[:n])


def test_no_device_allocation_after_setup():
    n = (1 << 22) + 5
    x = torch.from_numpy(inputs.lognormal_signed_f32(22, 0, n)).cuda()
    outs = torch.zeros(16, 2, dtype=torch.int64, device="cuda")
    names = ["sum_f32", "sum_f32_comp", "max_f32", "argmin_f32"]
    hs = [stock.create(k) for k in names]
    for h in hs:  # set-up: first call on this device for each handle
        pyc.pyc_reduce_launch_static(h, n, [x.data_ptr()], None, outs[0].data_ptr(), _s())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(16):
        h = hs[k % len(hs)]
        pyc.pyc_reduce_launch_static(h, n - 7 * k, [x.data_ptr()], None, outs[k].data_ptr(), _s())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_rejects_bad_arguments():
    h = stock.create("sum_f32")
    x = torch.zeros(8, device="cuda")
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_launch_static(h, -1, [x.data_ptr()], None, x.data_ptr(), _s())
    assert e.value.status == pyc.PYC_E_ARG
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_launch_static(h, 8, [x.data_ptr()], None, 0, _s())
    assert e.value.status == pyc.PYC_E_ARG


def test_scratch_address_is_kept_per_context():
    """The scratch address is looked up and kept per context: a second context
    on the same device (as a caller's cuCtxCreate makes) gets its own area, and
    the primary context keeps its first one.  Only the address lookup runs here
    (pyc_reduce_static_scratch); no kernel is launched in the second context."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    torch.zeros(1, device="cuda")  # the primary context is current
    CU_POINTER_ATTRIBUTE_CONTEXT = 1

    def owner(addr):
        c = ctypes.c_void_p()
        r = cu.cuPointerGetAttribute(ctypes.byref(c), CU_POINTER_ATTRIBUTE_CONTEXT,
                                     ctypes.c_uint64(addr))
        return c.value if r == 0 else None

    cur = ctypes.c_void_p()
    assert cu.cuCtxGetCurrent(ctypes.byref(cur)) == 0 and cur.value
    primary = cur.value
    a1, nbytes = pyc.pyc_reduce_static_scratch()
    assert a1 and nbytes == 4096 * 16 + 256
    assert owner(a1) in (primary, None)
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    ctx2 = ctypes.c_void_p()
    assert cu.cuCtxCreate_v2(ctypes.byref(ctx2), 0, dev) == 0  # made current on this thread
    try:
        a2, _ = pyc.pyc_reduce_static_scratch()
        assert a2 and a2 != a1  # one address space: the two areas cannot coincide
        assert owner(a2) in (ctx2.value, None)
        assert owner(a1) != owner(a2) or owner(a1) is None
        assert pyc.pyc_reduce_static_scratch()[0] == a2
    finally:
        popped = ctypes.c_void_p()
        assert cu.cuCtxPopCurrent_v2(ctypes.byref(popped)) == 0 and popped.value == ctx2.value
        assert cu.cuCtxDestroy_v2(ctx2) == 0
    assert cu.cuCtxGetCurrent(ctypes.byref(cur)) == 0 and cur.value == primary
    assert pyc.pyc_reduce_static_scratch()[0] == a1
