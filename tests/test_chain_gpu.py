"""Chains of dependent launches on one stream: maps and map-reduces are
launched as programmatic dependents (each may be scheduled while the previous
kernel drains and waits for it before touching memory), so every launch must
still see its predecessor's results.  A chain in which each step consumes the
previous step's output is run directly, around kernels of another library, and
captured in a CUDA graph and replayed; every result is checked exactly against
the same chain on the host."""
import numpy as np
import pytest
import torch

from paper_1304_5553_gb300 import inputs, pyc

pytestmark = pytest.mark.gpu

STEPS = 30


def _handles():
    # values stay below 2^21 in magnitude: no signed overflow anywhere
    a = pyc.pyc_map_create("int *x, int *y", "y[i] = (x[i] * 3 + 1) & 0xFFFFF")
    b = pyc.pyc_map_create("int *x, int *y", "x[i] = y[i] - (y[i] >> 3)")
    r = pyc.pyc_reduce_create(pyc.PYC_I64, "0", "a+b", "(long long)y[i]", "int *y")
    return a, b, r


def _host_chain(x0, torch_add):
    x = x0.astype(np.int32).copy()
    sums = []
    with np.errstate(over="ignore"):
        for k in range(STEPS):
            y = (x * np.int32(3) + np.int32(1)) & np.int32(0xFFFFF)
            sums.append(int(y.astype(np.int64).sum()))
            x = y - (y >> 3)
            if torch_add:
                x = x + np.int32(k)
    return np.array(sums, np.int64), x


def _device_chain(hs, dx, dy, out, s, torch_add):
    a, b, r = hs
    n = dx.numel()
    for k in range(STEPS):
        pyc.pyc_map_launch(a, n, [dx.data_ptr(), dy.data_ptr()], None, s)
        pyc.pyc_reduce_launch(r, n, [dy.data_ptr()], None, out[k:].data_ptr(), s)
        pyc.pyc_map_launch(b, n, [dx.data_ptr(), dy.data_ptr()], None, s)
        if torch_add:
            dx.add_(k)  # a kernel of another library between two of ours


@pytest.mark.parametrize("n", [1000, (1 << 20) + 3])
@pytest.mark.parametrize("torch_add", [False, True])
def test_dependent_chain_direct(n, torch_add):
    x0 = inputs.int_uniform_i32(80, 0, n)
    want_sums, want_x = _host_chain(x0, torch_add)
    hs = _handles()
    try:
        dx = torch.from_numpy(x0).cuda()
        dy = torch.zeros(n, dtype=torch.int32, device="cuda")
        out = torch.zeros(STEPS, dtype=torch.int64, device="cuda")
        _device_chain(hs, dx, dy, out, torch.cuda.current_stream().cuda_stream, torch_add)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want_sums)
        assert np.array_equal(dx.cpu().numpy(), want_x)
    finally:
        pyc.pyc_map_destroy(hs[0])
        pyc.pyc_map_destroy(hs[1])
        pyc.pyc_reduce_destroy(hs[2])


@pytest.mark.parametrize("n", [1000, (1 << 20) + 3])
def test_dependent_chain_in_a_graph(n):
    x0 = inputs.int_uniform_i32(81, 0, n)
    want_sums, want_x = _host_chain(x0, False)
    hs = _handles()
    try:
        dx = torch.from_numpy(x0).cuda()
        dy = torch.zeros(n, dtype=torch.int32, device="cuda")
        out = torch.zeros(STEPS, dtype=torch.int64, device="cuda")
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gs):  # first launches (set-up) outside the capture
            _device_chain(hs, dx, dy, out, gs.cuda_stream, False)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            _device_chain(hs, dx, dy, out, gs.cuda_stream, False)
        for _ in range(2):
            dx.copy_(torch.from_numpy(x0).cuda())
            out.zero_()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want_sums)
            assert np.array_equal(dx.cpu().numpy(), want_x)
        del g
    finally:
        pyc.pyc_map_destroy(hs[0])
        pyc.pyc_map_destroy(hs[1])
        pyc.pyc_reduce_destroy(hs[2])
