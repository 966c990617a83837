"""Injected host-side failures on a GPU machine (pyc_test_inject).

Every failure here is made on the host -- an allocation call that reports
"out of memory", a scheduler that sleeps -- never on the GPU.  Each test checks
the documented status, that nothing leaks (pool and server statistics), and
that the next call succeeds.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clear():
    yield
    for k in (pyc.PYC_INJECT_ALLOC, pyc.PYC_INJECT_COMPILE, pyc.PYC_INJECT_STALL_MS,
              pyc.PYC_INJECT_ADMIT):
        pyc.pyc_test_inject(k, 0)


def test_reduce_workspace_allocation_failure():
    """The first launch on a new stream allocates the handle's workspace there."""
    n = 100003
    x = inputs.int_uniform_i32(60, 0, n)
    d = torch.from_numpy(x).cuda()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    h = stock.create("sum_i32_i64")
    s2 = torch.cuda.Stream()
    pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 1)
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_launch(h, n, [d.data_ptr()], None, out.data_ptr(), s2.cuda_stream)
    assert e.value.status == pyc.PYC_E_NOMEM
    pyc.pyc_reduce_launch(h, n, [d.data_ptr()], None, out.data_ptr(), s2.cuda_stream)
    s2.synchronize()
    assert int(out.item()) == oracle.sum_i32_i64(x)


def test_device_pool_retry_and_failure():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE)
    s = torch.cuda.current_stream().cuda_stream
    try:
        for q in [pyc.pyc_pool_alloc(p, 1 << 22, s) for _ in range(2)]:
            pyc.pyc_pool_free(p, q, s)
        st0 = pyc.pyc_pool_get_stats(p)
        pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 1)
        q = pyc.pyc_pool_alloc(p, 3 << 22, s)  # fails once, retained blocks go back, retry
        st = pyc.pyc_pool_get_stats(p)
        assert st["retained_blocks"] == 0 and st["system_frees"] == st0["system_frees"] + 2
        pyc.pyc_pool_free(p, q, s)
        st1 = pyc.pyc_pool_get_stats(p)
        pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 2)
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_pool_alloc(p, 5 << 22, s)
        assert e.value.status == pyc.PYC_E_NOMEM
        st2 = pyc.pyc_pool_get_stats(p)
        assert st2["live_blocks"] == st1["live_blocks"] == 0
        assert st2["system_allocs"] == st1["system_allocs"]
        assert st2["system_bytes"] == st2["retained_bytes"]
        q = pyc.pyc_pool_alloc(p, 5 << 22, s)
        pyc.pyc_pool_free(p, q, s)
    finally:
        pyc.pyc_pool_destroy(p)


def test_batched_plan_allocation_failure():
    lens = np.array([1, 5000, 70000, 0, 300], np.int64)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    x = inputs.uniform_f32(61, 0, int(off[-1]), -1.0, 1.0)
    y = inputs.uniform_f32(61, 1, int(off[-1]), -1.0, 1.0)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.zeros(len(lens), device="cuda")
    h = stock.create("dot_f32")
    args = (h, len(lens), off, [dx.data_ptr(), dy.data_ptr()], None, out.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 1)
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_batched(*args)
    assert e.value.status == pyc.PYC_E_NOMEM
    pyc.pyc_reduce_batched(*args)
    torch.cuda.synchronize()
    ref, ab = oracle.dot_segments_f32(off, x, y)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 8 * 2.0 ** -24 * ab)


def test_server_creation_allocation_failure():
    """The server's first device allocation fails: creation reports PYC_E_NOMEM
    (after freeing what it had made) and the next creation succeeds."""
    pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 1)
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_server_create(1 << 30, arena_bytes=1 << 24, max_inflight=2)
    assert e.value.status == pyc.PYC_E_NOMEM
    srv = pyc.pyc_server_create(1 << 30, arena_bytes=1 << 24, max_inflight=2)
    pyc.pyc_server_destroy(srv)


def _dot_request(n, off, dev, deadline_us=0):
    h = stock.create("dot_f32")
    return pyc.make_request(pyc.PYC_REQ_REDUCE, h, n,
                            [dev[0].data_ptr() + 4 * off, dev[1].data_ptr() + 4 * off],
                            None, deadline_us)


def test_stalled_scheduler_misses_deadlines_then_recovers():
    n = 1 << 16
    x = inputs.uniform_f32(62, 0, n + 64, -1.0, 1.0)
    y = inputs.uniform_f32(62, 1, n + 64, -1.0, 1.0)
    dev = (torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    srv = pyc.pyc_server_create(1 << 30, num_streams=1)
    try:
        warm = _dot_request(n, 0, dev)
        rid = pyc.pyc_server_submit(srv, warm)
        assert pyc.pyc_server_poll(srv, rid, 10_000_000).status == pyc.PYC_OK
        pyc.pyc_server_release(srv, rid)
        pyc.pyc_test_inject(pyc.PYC_INJECT_STALL_MS, 300)
        late = [_dot_request(n, k, dev, deadline_us=20_000) for k in range(3)]
        ids = [pyc.pyc_server_submit(srv, r) for r in late]
        for rid in ids:
            res = pyc.pyc_server_poll(srv, rid, 10_000_000)
            assert res is not None and res.status == pyc.PYC_E_TIMEOUT
            pyc.pyc_server_release(srv, rid)
        st = pyc.pyc_server_get_stats(srv)
        assert st["failed"] == 3 and st["admitted_bytes"] == 0 and st["queued"] == 0
        ok = _dot_request(n, 7, dev, deadline_us=5_000_000)
        rid = pyc.pyc_server_submit(srv, ok)
        res = pyc.pyc_server_poll(srv, rid, 10_000_000)
        assert res is not None and res.status == pyc.PYC_OK
        ref, ab = oracle.dot_f32(x[7:7 + n], y[7:7 + n])
        assert abs(np.frombuffer(bytes(res.value)[:4], np.float32)[0] - ref) <= \
            8 * 2.0 ** -24 * ab
        pyc.pyc_server_release(srv, rid)
    finally:
        pyc.pyc_server_destroy(srv)


def test_arena_running_dry_waits_for_a_release():
    """Map outputs the server allocates come from its arena: with room for two,
    a third request waits (it neither fails nor runs) until one is released."""
    n = 3 << 18                     # 3 MiB of binary32 output each
    x = torch.from_numpy(inputs.uniform_f32(63, 0, n, -1.0, 1.0)).cuda()
    y = torch.from_numpy(inputs.uniform_f32(63, 1, n, -1.0, 1.0)).cuda()
    h = stock.create("lin_comb_f32")
    sc = pyc.pack_scalars(h, [2.5, -0.75])
    srv = pyc.pyc_server_create(1 << 30, arena_bytes=7 << 20, num_streams=2)
    try:
        reqs = [pyc.make_request(pyc.PYC_REQ_MAP, h, n, [x.data_ptr(), y.data_ptr(), 0], sc)
                for _ in range(3)]
        ids = [pyc.pyc_server_submit(srv, r) for r in reqs]
        for rid in ids[:2]:
            assert pyc.pyc_server_poll(srv, rid, 10_000_000).status == pyc.PYC_OK
        assert pyc.pyc_server_poll(srv, ids[2], 200_000) is None  # waiting for arena room
        assert pyc.pyc_server_get_stats(srv)["queued"] == 1
        pyc.pyc_server_release(srv, ids[0])
        res = pyc.pyc_server_poll(srv, ids[2], 10_000_000)
        assert res is not None and res.status == pyc.PYC_OK
        want = oracle.map_lin_comb_f32ops(2.5, x.cpu().numpy(), -0.75, y.cpu().numpy())
        out = torch.empty(n, device="cuda")
        pyc.pyc_map_launch(stock.create("copy_f32"), n, [res.d_out, out.data_ptr()], None,
                           torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
        for rid in ids[1:]:
            pyc.pyc_server_release(srv, rid)
        st = pyc.pyc_server_get_stats(srv)
        assert st["arena_in_use"] == 0 and st["admitted_bytes"] == 0 and st["failed"] == 0
    finally:
        pyc.pyc_server_destroy(srv)


def test_cg_work_space_allocation_failure():
    """A solver's first use on a stream allocates its work space (and its dot
    products' workspaces): an injected failure there is PYC_E_NOMEM, x is left
    as it was, and the next solve on the same stream converges."""
    nx = 64
    rp, c, v = inputs.poisson2d(nx, nx, np.float64)
    n = nx * nx
    d = [torch.from_numpy(t).cuda() for t in (rp, c, v)]
    a = pyc.pyc_csr_create(n, n, c.size, *(t.data_ptr() for t in d), pyc.PYC_F64)
    try:
        b = torch.ones(n, dtype=torch.float64, device="cuda")
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        s2 = torch.cuda.Stream()
        pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 1)
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_cg_solve(a, b.data_ptr(), x.data_ptr(), 1e-10, 2000, s2.cuda_stream)
        assert e.value.status == pyc.PYC_E_NOMEM
        s2.synchronize()
        assert torch.count_nonzero(x).item() == 0
        info = pyc.pyc_cg_solve(a, b.data_ptr(), x.data_ptr(), 1e-10, 2000, s2.cuda_stream)
        s2.synchronize()
        assert info["converged"]
        # the true residual of the solution, in binary64 on the host
        xs = x.cpu().numpy()
        rows = np.repeat(np.arange(n), np.diff(rp))
        ax = np.zeros(n)
        np.add.at(ax, rows, v * xs[c])
        assert np.linalg.norm(1.0 - ax) <= 1e-9 * np.sqrt(n)
    finally:
        pyc.pyc_csr_destroy(a)
