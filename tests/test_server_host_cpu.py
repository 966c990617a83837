"""The serving loop without a GPU: pyc_server_create_host runs the same
scheduler (admission against the budget in arrival order, grouping by handle,
batch slots, in-flight limits, deadlines, queue limits, server-allocated
outputs, release, replay) with the batches executed on the host by the oracle.
These tests check the loop's own logic; the GPU tests check its kernels."""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1304_5553_gb300 import inputs, pyc, stock

A, B = 2.5, -0.75
POOL = 1 << 16


def _view(ptr, n, ct=ctypes.c_float):
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ct)), shape=(n,))


class Executor:
    """Runs each request with the oracle; optionally slow, blocked or failing."""

    def __init__(self, delay=0.0, fail_n=None):
        self.dot = stock.create("dot_f32").value
        self.lin = stock.create("lin_comb_f32").value
        self.delay, self.fail_n = delay, fail_n
        self.gate = threading.Event()
        self.gate.set()
        self.calls = 0

    def __call__(self, req, value):
        self.gate.wait()
        self.calls += 1
        if self.delay:
            time.sleep(self.delay)
        if self.fail_n is not None and req.n == self.fail_n:
            return pyc.PYC_E_INTERNAL
        x, y = _view(req.ptrs[0], req.n), _view(req.ptrs[1], req.n)
        if req.handle == self.dot:
            ctypes.cast(value, ctypes.POINTER(ctypes.c_float))[0] = oracle.dot_f32(x, y)[0]
        elif req.handle == self.lin:
            _view(req.ptrs[2], req.n)[:] = oracle.map_lin_comb_f32ops(A, x, B, y)
        else:
            return pyc.PYC_E_ARG
        return pyc.PYC_OK


@pytest.fixture(scope="module")
def pool():
    return (inputs.uniform_f32(60, 0, POOL, -1.0, 1.0), inputs.uniform_f32(60, 1, POOL, -1.0, 1.0))


def _until(cond, timeout=5.0):
    t = time.time() + timeout
    while not cond():
        assert time.time() < t, "timed out waiting for the server"
        time.sleep(0.0005)


def _req(pool, kind, n, off, deadline_us=0):
    x, y = pool
    ptrs = [x.ctypes.data + 4 * off, y.ctypes.data + 4 * off]
    if kind == pyc.PYC_REQ_MAP:
        h = stock.create("lin_comb_f32")
        return pyc.make_request(kind, h, n, ptrs + [0], pyc.pack_scalars(h, [A, B]), deadline_us)
    return pyc.make_request(kind, stock.create("dot_f32"), n, ptrs, None, deadline_us)


def _check(pool, kind, n, off, res):
    x, y = pool
    assert res.status == pyc.PYC_OK
    if kind == pyc.PYC_REQ_MAP:
        want = oracle.map_lin_comb_f32ops(A, x[off:off + n], B, y[off:off + n])
        assert np.array_equal(_view(res.d_out, n), want)
        # the output starts at its first input's address modulo 256
        assert res.d_out % 256 == (x.ctypes.data + 4 * off) % 256
    else:
        got = ctypes.c_float.from_buffer_copy(bytes(res.value[:4])).value
        assert got == np.float32(oracle.dot_f32(x[off:off + n], y[off:off + n])[0])


def test_every_result_reaches_its_request(pool):
    ex = Executor()
    srv = pyc.pyc_server_create_host(ex, 1 << 26, arena_bytes=1 << 24, max_batch=16)
    rng = np.random.default_rng(61)
    try:
        plan, live = [], []
        for k in range(300):
            kind = pyc.PYC_REQ_MAP if rng.random() < 0.4 else pyc.PYC_REQ_REDUCE
            n = int(rng.integers(1, 3000))
            off = int(rng.integers(0, POOL - n))
            r = _req(pool, kind, n, off)
            plan.append((kind, n, off, r, pyc.pyc_server_submit(srv, r)))
        outs = []
        for kind, n, off, r, rid in plan:
            res = pyc.pyc_server_poll(srv, rid, 10_000_000)
            _check(pool, kind, n, off, res)
            if kind == pyc.PYC_REQ_MAP:
                outs.append((res.d_out, res.d_out + 4 * n))
            assert 1 <= res.batch_size <= 16
            assert res.t_submit_ns <= res.t_admit_ns <= res.t_launch_ns <= res.t_done_ns
        # outputs of unreleased requests never overlap
        outs.sort()
        assert all(a[1] <= b[0] for a, b in zip(outs, outs[1:]))
        for *_, rid in plan:
            pyc.pyc_server_release(srv, rid)
        st = pyc.pyc_server_get_stats(srv)
        assert st["completed"] == 300 and st["failed"] == 0
        assert st["admitted_bytes"] == 0 and st["arena_in_use"] == 0
        assert st["batches"] < 300  # requests were grouped
    finally:
        pyc.pyc_server_destroy(srv)


def test_budget_and_continuous_batching(pool):
    """A slow executor and a budget of a few requests: admission never exceeds the
    budget, requests that arrive while a batch runs are grouped into the next
    ones, and releasing finished requests lets the queue drain."""
    ex = Executor(delay=0.002)
    n = 4096
    per = n * 8 + 4
    srv = pyc.pyc_server_create_host(ex, 6 * per, num_streams=1, max_batch=64, max_inflight=2)
    try:
        ids = [pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 16 * k)[0])
               for k in range(40)]
        peak, done, sizes = 0, set(), []
        while len(done) < len(ids):
            st = pyc.pyc_server_get_stats(srv)
            peak = max(peak, st["admitted_bytes"])
            for k, rid in enumerate(ids):
                if k in done:
                    continue
                res = pyc.pyc_server_poll(srv, rid, 0)
                if res is not None:
                    _check(pool, pyc.PYC_REQ_REDUCE, n, 16 * k, res)
                    sizes.append(res.batch_size)
                    pyc.pyc_server_release(srv, rid)
                    done.add(k)
            time.sleep(0.0005)
        st = pyc.pyc_server_get_stats(srv)
        assert peak <= 6 * per and st["peak_admitted_bytes"] <= 6 * per
        assert max(sizes) > 1                      # continuous batching
        assert st["batches"] < 40
    finally:
        pyc.pyc_server_destroy(srv)


def test_deadline_queue_limit_and_failed_requests(pool):
    ex = Executor(fail_n=777)
    n = 1000
    per = n * 8 + 4
    srv = pyc.pyc_server_create_host(ex, 2 * per, num_streams=1, max_queue=2)
    try:
        ex.gate.clear()                            # the executor is held
        first = [pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, k)[0])
                 for k in range(2)]                # fill the budget
        _until(lambda: pyc.pyc_server_get_stats(srv)["admitted_bytes"] == 2 * per)
        late = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 5, 3000)[0])
        waiting = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, 777, 9)[0])
        res = pyc.pyc_server_poll(srv, late, 2_000_000)
        assert res is not None and res.status == pyc.PYC_E_TIMEOUT  # not admitted in time
        _until(lambda: pyc.pyc_server_get_stats(srv)["queued"] == 1)
        pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 6)[0])  # queue: 2
        with pytest.raises(pyc.PycError) as e:     # a queue of 2 is full
            pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 8)[0])
        assert e.value.status == pyc.PYC_E_BUSY
        ex.gate.set()
        for rid in first:
            _check(pool, pyc.PYC_REQ_REDUCE, n, first.index(rid),
                   pyc.pyc_server_poll(srv, rid, 5_000_000))
            pyc.pyc_server_release(srv, rid)
        res = pyc.pyc_server_poll(srv, waiting, 5_000_000)
        assert res is not None and res.status == pyc.PYC_E_INTERNAL  # its own failure only
        pyc.pyc_server_release(srv, waiting)
        pyc.pyc_server_release(srv, late)
    finally:
        ex.gate.set()  # destroy waits for launched batches: never leave one held
        pyc.pyc_server_destroy(srv)


def test_a_client_thread_that_dies_leaves_the_server_usable(pool):
    """A client thread submits and dies without polling or releasing: its
    finished requests keep their budget until released (by anyone holding the
    ids) or until destroy; other clients are served meanwhile."""
    ex = Executor()
    n = 1000
    per = n * 8 + 4
    srv = pyc.pyc_server_create_host(ex, 8 * per)
    leaked = []

    def client():
        for k in range(4):
            leaked.append(pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, k)[0]))
        raise RuntimeError("client dies")

    def thread_main():
        try:
            client()
        except RuntimeError:
            pass  # the thread ends here, its requests neither polled nor released

    th = threading.Thread(target=thread_main)
    th.start()
    th.join()
    try:
        assert len(leaked) == 4
        mine = [pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 10 + k)[0])
                for k in range(4)]
        for k, rid in enumerate(mine):
            _check(pool, pyc.PYC_REQ_REDUCE, n, 10 + k, pyc.pyc_server_poll(srv, rid, 5_000_000))
            pyc.pyc_server_release(srv, rid)
        for rid in leaked:                          # finished, still holding the budget
            assert pyc.pyc_server_poll(srv, rid, 5_000_000).status == pyc.PYC_OK
        assert pyc.pyc_server_get_stats(srv)["admitted_bytes"] == 4 * per
        # the budget held by the dead client leaves room for four more at a time
        more = [pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 20 + k)[0])
                for k in range(5)]
        _until(lambda: pyc.pyc_server_get_stats(srv)["queued"] >= 1)
        pyc.pyc_server_release(srv, leaked[0])      # any holder of an id may release it
        for rid in more:
            assert pyc.pyc_server_poll(srv, rid, 5_000_000).status == pyc.PYC_OK
    finally:
        pyc.pyc_server_destroy(srv)                 # frees the rest, returns promptly


def test_replay_through_the_host_executed_loop(pool):
    ex = Executor()
    srv = pyc.pyc_server_create_host(ex, 1 << 26, arena_bytes=1 << 24)
    rng = np.random.default_rng(62)
    try:
        table = pyc.RequestTable(200)
        plan = []
        for k in range(200):
            kind = pyc.PYC_REQ_MAP if k % 3 == 0 else pyc.PYC_REQ_REDUCE
            n = int(rng.integers(1, 2000))
            off = int(rng.integers(0, POOL - n))
            x, y = pool
            ptrs = [x.ctypes.data + 4 * off, y.ctypes.data + 4 * off]
            if kind == pyc.PYC_REQ_MAP:
                h = stock.create("lin_comb_f32")
                table.set(k, kind, h, n, ptrs + [0], bytes(pyc.pack_scalars(h, [A, B])))
            else:
                table.set(k, kind, stock.create("dot_f32"), n, ptrs)
            plan.append((kind, n, off))
        arrivals = np.cumsum(rng.exponential(20_000, 200)).astype(np.int64)
        res = pyc.pyc_server_replay(srv, table, arrivals, pyc.PYC_REPLAY_SERVER)
        for (kind, n, off), r in zip(plan, res):
            if kind == pyc.PYC_REQ_REDUCE:
                _check(pool, kind, n, off, r)
            else:
                assert r.status == pyc.PYC_OK  # outputs were released by the replay
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_server_replay(srv, table, None, pyc.PYC_REPLAY_DIRECT)
        assert e.value.status == pyc.PYC_E_ARG
    finally:
        pyc.pyc_server_destroy(srv)


def test_size_limits_and_empty_requests(pool):
    """n = 0 requests complete (a map-reduce gives its neutral element, a map
    writes nothing and gets no output); n above 2^34 and negative n are argument
    errors; a request larger than the whole budget is refused at submit with
    PYC_E_NOMEM while smaller ones go on being served."""
    ex = Executor()
    n = 1000
    per = n * 8 + 4
    srv = pyc.pyc_server_create_host(ex, 3 * per)
    try:
        z_dot = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, 0, 0)[0])
        z_map = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_MAP, 0, 0)[0])
        res = pyc.pyc_server_poll(srv, z_dot, 5_000_000)
        assert res.status == pyc.PYC_OK
        assert ctypes.c_float.from_buffer_copy(bytes(res.value[:4])).value == 0.0
        pyc.pyc_server_release(srv, z_dot)
        res = pyc.pyc_server_poll(srv, z_map, 5_000_000)
        assert res.status == pyc.PYC_OK
        pyc.pyc_server_release(srv, z_map)
        for bad_n, status in ((-1, pyc.PYC_E_ARG), ((1 << 34) + 1, pyc.PYC_E_ARG),
                              (4 * n, pyc.PYC_E_NOMEM)):
            x, y = pool
            r = pyc.make_request(pyc.PYC_REQ_REDUCE, stock.create("dot_f32"), bad_n,
                                 [x.ctypes.data, y.ctypes.data])
            with pytest.raises(pyc.PycError) as e:
                pyc.pyc_server_submit(srv, r)
            assert e.value.status == status, bad_n
        ok = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, n, 3)[0])
        _check(pool, pyc.PYC_REQ_REDUCE, n, 3, pyc.pyc_server_poll(srv, ok, 5_000_000))
        pyc.pyc_server_release(srv, ok)
        assert pyc.pyc_server_get_stats(srv)["admitted_bytes"] == 0
    finally:
        pyc.pyc_server_destroy(srv)


def test_an_executor_that_raises_fails_its_request(pool):
    def exec_fn(req, value):
        if req.n == 13:
            raise ValueError("executor fault")
        ctypes.cast(value, ctypes.POINTER(ctypes.c_float))[0] = 1.0
        return pyc.PYC_OK

    srv = pyc.pyc_server_create_host(exec_fn, 1 << 24)
    try:
        bad = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, 13, 0)[0])
        good = pyc.pyc_server_submit(srv, _req(pool, pyc.PYC_REQ_REDUCE, 14, 0)[0])
        assert pyc.pyc_server_poll(srv, bad, 5_000_000).status == pyc.PYC_E_INTERNAL
        assert pyc.pyc_server_poll(srv, good, 5_000_000).status == pyc.PYC_OK
    finally:
        pyc.pyc_server_destroy(srv)
