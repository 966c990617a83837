"""Injected host-side failures that need no GPU (pyc_test_inject).

A failed run-time compilation must surface as PYC_E_COMPILE and leave nothing
behind (the next creation of the same spec compiles it); a failed system
allocation in a memory pool must first give the retained blocks back and retry
once, and when that fails too, report PYC_E_NOMEM with the pool's statistics
unchanged; a rejection injected at a serving loop's admission fails that
request alone (the loop runs here with host-executed batches).
"""
import os
import threading
import time

import pytest

from paper_1304_5553_gb300 import pyc


@pytest.fixture(autouse=True)
def _clear():
    yield
    for k in (pyc.PYC_INJECT_ALLOC, pyc.PYC_INJECT_COMPILE, pyc.PYC_INJECT_STALL_MS,
              pyc.PYC_INJECT_ADMIT):
        pyc.pyc_test_inject(k, 0)


def _unique_stmt():
    return "z[i] = x[i] * %d.25f" % (os.getpid() * 1000003 + time.time_ns() % 1000003)


def test_argument_errors():
    lib = pyc.load()
    assert lib.pyc_test_inject(4, 1) == pyc.PYC_E_ARG
    assert lib.pyc_test_inject(-1, 1) == pyc.PYC_E_ARG
    assert lib.pyc_test_inject(pyc.PYC_INJECT_ALLOC, -1) == pyc.PYC_E_ARG


def test_injected_compile_failure_then_clean_compile():
    stmt = _unique_stmt()
    before = pyc.pyc_cache_stats()["compiled"]
    pyc.pyc_test_inject(pyc.PYC_INJECT_COMPILE, 1)
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_map_create("float *x, float *z", stmt)
    assert e.value.status == pyc.PYC_E_COMPILE and "injected" in e.value.message
    assert pyc.pyc_cache_stats()["compiled"] == before  # nothing was compiled or cached
    h = pyc.pyc_map_create("float *x, float *z", stmt)  # the next attempt compiles
    assert pyc.pyc_cache_stats()["compiled"] == before + 1
    pyc.pyc_map_destroy(h)
    # a cache hit does not compile, so it neither fails nor consumes the injection
    pyc.pyc_test_inject(pyc.PYC_INJECT_COMPILE, 1)
    h = pyc.pyc_map_create("float *x, float *z", stmt)
    pyc.pyc_map_destroy(h)
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i] * %d.5f" % time.time_ns(), "float *x")
    assert e.value.status == pyc.PYC_E_COMPILE


def test_threads_waiting_on_a_failed_compile_see_its_error():
    stmt = _unique_stmt()
    pyc.pyc_test_inject(pyc.PYC_INJECT_COMPILE, 1)
    out = []

    def make():
        try:
            out.append(pyc.pyc_map_create("float *x, float *z", stmt))
        except pyc.PycError as e:
            out.append(e.status)

    ts = [threading.Thread(target=make) for _ in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    fails = [r for r in out if r == pyc.PYC_E_COMPILE]
    assert len(out) == 4 and len(fails) >= 1  # the injected failure reached its waiters
    for r in out:
        if r != pyc.PYC_E_COMPILE:
            pyc.pyc_map_destroy(r)
    h = pyc.pyc_map_create("float *x, float *z", stmt)  # afterwards it compiles
    pyc.pyc_map_destroy(h)


def test_pool_retries_after_returning_retained_blocks():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_HOST)
    try:
        kept = [pyc.pyc_pool_alloc(p, 1 << 20) for _ in range(3)]
        for q in kept:
            pyc.pyc_pool_free(p, q)
        st0 = pyc.pyc_pool_get_stats(p)
        assert st0["retained_blocks"] == 3
        pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 1)  # the first system allocation fails
        q = pyc.pyc_pool_alloc(p, 5 << 20)            # another class: needs the system
        st = pyc.pyc_pool_get_stats(p)
        assert st["retained_blocks"] == 0 and st["live_blocks"] == 1
        assert st["system_frees"] == st0["system_frees"] + 3
        assert st["system_allocs"] == st0["system_allocs"] + 1
        pyc.pyc_pool_free(p, q)
        # both the allocation and its retry fail: PYC_E_NOMEM, nothing changes
        st1 = pyc.pyc_pool_get_stats(p)
        pyc.pyc_test_inject(pyc.PYC_INJECT_ALLOC, 2)
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_pool_alloc(p, 9 << 20)
        assert e.value.status == pyc.PYC_E_NOMEM
        st2 = pyc.pyc_pool_get_stats(p)
        assert (st2["live_blocks"], st2["live_bytes"], st2["system_allocs"]) == \
            (st1["live_blocks"], st1["live_bytes"], st1["system_allocs"])
        assert st2["system_bytes"] == st2["live_bytes"] + st2["retained_bytes"]
        q = pyc.pyc_pool_alloc(p, 9 << 20)  # the next request succeeds
        assert pyc.pyc_pool_get_stats(p)["live_blocks"] == 1
        pyc.pyc_pool_free(p, q)
    finally:
        pyc.pyc_pool_destroy(p)


def test_injected_admission_rejection_fails_only_those_requests():
    """Two injected rejections at admission: the first two requests reaching
    admission fail with PYC_E_NOMEM, the others are admitted and served, and no
    budget is left counted for the rejected ones."""
    import ctypes

    import numpy as np

    from paper_1304_5553_gb300 import stock
    x = np.arange(4096, dtype=np.float32)
    h = stock.create("dot_f32")

    def exec_fn(req, value):
        a = np.ctypeslib.as_array(ctypes.cast(req.ptrs[0], ctypes.POINTER(ctypes.c_float)),
                                  shape=(req.n,))
        ctypes.cast(value, ctypes.POINTER(ctypes.c_float))[0] = float(np.dot(a, a))
        return pyc.PYC_OK

    srv = pyc.pyc_server_create_host(exec_fn, 1 << 24)
    try:
        pyc.pyc_test_inject(pyc.PYC_INJECT_ADMIT, 2)
        reqs = [pyc.make_request(pyc.PYC_REQ_REDUCE, h, 100 + k, [x.ctypes.data] * 2)
                for k in range(5)]
        ids = [pyc.pyc_server_submit(srv, r) for r in reqs]
        st = [pyc.pyc_server_poll(srv, i, 5_000_000).status for i in ids]
        assert st == [pyc.PYC_E_NOMEM] * 2 + [pyc.PYC_OK] * 3
        stats = pyc.pyc_server_get_stats(srv)
        assert stats["failed"] == 2 and stats["completed"] == 3
        for i in ids:
            pyc.pyc_server_release(srv, i)
        assert pyc.pyc_server_get_stats(srv)["admitted_bytes"] == 0
    finally:
        pyc.pyc_server_destroy(srv)
