"""Device and page-locked memory pools on the GPU (Sec. 3.2.6)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import expr as ox
from paper_1304_5553_gb300 import gpuarray as ga
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu


def _copy(src, dst, stream):
    h = stock.create("copy_f32")
    pyc.pyc_map_launch(h, src.numel(), [src.data_ptr(), dst.data_ptr()], None, stream)


def test_device_blocks_same_stream_reuse():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE)
    try:
        s = torch.cuda.current_stream().cuda_stream
        n = (1 << 24) - 3   # 4n bytes and 4(n - 1000) bytes: both in the 2^26 class
        src = torch.from_numpy(inputs.uniform_f32(80, 0, n)).cuda()
        t = pyc.pool_empty(p, n, torch.float32)
        ptr = t.data_ptr()
        _copy(src, t, s)
        assert torch.equal(t, src)
        del t  # freed on the current stream: reusable there at once
        t2 = pyc.pool_empty(p, n - 1000, torch.float32)   # same size class
        assert t2.data_ptr() == ptr
        st = pyc.pyc_pool_get_stats(p)
        assert st["hits"] == 1 and st["misses"] == 1 and st["live_blocks"] == 1
        del t2
    finally:
        torch.cuda.synchronize()
        pyc.pyc_pool_destroy(p)


def test_cross_stream_reuse_waits_for_the_work():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE)
    try:
        n = 1 << 28   # 1 GiB: each copy takes ~0.3 ms
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        src = torch.empty(n, dtype=torch.float32, device="cuda").fill_(1.5)
        torch.cuda.synchronize()
        a = pyc.pyc_pool_alloc(p, 4 * n, s1.cuda_stream)
        for _ in range(3):  # ~1 ms of work on s1 that writes block a
            h = stock.create("copy_f32")
            pyc.pyc_map_launch(h, n, [src.data_ptr(), a], None, s1.cuda_stream)
        pyc.pyc_pool_free(p, a, s1.cuda_stream)
        b = pyc.pyc_pool_alloc(p, 4 * n, s2.cuda_stream)   # s1 still busy: a new block
        assert b != a
        pyc.pyc_pool_free(p, b, s2.cuda_stream)
        s1.synchronize()
        s2.synchronize()
        c = pyc.pyc_pool_alloc(p, 4 * n, s2.cuda_stream)   # both retained and done
        assert c in (a, b)
        st = pyc.pyc_pool_get_stats(p)
        assert st["misses"] == 2 and st["hits"] == 1
        pyc.pyc_pool_free(p, c, s2.cuda_stream)
        pyc.pyc_pool_trim(p)
        assert pyc.pyc_pool_get_stats(p)["system_bytes"] == 0
    finally:
        torch.cuda.synchronize()
        pyc.pyc_pool_destroy(p)


def test_expressions_from_a_pool():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE)
    ga.set_pool(p)
    try:
        n = 300007
        x, y = (inputs.uniform_f32(81, k, n) for k in range(2))
        X = ga.GArray(torch.from_numpy(x).cuda())
        Y = ga.GArray(torch.from_numpy(y).cuda())
        for _ in range(4):
            e = (X * Y + 2.5) * (X - Y)
            r, k = ga.evaluate_eager(e)
            assert k == 4
            want = ox.eval_f32(("*", ("+", ("*", x, y), np.float32(2.5)), ("-", x, y)))
            assert np.array_equal(r.tensor.cpu().numpy(), want)
            del r
        st = pyc.pyc_pool_get_stats(p)
        # the first round allocates; later rounds reuse the freed temporaries
        assert st["hits"] >= 9 and st["misses"] <= 4, st
    finally:
        ga.set_pool(None)
        torch.cuda.synchronize()
        pyc.pyc_pool_destroy(p)


def test_pinned_pool_round_trip():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_PINNED)
    try:
        n = 1 << 20
        q = pyc.pyc_pool_alloc(p, 4 * n)
        host = np.frombuffer((ctypes.c_char * (4 * n)).from_address(q), dtype=np.float32)
        host[:] = np.arange(n, dtype=np.float32)
        t = torch.frombuffer((ctypes.c_char * (4 * n)).from_address(q), dtype=torch.float32)
        d = t.to("cuda", non_blocking=True)
        torch.cuda.synchronize()
        assert torch.equal(d.cpu(), torch.arange(n, dtype=torch.float32))
        pyc.pyc_pool_free(p, q)
        assert pyc.pyc_pool_alloc(p, 4 * n - 64) == q
        pyc.pyc_pool_free(p, q)
    finally:
        torch.cuda.synchronize()
        pyc.pyc_pool_destroy(p)


def test_device_limit_releases_retained_blocks():
    cls = pyc.pyc_pool_block_size(1 << 26)
    p = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE, max_bytes=3 * cls)
    try:
        blocks = [pyc.pyc_pool_alloc(p, 1 << 26) for _ in range(3)]
        with pytest.raises(pyc.PycError):
            pyc.pyc_pool_alloc(p, 1 << 26)
        for q in blocks:
            pyc.pyc_pool_free(p, q)
        big = pyc.pyc_pool_alloc(p, 2 * cls)   # another class: retained blocks are released
        st = pyc.pyc_pool_get_stats(p)
        assert st["system_bytes"] <= 3 * cls and st["system_frees"] >= 2
        pyc.pyc_pool_free(p, big)
    finally:
        torch.cuda.synchronize()
        pyc.pyc_pool_destroy(p)
