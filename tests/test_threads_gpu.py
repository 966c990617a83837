"""Host threads sharing handles on the GPU.

Eight threads, each with a stream of its own, launch the same map, map-reduce,
scan and batched handles again and again (the C ABI releases the GIL, so the
calls overlap in the library: per-stream workspaces, kernel lookup, tuned
configurations), and all of them create one spec never seen before at the same
moment (one compilation, shared).  Every result is checked against the oracle.
"""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
from bounds import plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu

THREADS = 8
ROUNDS = 12


def test_threads_share_handles_and_a_first_compile():
    n = (1 << 20) + 3
    x = inputs.uniform_f32(90, 0, n, -1.0, 1.0)
    y = inputs.uniform_f32(90, 1, n, -1.0, 1.0)
    xi = inputs.int_uniform_i32(90, 2, n)
    dx, dy, dxi = (torch.from_numpy(a).cuda() for a in (x, y, xi))
    off = np.array([0, 1, 4097, 4097, 70000, n], np.int64)
    h_map, h_dot = stock.create("lin_comb_f32"), stock.create("dot_f32")
    h_scan, h_sum = stock.create("cumsum_excl_i32_i64"), stock.create("sum_i32_i64")
    sc = pyc.pack_scalars(h_map, [2.5, -0.75])
    k = time.time_ns() % 1000003  # a constant no earlier run compiled
    stmt = "z[i] = x[i] * 3.5f + %d.0f" % k
    before = pyc.pyc_cache_stats()["compiled"]
    outs, errors = {}, []
    start = threading.Barrier(THREADS)

    def work(t):
        try:
            s = torch.cuda.Stream()
            z = torch.empty(n, device="cuda")
            yi = torch.empty(n, dtype=torch.int64, device="cuda")
            w = torch.empty(n, device="cuda")
            dots = torch.zeros(ROUNDS, device="cuda")
            segs = torch.zeros(ROUNDS, len(off) - 1, dtype=torch.int64, device="cuda")
            start.wait()
            h_new = pyc.pyc_map_create("float *x, float *z", stmt)
            for r in range(ROUNDS):
                pyc.pyc_map_launch(h_map, n, [dx.data_ptr(), dy.data_ptr(), z.data_ptr()], sc,
                                   s.cuda_stream)
                pyc.pyc_reduce_launch(h_dot, n, [dx.data_ptr(), dy.data_ptr()], None,
                                      dots[r:].data_ptr(), s.cuda_stream)
                pyc.pyc_scan_launch(h_scan, n, [dxi.data_ptr(), yi.data_ptr()], None,
                                    s.cuda_stream)
                pyc.pyc_reduce_batched(h_sum, len(off) - 1, off, [dxi.data_ptr()], None,
                                       segs[r].data_ptr(), s.cuda_stream)
                pyc.pyc_map_launch(h_new, n, [dx.data_ptr(), w.data_ptr()], None, s.cuda_stream)
            pyc.pyc_scan_sync(h_scan, s.cuda_stream)
            s.synchronize()
            outs[t] = (z.cpu().numpy(), dots.cpu().numpy(), yi.cpu().numpy(), segs.cpu().numpy(),
                       w.cpu().numpy())
            pyc.pyc_map_destroy(h_new)
        except Exception as e:  # reported after the join
            errors.append((t, repr(e)))

    ts = [threading.Thread(target=work, args=(t,)) for t in range(THREADS)]
    for th in ts:
        th.start()
    for th in ts:
        th.join()
    assert not errors, errors
    assert pyc.pyc_cache_stats()["compiled"] == before + 1  # one compilation for all threads
    want_z = oracle.map_lin_comb_f32ops(2.5, x, -0.75, y)
    ref_dot, ab = oracle.dot_f32(x, y)
    want_scan = oracle.scan_sum_i32_i64(xi, exclusive=True)
    want_segs = [oracle.sum_i32_i64(xi[a:b]) for a, b in zip(off[:-1], off[1:])]
    want_w = x * np.float32(3.5) + np.float32(k)  # binary32: each operation rounds
    dot0 = None
    for t in range(THREADS):
        z, dots, yi, segs, w = outs[t]
        assert np.array_equal(z, want_z), t
        assert np.all(np.abs(dots.astype(np.float64) - ref_dot) <= plain_sum_bound(ab)), t
        # the same configuration on every stream: the same value every time
        dot0 = dots[0] if dot0 is None else dot0
        assert np.all(dots == dot0), t
        assert np.array_equal(yi, want_scan), t
        assert all(list(row) == want_segs for row in segs), t
        assert np.array_equal(w, want_w), t
