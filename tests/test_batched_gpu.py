"""Segmented (batched) map-reduce parity on the GPU: one persistent launch over a
segment table, replayed as a CUDA graph, against the oracle per segment."""
import numpy as np
import pytest
import torch

import oracle
from bounds import plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu


def _s():
    return torch.cuda.current_stream().cuda_stream


def _offsets(lens):
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


def _batched(name, off, arrays, out_dtype=torch.float32, out_cols=1, **opts):
    h = stock.create(name, **opts)
    ds = [a if isinstance(a, torch.Tensor) else torch.from_numpy(a).cuda() for a in arrays]
    nseg = len(off) - 1
    out = torch.full((nseg, out_cols), -7, dtype=out_dtype, device="cuda")
    pyc.pyc_reduce_batched(h, nseg, off, [d.data_ptr() for d in ds], None, out.data_ptr(), _s())
    torch.cuda.synchronize()
    return out, h, ds


def test_mixed_lengths_including_empty():
    lens = np.array([0, 1, 2, 31, 32, 33, 0, 2048, 2049, 5000, 70001, 0, 3, (1 << 20) + 7, 1,
                     300000, 4095, 4097], np.int64)
    off = _offsets(lens)
    x = inputs.uniform_f32(11, 0, int(off[-1]), -1.0, 1.0)
    y = inputs.uniform_f32(11, 1, int(off[-1]), -1.0, 1.0)
    out, _, _ = _batched("dot_f32", off, [x, y])
    ref, ab = oracle.dot_segments_f32(off, x, y)
    got = out[:, 0].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= plain_sum_bound(ab))
    assert np.all(got[lens == 0] == 0.0)


def test_int_segments_exact_and_sum_of_segments():
    lens = inputs.segment_lengths(nseg=3000, seed=12, max_log2=16)
    off = _offsets(lens)
    xi = inputs.int_uniform_i32(12, 0, int(off[-1]))
    yi = inputs.int_uniform_i32(12, 1, int(off[-1]))
    out, _, _ = _batched("dot_i32_i64", off, [xi, yi], out_dtype=torch.int64)
    got = out[:, 0].cpu().numpy()
    want = np.array([oracle.dot_i32_i64(xi[a:b], yi[a:b]) for a, b in zip(off[:-1], off[1:])])
    assert np.array_equal(got, want)
    s_out, _, _ = _batched("sum_i32_i64", off, [xi], out_dtype=torch.int64)
    assert int(s_out.sum().item()) == oracle.sum_i32_i64(xi)


def test_segments_beyond_2e31_elements():
    """2^31 + 100003 int32 elements in segments whose offsets, lengths and
    chunks pass 2^31 (one segment of ~2^31 elements, an empty one at 2^31 - 3,
    one of a single element after 2^31), summed into int64 exactly.  The input
    is 1 everywhere except two windows of seeded values in [-2^30, 2^30), so a
    segment's sum is P(b) - P(a), P(i) the ones before i plus the windows'
    elements before i (each window summed by the oracle)."""
    n = (1 << 31) + 100003
    wins = [((1 << 31) - 70000, (1 << 31) + 70001), (n - 3000, n)]
    x = torch.ones(n, dtype=torch.int32, device="cuda")
    vals = []
    for k, (a, b) in enumerate(wins):
        v = inputs.int_uniform_i32(38, k, b - a, -(1 << 30), 1 << 30)
        x[a:b] = torch.from_numpy(v).cuda()
        vals.append(v)

    def prefix(i):
        s = i
        for (a, b), v in zip(wins, vals):
            m = min(max(i - a, 0), b - a)
            s += oracle.sum_i32_i64(v[:m]) - m
        return s

    off = np.array([0, 100, (1 << 31) - 3, (1 << 31) - 3, (1 << 31) + 40000, (1 << 31) + 40001,
                    n - 1500, n], np.int64)
    out, _, _ = _batched("sum_i32_i64", off, [x], out_dtype=torch.int64)
    got = out[:, 0].cpu().numpy()
    want = [prefix(int(b)) - prefix(int(a)) for a, b in zip(off[:-1], off[1:])]
    assert [int(g) for g in got] == want
    del x
    torch.cuda.empty_cache()


def test_argmin_segments_exact():
    lens = inputs.segment_lengths(nseg=500, seed=13, max_log2=18)
    off = _offsets(lens)
    x = np.random.default_rng(13).integers(-50, 50, int(off[-1])).astype(np.float32)
    out, _, _ = _batched("argmin_f32", off, [x], out_dtype=torch.int64, out_cols=2)
    v, idx = pyc.argf32_from_tensor(out)
    v, idx = v.cpu().numpy(), idx.cpu().numpy()
    for s in range(len(lens)):
        a, b = off[s], off[s + 1]
        assert (float(v[s]), int(idx[s])) == oracle.argmin_f32(x[a:b]), s


def test_unaligned_base_pointers_and_variants():
    lens = inputs.segment_lengths(nseg=400, seed=14, max_log2=17)
    off = _offsets(lens)
    total = int(off[-1])
    x = inputs.uniform_f32(14, 0, total + 8, -1.0, 1.0)
    y = inputs.uniform_f32(14, 1, total + 8, -1.0, 1.0)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for shift in (1, 3):
        for opts in ({}, {"vec_bytes": 32, "items_per_thread": 2, "block": 128}):
            h = stock.create("dot_f32", **opts)
            out = torch.zeros(len(lens), device="cuda")
            pyc.pyc_reduce_batched(h, len(lens), off, [dx.data_ptr() + 4 * shift,
                                                       dy.data_ptr() + 4 * shift],
                                   None, out.data_ptr(), _s())
            torch.cuda.synchronize()
            ref, ab = oracle.dot_segments_f32(off, x[shift:shift + total], y[shift:shift + total])
            assert np.all(np.abs(out.cpu().numpy() - ref) <= plain_sum_bound(ab))


@pytest.mark.parametrize("tuned", [False, True])
@pytest.mark.parametrize("bf16", [False, True])
def test_config_20000_segments(bf16, tuned):
    """20,000 segments, lengths log-uniform in [1, 2^20]; graph replay gives the
    same bits; every segment within the plain-sum bound of the oracle; integer-free
    cross-check against one launch per segment.  `tuned`: after the batched
    autotuner has run on the table, as the benchmark does, so that the
    configuration it times (on GB300 the register-lean build) is the one checked."""
    lens = inputs.segment_lengths()
    off = _offsets(lens)
    total = int(off[-1])
    x = inputs.uniform_f32(2, 0, total, -1.0, 1.0)
    y = inputs.uniform_f32(2, 1, total, -1.0, 1.0)
    if bf16:
        x, y = inputs.to_bf16_values(x), inputs.to_bf16_values(y)
        dx = torch.from_numpy(x).to(torch.bfloat16).cuda()
        dy = torch.from_numpy(y).to(torch.bfloat16).cuda()
    else:
        dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    name = "dot_bf16" if bf16 else "dot_f32"
    if tuned:
        h = stock.create(name)
        o = torch.zeros(len(lens), device="cuda")
        pyc.pyc_reduce_batched_autotune(h, len(lens), off, [dx.data_ptr(), dy.data_ptr()], None,
                                        o.data_ptr(), _s())
        print("tuned batched configuration:", pyc.batched_config_name(h))
    out, h, _ = _batched(name, off, [dx, dy])
    first = out.clone()
    pyc.pyc_reduce_batched(h, len(lens), off, [dx.data_ptr(), dy.data_ptr()], None,
                           out.data_ptr(), _s())  # graph replay
    torch.cuda.synchronize()
    assert torch.equal(first, out)
    ref, ab = oracle.dot_segments_f32(off, x, y)
    got = out[:, 0].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= plain_sum_bound(ab))
    # one launch per segment (the plain path) agrees within the same bound
    per = torch.zeros(len(lens), device="cuda")
    es = dx.element_size()
    for k in range(0, len(lens), 97):
        pyc.pyc_reduce_launch(h, int(lens[k]), [dx.data_ptr() + int(off[k]) * es,
                                               dy.data_ptr() + int(off[k]) * es],
                              None, per.data_ptr() + 4 * k, _s())
    torch.cuda.synchronize()
    sel = np.arange(0, len(lens), 97)
    p = per.cpu().numpy()[sel].astype(np.float64)
    assert np.all(np.abs(p - ref[sel]) <= plain_sum_bound(ab[sel]))
    del dx, dy
    torch.cuda.empty_cache()


def test_capture_into_caller_graph():
    lens = np.array([5, 4000, 100000, 0, 17], np.int64)
    off = _offsets(lens)
    x = inputs.uniform_f32(15, 0, int(off[-1]), -1.0, 1.0)
    y = inputs.uniform_f32(15, 1, int(off[-1]), -1.0, 1.0)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    h = stock.create("dot_f32")
    out = torch.zeros(len(lens), device="cuda")
    # first call builds the plan outside capture
    pyc.pyc_reduce_batched(h, len(lens), off, [dx.data_ptr(), dy.data_ptr()], None,
                           out.data_ptr(), _s())
    torch.cuda.synchronize()
    want = out.clone()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pyc.pyc_reduce_batched(h, len(lens), off, [dx.data_ptr(), dy.data_ptr()], None,
                                   out.data_ptr(), s.cuda_stream)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, want)


def test_batched_autotune_keeps_results_within_bound():
    lens = inputs.segment_lengths(nseg=2000, seed=16, max_log2=18)
    off = _offsets(lens)
    x = inputs.uniform_f32(16, 0, int(off[-1]), -1.0, 1.0)
    y = inputs.uniform_f32(16, 1, int(off[-1]), -1.0, 1.0)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y")
    try:
        out = torch.zeros(len(lens), device="cuda")
        ptrs = [dx.data_ptr(), dy.data_ptr()]
        pyc.pyc_reduce_batched_autotune(h, len(lens), off, ptrs, None, out.data_ptr(), _s())
        out.zero_()
        pyc.pyc_reduce_batched(h, len(lens), off, ptrs, None, out.data_ptr(), _s())
        torch.cuda.synchronize()
        ref, ab = oracle.dot_segments_f32(off, x, y)
        assert np.all(np.abs(out.cpu().numpy() - ref) <= plain_sum_bound(ab))
    finally:
        pyc.pyc_reduce_destroy(h)
