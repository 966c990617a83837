"""Segmented (batched) map-reduce over the other storage types of the argument
spec, on the GPU through the C ABI, per segment against the storage oracle:
binary64 and 64-bit integer sums (exact), a binary16 dot into binary32 (within
the plain-sum bound of the exact dot), the compensated binary32 sum (within its
bound), and binary32 maxima and int64 minima (exact).  The table mixes empty
segments, one-warp tasks (up to 2048 elements) and multi-chunk segments, and
two launch configurations are checked."""
import numpy as np
import pytest
import torch

import oracle
from bounds import compensated_sum_bound, plain_sum_bound
from oracle import storage
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu

LENS = np.array([0, 1, 2, 31, 2047, 2048, 2049, 5000, 70001, 0, 3, 300000, 4097, (1 << 20) + 7],
                np.int64)
OFF = np.concatenate([[0], np.cumsum(LENS)]).astype(np.int64)
TOTAL = int(OFF[-1])
CONFIGS = [None, dict(vec_bytes=32, items_per_thread=2, block=128)]


def _s():
    return torch.cuda.current_stream().cuda_stream


def _run(h, arrays, out_dtype, cols=1):
    out = torch.full((len(LENS), cols), -7, dtype=out_dtype, device="cuda")
    pyc.pyc_reduce_batched(h, len(LENS), OFF, [a.data_ptr() for a in arrays], None,
                           out.data_ptr(), _s())
    torch.cuda.synchronize()
    return out[:, 0].cpu().numpy()


def _segments(a):
    return [a[OFF[s]:OFF[s + 1]] for s in range(len(LENS))]


def _create(spec, opts):
    dt, neu, red, mp, args, extra = spec
    o = dict(extra, **(opts or {}))
    return pyc.pyc_reduce_create(dt, neu, red, mp, args, o or None)


@pytest.mark.parametrize("cfg", range(len(CONFIGS)))
def test_exact_sums_and_extrema(cfg):
    opts = CONFIGS[cfg]
    k20 = inputs.int_uniform_i32(50, 0, TOTAL)
    k40 = (inputs.int_uniform_i32(50, 1, TOTAL).astype(np.int64) << 20) + inputs.int_uniform_i32(
        50, 2, TOTAL, 0, (1 << 20) - 1)
    x = inputs.uniform_f32(50, 3, TOTAL, -2.0, 2.0)
    cases = [
        # binary64 sum of integer multiples of 2^-10: every partial sum is exact
        ((pyc.PYC_F64, "0", "a+b", "x[i]", "double *x", {}), k20.astype(np.float64) * 2.0 ** -10,
         torch.float64, lambda seg: storage.sum_int(seg * 2 ** 10) * 2.0 ** -10),
        ((pyc.PYC_I64, "0", "a+b", "x[i]", "long long *x", {}), k40, torch.int64,
         storage.sum_int),
        ((pyc.PYC_F32, "-INFINITY", "a > b ? a : b", "x[i]", "float *x", {}), x, torch.float32,
         lambda seg: storage.max_value(seg, -np.inf)),
        ((pyc.PYC_I64, "9223372036854775807LL", "a < b ? a : b", "x[i]", "long long *x", {}),
         k40, torch.int64, lambda seg: storage.min_value(seg, 2 ** 63 - 1)),
    ]
    for spec, data, tdt, want_fn in cases:
        h = _create(spec, opts)
        try:
            d = torch.from_numpy(data).cuda()
            got = _run(h, [d], tdt)
            for s, seg in enumerate(_segments(data)):
                assert got[s] == want_fn(seg), (spec[1:4], cfg, s, LENS[s], got[s])
        finally:
            pyc.pyc_reduce_destroy(h)


@pytest.mark.parametrize("cfg", range(len(CONFIGS)))
def test_half_dot_and_compensated_sum_within_bounds(cfg):
    opts = CONFIGS[cfg]
    xh = inputs.to_f16_values(inputs.uniform_f32(51, 0, TOTAL, -1.0, 1.0))
    yh = inputs.to_f16_values(inputs.uniform_f32(51, 1, TOTAL, -1.0, 1.0))
    h = _create((pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "__half *x, __half *y", {}), opts)
    try:
        got = _run(h, [torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()], torch.float32)
        for s in range(len(LENS)):
            a, b = OFF[s], OFF[s + 1]
            ex, ab = storage.dot_exact_f16(xh[a:b], yh[a:b])
            assert abs(float(got[s]) - ex) <= plain_sum_bound(ab), (cfg, s, LENS[s])
    finally:
        pyc.pyc_reduce_destroy(h)
    ln = inputs.lognormal_signed_f32(51, 2, TOTAL)
    hc = stock.create("sum_f32_comp", **(opts or {}))
    got = _run(hc, [torch.from_numpy(ln).cuda()], torch.float32)
    for s in range(len(LENS)):
        seg = ln[OFF[s]:OFF[s + 1]]
        ex = oracle.exact_sum_f32(seg)
        ab = oracle.sum_f32(seg)[1]
        assert abs(float(got[s]) - ex) <= compensated_sum_bound(ex, ab), (cfg, s, LENS[s])
