"""Prefix scans (Sec. 3.2.6) over the other storage types of the argument spec
(the C type strings of Sec. 3.1), on the GPU through the C ABI, element by
element against the storage-type oracle: bfloat16 and binary16 inputs widened
to binary32, binary64, 64-bit integers and one-byte arrays; a binary16 output
rounded once on store.  Sizes span several tiles with ragged tails, arrays start
at element offsets off the vector alignment, and three launch configurations
are checked.  Every case is exact: integer sums below 2^53 / 2^63, integer-valued
floats whose prefix sums need few bits, and maxima."""
import numpy as np
import pytest
import torch

from oracle import storage
from paper_1304_5553_gb300 import inputs, pyc

pytestmark = pytest.mark.gpu

SIZES = [1, 31, 1000, 65543, (1 << 20) + 77]
OFFSETS = [0, 3]
CONFIGS = [None, dict(vec_bytes=16, items_per_thread=1, block=128),
           dict(vec_bytes=32, items_per_thread=4, block=512)]
NMAX = max(SIZES) + max(OFFSETS)


def _s():
    return torch.cuda.current_stream().cuda_stream


def _run(h, x, out_dtype, n, off):
    """Scan n elements of x starting at element off into y[off:off + n]."""
    y = torch.zeros(x.numel(), dtype=out_dtype, device="cuda")
    pyc.pyc_scan_launch(h, n, [x.data_ptr() + off * x.element_size(),
                               y.data_ptr() + off * y.element_size()], None, _s())
    pyc.pyc_scan_sync(h, _s())
    return y[off:off + n].cpu()


def _cases():
    # integer-valued inputs drawn from the seeded generator
    k8 = inputs.int_uniform_i32(40, 0, NMAX, -8, 8)           # exact in bfloat16
    k20 = inputs.int_uniform_i32(40, 1, NMAX)                 # [-2^20, 2^20]
    k40 = (inputs.int_uniform_i32(40, 2, NMAX).astype(np.int64) << 20) + \
        inputs.int_uniform_i32(40, 3, NMAX, 0, (1 << 20) - 1)  # about +-2^40
    u8 = np.where(inputs.int_uniform_i32(40, 4, NMAX, 0, 1) > 0,
                  inputs.int_uniform_i32(40, 5, NMAX, 1, 255), 0).astype(np.uint8)
    # binary16 values in [1, 2) and (-2, -1] (no zeros: the maximum has no sign-of-zero ties)
    h = inputs.to_f16_values(inputs.uniform_f32(40, 6, NMAX, 1.0, 2.0))
    h = np.where(inputs.int_uniform_i32(40, 7, NMAX, 0, 1) > 0, h, -h).astype(np.float16)
    return [
        # name, dtype, neutral, op, input, output, spec, x (numpy), torch in / out dtypes, oracle
        ("bf16 -> f32 sum", pyc.PYC_F32, "0", "a+b", "x[i]", "y[i] = item",
         "__nv_bfloat16 *x, float *y", k8.astype(np.float32), torch.bfloat16, torch.float32,
         lambda v: storage.scan_sum_int(k8[v]).astype(np.float32)),
        ("f16 -> f16 max", pyc.PYC_F32, "-INFINITY", "a > b ? a : b", "x[i]", "y[i] = item",
         "__half *x, __half *y", h, torch.float16, torch.float16,
         lambda v: storage.round_f16(storage.scan_max(h[v], -np.inf))),
        ("f64 sum", pyc.PYC_F64, "0", "a+b", "x[i]", "y[i] = item", "double *x, double *y",
         k20.astype(np.float64) * 2.0 ** -10, torch.float64, torch.float64,
         lambda v: storage.scan_sum_int(k20[v]).astype(np.float64) * 2.0 ** -10),
        ("i64 sum", pyc.PYC_I64, "0", "a+b", "x[i]", "y[i] = item", "long long *x, long long *y",
         k40, torch.int64, torch.int64, lambda v: storage.scan_sum_int(k40[v])),
        ("u8 -> i64 exclusive count", pyc.PYC_I64, "0", "a+b", "(long long)(x[i] != 0)",
         "y[i] = prev_item", "unsigned char *x, long long *y", u8, torch.uint8, torch.int64,
         lambda v: storage.scan_count_nonzero(u8[v])),
    ]


@pytest.mark.parametrize("case", range(5))
def test_scan_storage_types_exact(case):
    name, dt, neu, op, inp, outs, spec, x, tin, tout, want_fn = _cases()[case]
    dx = torch.from_numpy(np.ascontiguousarray(x)).to(tin).cuda()  # exact conversions
    for cfg in CONFIGS:
        h = pyc.pyc_scan_create(dt, neu, op, inp, outs, spec, cfg)
        try:
            for off in OFFSETS:
                for n in SIZES:
                    got = _run(h, dx, tout, n, off).numpy()
                    want = np.asarray(want_fn(slice(off, off + n)))
                    assert got.dtype == want.dtype, (name, got.dtype, want.dtype)
                    # bit for bit: compare each element's bytes
                    bad = np.flatnonzero((got.view(np.uint8).reshape(n, -1) !=
                                          want.view(np.uint8).reshape(n, -1)).any(axis=1))
                    assert bad.size == 0, (name, cfg, off, n, bad[:5], got[bad[:5]], want[bad[:5]])
        finally:
            pyc.pyc_scan_destroy(h)
