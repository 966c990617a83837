"""Bounds-checked builds (pyc_opts.debug_bounds) on the GPU.

compute-sanitizer is not available to these tests, so the library carries its
own checker: in a checked build every array access of the generated map,
map-reduce, batched, sharded and served kernels is tested against the array's
index range and access width, and the first violation is recorded (the access
is skipped).  Each test runs a workload in a checked build and in the plain
build with the same launch configuration: the checked build must record no
violation and give the same bits.  A last test narrows the checked ranges on
purpose (a host-side test hook; no access leaves its array) to show that the
checks fire and that the host reads and clears the record.
"""
import re

import numpy as np
import pytest
import torch

from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu

A, B = 2.5, -0.75
CFG = dict(vec_bytes=16, items_per_thread=2, block=128)  # fixed: both builds launch alike
SMALL = list(range(0, 300)) + list(range(300, 1101, 7)) + [1100]


def _s():
    return torch.cuda.current_stream().cuda_stream


def _pair(name, **cfg):
    return stock.create(name, **cfg), stock.create(name, debug_bounds=1, **cfg)


@pytest.mark.parametrize("bf16", [False, True])
def test_maps_small_sizes_all_offsets(bf16):
    name = "lin_comb_bf16" if bf16 else "lin_comb_f32"
    hp, hc = _pair(name, **CFG)
    assert "#define PYC_BOUNDS 1" in pyc.pyc_map_source(hc)
    total = sum(n + 64 for n in SMALL) * 16 + 64
    dt = torch.bfloat16 if bf16 else torch.float32
    x = torch.from_numpy(inputs.uniform_f32(5, 0, total, -2.0, 2.0)).to(dt).cuda()
    y = torch.from_numpy(inputs.uniform_f32(5, 1, total, -2.0, 2.0)).to(dt).cuda()
    zs = [torch.full((total,), -4096.0, dtype=dt, device="cuda") for _ in range(2)]
    es = x.element_size()
    pos = 0
    for o in range(16):
        for n in SMALL:
            b = pos + o
            for h, z in ((hp, zs[0]), (hc, zs[1])):
                pyc.pyc_map_launch(h, n, [x.data_ptr() + b * es, y.data_ptr() + b * es,
                                          z.data_ptr() + b * es], pyc.pack_scalars(h, [A, B]),
                                   _s())
            pos += n + 64
    pyc.pyc_map_check_bounds(hc)
    assert torch.equal(zs[0].view(torch.int16) if bf16 else zs[0].view(torch.int32),
                       zs[1].view(torch.int16) if bf16 else zs[1].view(torch.int32))


@pytest.mark.parametrize("name,step", [("dot_f32", 3), ("sum_i32_i64", 1), ("argmin_f32", 3),
                                       ("sum_f32_comp", 5), ("max_f32", 5)])
def test_reductions_small_sizes_all_offsets(name, step):
    hp, hc = _pair(name, **CFG)
    nmax = 1100 + 16
    if name == "sum_i32_i64":
        arrays = [inputs.int_uniform_i32(6, 0, nmax)]
    elif name == "dot_f32":
        arrays = [inputs.uniform_f32(6, s, nmax, -1.0, 1.0) for s in range(2)]
    else:  # few distinct values: ties for argmin
        arrays = [np.round(inputs.uniform_f32(6, 0, nmax, -4.0, 4.0)).astype(np.float32)]
    ds = [torch.from_numpy(a).cuda() for a in arrays]
    es = ds[0].element_size()
    cases = [(o, n) for o in range(16) for n in range(0, 1101, step)]
    outs = [torch.zeros(len(cases), 2, dtype=torch.int64, device="cuda") for _ in range(2)]
    for k, (o, n) in enumerate(cases):
        for h, out in ((hp, outs[0]), (hc, outs[1])):
            pyc.pyc_reduce_launch(h, n, [d.data_ptr() + o * es for d in ds], None,
                                  out[k].data_ptr(), _s())
    pyc.pyc_reduce_check_bounds(hc)
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("bf16", [False, True])
def test_segmented_20000_segments(bf16):
    lens = inputs.segment_lengths()
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(off[-1])
    dt = torch.bfloat16 if bf16 else torch.float32
    x = torch.from_numpy(inputs.uniform_f32(2, 0, total, -1.0, 1.0)).to(dt).cuda()
    y = torch.from_numpy(inputs.uniform_f32(2, 1, total, -1.0, 1.0)).to(dt).cuda()
    hp, hc = _pair("dot_bf16" if bf16 else "dot_f32", vec_bytes=32, items_per_thread=1,
                   block=128)
    outs = [torch.zeros(lens.size, device="cuda") for _ in range(2)]
    for h, out in zip((hp, hc), outs):
        pyc.pyc_reduce_batched(h, lens.size, off, [x.data_ptr(), y.data_ptr()], None,
                               out.data_ptr(), _s())
    pyc.pyc_reduce_check_bounds(hc)
    assert torch.equal(outs[0], outs[1])
    del x, y
    torch.cuda.empty_cache()


def test_sharded_reduction():
    n = (1 << 20) + 77
    x = torch.from_numpy(inputs.int_uniform_i32(8, 0, n)).cuda()
    hp, hc = _pair("sum_i32_i64", **CFG)
    res = []
    for h in (hp, hc):
        cuts = [0, 4097, 4098, 500001, n]
        recs = torch.zeros(len(cuts) - 1, 16, dtype=torch.uint8, device="cuda")
        for r in range(len(cuts) - 1):
            pyc.pyc_reduce_shard(h, n, cuts[r], cuts[r + 1] - cuts[r],
                                 [x.data_ptr() + 4 * cuts[r]], None, recs[r].data_ptr(), _s())
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        pyc.pyc_reduce_combine(h, len(cuts) - 1, recs.data_ptr(), out.data_ptr(), _s())
        res.append((recs.cpu(), out.cpu()))
    pyc.pyc_reduce_check_bounds(hc)
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


def test_server_replay():
    """A mixed replay (binary32 / bfloat16 / int32 maps and dots, sizes log-uniform
    in [2^4, 2^20], random offsets) through the serving loop, once with plain and
    once with checked handles."""
    P, nreq = 1 << 21, 1500
    x = inputs.uniform_f32(9, 0, P, -1.0, 1.0)
    y = inputs.uniform_f32(9, 1, P, -1.0, 1.0)
    pools = {"f32": (torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()),
             "bf16": (torch.from_numpy(x).to(torch.bfloat16).cuda(),
                      torch.from_numpy(y).to(torch.bfloat16).cuda()),
             "i32": (torch.from_numpy(inputs.int_uniform_i32(9, 2, P)).cuda(),
                     torch.from_numpy(inputs.int_uniform_i32(9, 3, P)).cuda())}
    maps = {"f32": "lin_comb_f32", "bf16": "lin_comb_bf16", "i32": "lin_comb_i32"}
    reds = {"f32": "dot_f32", "bf16": "dot_bf16", "i32": "dot_i32_i64"}
    rng = np.random.default_rng(12)
    plan = []
    for k in range(nreq):
        dt = ["f32", "bf16", "i32"][int(rng.integers(0, 3))]
        n = int(2 ** rng.uniform(4, 20))
        plan.append((rng.random() < 0.6, dt, n, int(rng.integers(0, P - n))))
    results = []
    for checked in (False, True):
        opts = dict(CFG, debug_bounds=1) if checked else dict(CFG)
        outs = {}
        table = pyc.RequestTable(nreq)
        for k, (red, dt, n, off) in enumerate(plan):
            a, b = pools[dt]
            es = a.element_size()
            ptrs = [a.data_ptr() + off * es, b.data_ptr() + off * es]
            if red:
                table.set(k, pyc.PYC_REQ_REDUCE, stock.create(reds[dt], **opts), n, ptrs)
            else:
                h = stock.create(maps[dt], **opts)
                outs[k] = torch.empty(n, dtype=a.dtype, device="cuda")
                table.set(k, pyc.PYC_REQ_MAP, h, n, ptrs + [outs[k].data_ptr()],
                          bytes(pyc.pack_scalars(h, [3, -2] if dt == "i32" else [A, B])))
        srv = pyc.pyc_server_create(1 << 32, max_batch=128)
        try:
            res = pyc.pyc_server_replay(srv, table, None, pyc.PYC_REPLAY_SERVER)
        finally:
            pyc.pyc_server_destroy(srv)
        assert all(r.status == pyc.PYC_OK for r in res)
        assert max(r.batch_size for r in res) > 1
        if checked:
            for dt in pools:
                pyc.pyc_map_check_bounds(stock.create(maps[dt], **opts))
                pyc.pyc_reduce_check_bounds(stock.create(reds[dt], **opts))
        results.append(([bytes(r.value) for r in res],
                        {k: v.view(torch.uint8).cpu() for k, v in outs.items()}))
    assert results[0][0] == results[1][0]
    assert all(torch.equal(results[0][1][k], results[1][1][k]) for k in results[0][1])


def test_narrowed_ranges_make_the_checks_fire(monkeypatch):
    """With every checked range narrowed by one element at its top, the access of
    the last element (or its vector group) is rejected: it is skipped, recorded,
    reported once by the check call, and the record is then clear."""
    monkeypatch.setenv("PYC_DEBUG_BOUNDS_SHRINK", "1")
    n = 1000
    x = torch.arange(n + 64, dtype=torch.float32, device="cuda")
    z = torch.full((n + 64,), -1.0, device="cuda")
    h = pyc.pyc_map_create("float *x, float *z", "z[i] = x[i] + 1", "narrowed_map",
                           dict(CFG, debug_bounds=1))
    src = pyc.pyc_map_source(h)
    assert "#define PYC_BOUNDS_SHRINK 1LL" in src
    pyc.pyc_map_launch(h, n, [x.data_ptr(), z.data_ptr()], None, _s())
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_map_check_bounds(h)
    assert e.value.status == pyc.PYC_E_INTERNAL and "outside" in e.value.message
    zc = z.cpu().numpy()
    assert np.array_equal(zc[:n - 4], np.arange(1, n - 3, dtype=np.float32))
    assert np.all(zc[n - 1:] == -1.0)  # the rejected store did not happen
    pyc.pyc_map_check_bounds(h)  # cleared
    r = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]", "float *x",
                              dict(CFG, debug_bounds=1))
    out = torch.zeros(1, device="cuda")
    pyc.pyc_reduce_launch(r, n, [x.data_ptr()], None, out.data_ptr(), _s())
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_check_bounds(r)
    assert e.value.status == pyc.PYC_E_INTERNAL and "load" in e.value.message
    pyc.pyc_reduce_check_bounds(r)  # cleared
    # a sharded launch runs in the handle's second module, whose records are read too
    rec = torch.zeros(16, dtype=torch.uint8, device="cuda")
    pyc.pyc_reduce_shard(r, n, 100, n - 100, [x.data_ptr() + 400], None, rec.data_ptr(), _s())
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_reduce_check_bounds(r)
    assert e.value.status == pyc.PYC_E_INTERNAL and "load" in e.value.message
    pyc.pyc_reduce_check_bounds(r)
    pyc.pyc_map_destroy(h)
    pyc.pyc_reduce_destroy(r)


SCAN_CFGS = [dict(vec_bytes=16, items_per_thread=1, block=128),
             dict(vec_bytes=32, items_per_thread=4, block=512)]


@pytest.mark.parametrize("cfg", range(len(SCAN_CFGS)))
def test_scans_small_sizes_all_offsets(cfg):
    """The scan's checked build (its own PYC_CHECK build, selected by the same
    option): exact scans (int32 -> int64 exclusive sum, binary32 maximum, the
    non-commutative affine composition) at n <= 1100 from 16 element offsets and
    at 2^20 + 77 from offset 3, plain against checked, no violation, same bits."""
    c = SCAN_CFGS[cfg]
    N = (1 << 20) + 77 + 16
    xi = torch.from_numpy(inputs.int_uniform_i32(15, 0, N)).cuda()
    xf = torch.from_numpy(inputs.uniform_f32(15, 1, N, -1.0, 1.0)).cuda()
    ca = torch.from_numpy(inputs.int_uniform_i32(15, 2, N, 0, 2 ** 31 - 1)).cuda()
    cb = torch.from_numpy(inputs.int_uniform_i32(15, 3, N, 0, 2 ** 31 - 1)).cuda()
    cases = [("cumsum_excl_i32_i64", [xi], torch.int64), ("cummax_f32", [xf], torch.float32),
             ("affine_u32", [ca, cb], torch.int64)]
    sizes = [(n, off) for n in list(range(0, 70)) + [255, 256, 257, 1000, 1100]
             for off in range(16)] + [((1 << 20) + 77, 3)]
    for name, ins, odt in cases:
        hp, hc = _pair(name, **c)
        for n, off in sizes:
            outs = []
            for h in (hp, hc):
                y = torch.zeros(N, dtype=odt, device="cuda")
                es = [a.element_size() for a in ins]
                pyc.pyc_scan_launch(h, n, [a.data_ptr() + off * e for a, e in zip(ins, es)] +
                                    [y.data_ptr() + off * y.element_size()], None, _s())
                outs.append(y)
            pyc.pyc_scan_sync(hc, _s())  # raises if the checked build recorded a violation
            pyc.pyc_scan_sync(hp, _s())
            assert torch.equal(outs[0].view(torch.uint8), outs[1].view(torch.uint8)), (name, n, off)


def test_narrowed_scan_ranges_make_the_checks_fire(monkeypatch):
    """With the scan's array ranges narrowed by one element (the test hook), the
    access of the last element is skipped and recorded, and pyc_scan_sync reports
    it as PYC_E_INTERNAL naming that index; the record is then cleared."""
    monkeypatch.setenv("PYC_DEBUG_BOUNDS_SHRINK", "1")
    n = 1000
    h = pyc.pyc_scan_create(pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "y[i] = item",
                            "int *x, long long *y", dict(SCAN_CFGS[0], debug_bounds=1))
    monkeypatch.delenv("PYC_DEBUG_BOUNDS_SHRINK")
    try:
        x = torch.ones(n, dtype=torch.int32, device="cuda")
        y = torch.zeros(n, dtype=torch.int64, device="cuda")
        pyc.pyc_scan_launch(h, n, [x.data_ptr(), y.data_ptr()], None, _s())
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_scan_sync(h, _s())
        assert e.value.status == pyc.PYC_E_INTERNAL
        # the recorded access covers the last element (one element, or its vector group)
        idx = int(re.search(r"index (-?\d+)", str(e.value)).group(1))
        assert n - 32 <= idx <= n - 1, str(e.value)
        pyc.pyc_scan_sync(h, _s())  # cleared
        # accesses below the narrowed group are unaffected
        assert torch.equal(y[: n - 32].cpu(), torch.arange(1, n - 31, dtype=torch.int64))
    finally:
        pyc.pyc_scan_destroy(h)
