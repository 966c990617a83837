"""Serving loop on the GPU: continuous batching of map and map-reduce requests
through the C ABI.  Each result is the same alone and in a mix (bit for bit),
agrees with the oracle, admission never exceeds the memory budget, and
deadlines, queue limits and the per-request baseline behave as declared."""
import numpy as np
import pytest
import torch

import oracle
from bounds import lin_comb_f32_bound, plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu
A, B = 2.5, -0.75
POOL = 1 << 22


@pytest.fixture(scope="module")
def pools():
    x = inputs.uniform_f32(31, 0, POOL, -1.0, 1.0)
    y = inputs.uniform_f32(31, 1, POOL, -1.0, 1.0)
    xi = inputs.int_uniform_i32(31, 2, POOL)
    yi = inputs.int_uniform_i32(31, 3, POOL)
    dev = {"x": torch.from_numpy(x).cuda(), "y": torch.from_numpy(y).cuda(),
           "xi": torch.from_numpy(xi).cuda(), "yi": torch.from_numpy(yi).cuda()}
    return {"x": x, "y": y, "xi": xi, "yi": yi}, dev


def _req(kind, name, n, off, dev, scal=None):
    h = stock.create(name)
    if name.endswith("i32") or name == "dot_i32_i64":
        a, b = dev["xi"], dev["yi"]
    else:
        a, b = dev["x"], dev["y"]
    es = a.element_size()
    ptrs = [a.data_ptr() + off * es, b.data_ptr() + off * es]
    if kind == pyc.PYC_REQ_MAP:
        ptrs.append(0)  # output allocated by the server
        scal = pyc.pack_scalars(h, [3, -2] if name.endswith("i32") else [A, B])
    return pyc.make_request(kind, h, n, ptrs, scal)


def _run_one(srv, req):
    rid = pyc.pyc_server_submit(srv, req)
    res = pyc.pyc_server_poll(srv, rid, 10_000_000)
    assert res is not None and res.status == pyc.PYC_OK
    return rid, res


def _map_out(res, n):
    """Copy a server-owned binary32 map output into a tensor (a copy map)."""
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    pyc.pyc_map_launch(stock.create("copy_f32"), n, [res.d_out, out.data_ptr()], None,
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out


def test_alone_and_in_the_mix_are_identical(pools):
    """Each probe request gives the same bits alone and inside batches of other
    requests.  To make the batching deterministic, a blocker request holds the
    whole memory budget while the mix queues up; releasing it admits the queue
    at once, so the scheduler forms large batches."""
    host, dev = pools
    nb = 1 << 24
    zeros = torch.zeros(2 * nb, device="cuda")
    budget = 8 * nb + 12  # the blocker's bytes (two binary32 arrays + result) + 8
    srv = pyc.pyc_server_create(budget, arena_bytes=1 << 27, num_streams=3, max_batch=64,
                                max_inflight=6)
    try:
        probes = [(pyc.PYC_REQ_REDUCE, "dot_f32", 300001, 5),
                  (pyc.PYC_REQ_REDUCE, "dot_f32", 777, 3),
                  (pyc.PYC_REQ_REDUCE, "dot_i32_i64", 100003, 11),
                  (pyc.PYC_REQ_MAP, "lin_comb_f32", 50001, 7)]
        alone = []
        for p in probes:
            req = _req(*p, dev)
            rid, res = _run_one(srv, req)
            val = bytes(res.value)
            out = _map_out(res, p[2]).cpu().numpy().copy() if p[0] == pyc.PYC_REQ_MAP else None
            if p[0] == pyc.PYC_REQ_MAP:  # the output shares its inputs' address mod 256
                assert res.d_out % 256 == (dev["x"].data_ptr() + 4 * p[3]) % 256
            pyc.pyc_server_release(srv, rid)
            alone.append((val, out))
        blocker = pyc.make_request(pyc.PYC_REQ_REDUCE, stock.create("dot_f32"), nb,
                                   [zeros.data_ptr(), zeros.data_ptr() + 4 * nb])
        bid, _ = _run_one(srv, blocker)  # finished, not released: the budget is held
        rng = np.random.default_rng(5)
        ids, keep = [], []
        for k in range(300):
            if k % 50 == 25:
                probe = (k // 50) % len(probes)
                req = _req(*probes[probe], dev)
            else:
                kind = pyc.PYC_REQ_REDUCE if rng.random() < 0.6 else pyc.PYC_REQ_MAP
                name = rng.choice(["dot_f32", "dot_i32_i64"]) if kind else rng.choice(
                    ["lin_comb_f32", "lin_comb_i32"])
                n = int(2 ** rng.uniform(0, 17))
                req = _req(kind, str(name), n, int(rng.integers(0, POOL - n)), dev)
                probe = -1
            keep.append(req)
            ids.append((pyc.pyc_server_submit(srv, req), probe))
        assert pyc.pyc_server_get_stats(srv)["queued"] == 300
        pyc.pyc_server_release(srv, bid)
        batched_probe = 0
        for rid, probe in ids:
            res = pyc.pyc_server_poll(srv, rid, 20_000_000)
            assert res is not None and res.status == pyc.PYC_OK
            if probe >= 0:
                val, out = alone[probe]
                assert bytes(res.value) == val
                if out is not None:
                    assert np.array_equal(_map_out(res, probes[probe][2]).cpu().numpy(), out)
                batched_probe = max(batched_probe, res.batch_size)
            pyc.pyc_server_release(srv, rid)
        assert batched_probe > 1  # the probes really ran inside batches
        st = pyc.pyc_server_get_stats(srv)
        assert st["completed"] == 305 and st["failed"] == 0 and st["admitted_bytes"] == 0
        assert st["arena_in_use"] == 0
        # results against the oracle
        v = np.frombuffer(alone[0][0][:4], np.float32)[0]
        ref, ab = oracle.dot_f32(host["x"][5:300006], host["y"][5:300006])
        assert abs(v - ref) <= plain_sum_bound(ab)
        vi = np.frombuffer(alone[2][0][:8], np.int64)[0]
        assert vi == oracle.dot_i32_i64(host["xi"][11:100014], host["yi"][11:100014])
        z = alone[3][1]
        want = oracle.map_lin_comb_f32ops(A, host["x"][7:50008], B, host["y"][7:50008])
        assert np.array_equal(z, want)
    finally:
        pyc.pyc_server_destroy(srv)


def test_admission_respects_budget(pools):
    _, dev = pools
    budget = 24 << 20
    srv = pyc.pyc_server_create(budget, arena_bytes=16 << 20, num_streams=2, max_batch=16,
                                max_inflight=4)
    try:
        reqs, ids = [], []
        for k in range(200):
            n = 50000 + 997 * k
            r = _req(pyc.PYC_REQ_REDUCE, "dot_f32", n, k, dev)
            reqs.append(r)
            ids.append(pyc.pyc_server_submit(srv, r))
        for rid in ids:
            res = pyc.pyc_server_poll(srv, rid, 20_000_000)
            assert res is not None and res.status == pyc.PYC_OK
            pyc.pyc_server_release(srv, rid)
        st = pyc.pyc_server_get_stats(srv)
        assert 0 < st["peak_admitted_bytes"] <= budget
        with pytest.raises(pyc.PycError) as e:  # larger than the whole budget
            pyc.pyc_server_submit(srv, _req(pyc.PYC_REQ_REDUCE, "dot_f32", 4 << 20, 0, dev))
        assert e.value.status == pyc.PYC_E_NOMEM
    finally:
        pyc.pyc_server_destroy(srv)


def test_deadline_queue_limit_and_errors(pools):
    _, dev = pools
    n = 1 << 20
    per = n * 8 + 4  # two binary32 arrays + the result
    srv = pyc.pyc_server_create(per, num_streams=1, max_batch=4, max_inflight=2, max_queue=3)
    try:
        held = _req(pyc.PYC_REQ_REDUCE, "dot_f32", n, 0, dev)
        rid, _ = _run_one(srv, held)  # finished but not released: the budget is full
        late = _req(pyc.PYC_REQ_REDUCE, "dot_f32", n, 1, dev)
        late[0].deadline_us = 2000
        lid = pyc.pyc_server_submit(srv, late)
        res = pyc.pyc_server_poll(srv, lid, 5_000_000)
        assert res is not None and res.status == pyc.PYC_E_TIMEOUT
        pyc.pyc_server_release(srv, lid)
        waiting = [_req(pyc.PYC_REQ_REDUCE, "dot_f32", n, 2 + k, dev) for k in range(4)]
        wids = [pyc.pyc_server_submit(srv, w) for w in waiting[:3]]
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_server_submit(srv, waiting[3])
        assert e.value.status == pyc.PYC_E_BUSY  # queue full
        assert pyc.pyc_server_poll(srv, wids[0], 0) is None  # still waiting: budget held
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_server_release(srv, wids[0])
        assert e.value.status == pyc.PYC_E_BUSY
        pyc.pyc_server_release(srv, rid)  # frees the budget; the queue drains
        for w in wids:
            res = pyc.pyc_server_poll(srv, w, 10_000_000)
            assert res is not None and res.status == pyc.PYC_OK
            pyc.pyc_server_release(srv, w)
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_server_poll(srv, 123456789, 0)
        assert e.value.status == pyc.PYC_E_NOTFOUND
    finally:
        pyc.pyc_server_destroy(srv)


def test_bad_arrays_fail_at_submit_and_spare_the_batch(pools):
    """A NULL array (other than a written-only map output), one not aligned to its
    element size, or an output overlapping an input in part is refused by
    pyc_server_submit itself, also for an array the statement indexes other than
    as name[i]; a good request after it runs."""
    _, dev = pools
    srv = pyc.pyc_server_create(1 << 30, num_streams=1)
    diff = pyc.pyc_map_create("float *x, float *y", "y[i] = x[i + 1] - x[i]")
    try:
        x, y = dev["x"], dev["y"]
        out = torch.empty(1000, dtype=torch.float32, device="cuda")
        bad = [(pyc.PYC_REQ_MAP, diff, [0, out.data_ptr()]),
               (pyc.PYC_REQ_MAP, diff, [x.data_ptr() + 2, out.data_ptr()]),
               (pyc.PYC_REQ_REDUCE, stock.create("dot_f32"), [x.data_ptr() + 1, y.data_ptr()]),
               (pyc.PYC_REQ_REDUCE, stock.create("dot_f32"), [x.data_ptr(), 0]),
               # an output overlapping an input in part (exact aliasing would be allowed)
               (pyc.PYC_REQ_MAP, stock.create("lin_comb_f32"),
                [x.data_ptr(), y.data_ptr(), x.data_ptr() + 4])]
        for kind, h, ptrs in bad:
            scal = pyc.pack_scalars(h, [A, B]) if len(ptrs) == 3 else None
            with pytest.raises(pyc.PycError) as e:
                pyc.pyc_server_submit(srv, pyc.make_request(kind, h, 1000, ptrs, scal))
            assert e.value.status == pyc.PYC_E_ARG
        _run_one(srv, pyc.make_request(pyc.PYC_REQ_MAP, diff, 1000, [x.data_ptr(), out.data_ptr()]))
        want = (x[1:1001] - x[:1000]).cpu()
        assert torch.equal(out.cpu(), want)
        st = pyc.pyc_server_get_stats(srv)
        assert st["failed"] == 0 and st["completed"] == 1
    finally:
        pyc.pyc_server_destroy(srv)
        pyc.pyc_map_destroy(diff)


def test_replay_server_and_direct_agree(pools):
    host, dev = pools
    nreq = 3000
    rng = np.random.default_rng(8)
    srv = pyc.pyc_server_create(1 << 30, arena_bytes=1 << 28)
    try:
        table = pyc.RequestTable(nreq)
        plan = []
        for k in range(nreq):
            kind = pyc.PYC_REQ_REDUCE if rng.random() < 0.6 else pyc.PYC_REQ_MAP
            ints = rng.random() < 0.5
            name = ("dot_i32_i64" if ints else "dot_f32") if kind else (
                "lin_comb_i32" if ints else "lin_comb_f32")
            n = int(2 ** rng.uniform(4, 19))
            off = int(rng.integers(0, POOL - n))
            req, arr, sc = _req(kind, name, n, off, dev)
            ptrs = [arr[j] for j in range(len(arr))]
            table.set(k, kind, stock.create(name), n, ptrs, bytes(sc) if sc is not None else b"")
            plan.append((kind, name, n, off))
        gaps = rng.exponential(1e9 / 200000.0, nreq).astype(np.int64)
        arrival = np.cumsum(gaps)
        rs = pyc.pyc_server_replay(srv, table, arrival, pyc.PYC_REPLAY_SERVER)
        rd = pyc.pyc_server_replay(srv, table, None, pyc.PYC_REPLAY_DIRECT)
        assert all(r.status == pyc.PYC_OK for r in rs) and all(r.status == pyc.PYC_OK for r in rd)
        assert max(r.batch_size for r in rs) > 1 and max(r.batch_size for r in rd) == 1
        for k, (kind, name, n, off) in enumerate(plan):
            if kind != pyc.PYC_REQ_REDUCE:
                continue
            if name == "dot_i32_i64":
                want = oracle.dot_i32_i64(host["xi"][off:off + n], host["yi"][off:off + n])
                assert np.frombuffer(bytes(rs[k].value)[:8], np.int64)[0] == want
                assert np.frombuffer(bytes(rd[k].value)[:8], np.int64)[0] == want
            elif k % 7 == 0:
                ref, ab = oracle.dot_f32(host["x"][off:off + n], host["y"][off:off + n])
                for r in (rs[k], rd[k]):
                    assert abs(np.frombuffer(bytes(r.value)[:4], np.float32)[0] - ref) <= \
                        plain_sum_bound(ab)
        lat = np.array([r.t_done_ns - r.t_submit_ns for r in rs]) / 1e3
        print("replay 3000 req at 200k/s: p50 %.1f us p99 %.1f us" % tuple(np.percentile(lat, [50, 99])))
        st = pyc.pyc_server_get_stats(srv)
        assert st["admitted_bytes"] == 0 and st["arena_in_use"] == 0
    finally:
        pyc.pyc_server_destroy(srv)


def test_serving_config_mix_against_the_oracle():
    """The serving workload's own mix and sizes (50,000-request config, here its
    first 2,000 requests' recipe): Poisson arrivals at 20,000/s, 60 % dot / 40 %
    a*x+b*y, dtype uniform over binary32 / bfloat16 / int32, sizes log-uniform in
    [2^10, 2^26], inputs at random offsets of 2^26-element pools, a 40 GB cap.
    Every request of at most 2^16 elements and one in 100 of the rest is checked
    against the oracle (Sec. 3.2.4 / 3.2.5 define each request's result): map
    outputs element by element -- bit-exact binary32 source-order evaluation for
    binary32 and bfloat16 storage (rounded once on the store), exact for int32 --
    and dots within the plain-sum bound (exact for int32).  The other maps write
    into one shared sink per dtype that nothing reads."""
    nreq, P = 2000, 1 << 26
    x = inputs.uniform_f32(4, 0, P, -1.0, 1.0)
    y = inputs.uniform_f32(4, 1, P, -1.0, 1.0)
    xb, yb = inputs.to_bf16_values(x), inputs.to_bf16_values(y)
    xi, yi = inputs.int_uniform_i32(4, 2, P), inputs.int_uniform_i32(4, 3, P)
    host = {"f32": (x, y), "bf16": (xb, yb), "i32": (xi, yi)}
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "i32": torch.int32}
    dev = {k: (torch.from_numpy(a).to(tdt[k]).cuda(), torch.from_numpy(b).to(tdt[k]).cuda())
           for k, (a, b) in host.items()}
    sink = {k: torch.empty(P, dtype=tdt[k], device="cuda") for k in host}
    maps = {"f32": "lin_comb_f32", "bf16": "lin_comb_bf16", "i32": "lin_comb_i32"}
    reds = {"f32": "dot_f32", "bf16": "dot_bf16", "i32": "dot_i32_i64"}
    scal = {k: bytes(pyc.pack_scalars(stock.create(v), [3, -2] if k == "i32" else [A, B]))
            for k, v in maps.items()}
    u_kind = inputs.unit_f64(50, 0, nreq)
    u_dt = inputs.unit_f64(50, 1, nreq)
    sizes = inputs.loguniform_i64(50, 2, nreq, 10.0, 16.0, 1 << 10, 1 << 26)
    u_off = inputs.unit_f64(50, 3, nreq)
    arrival = np.cumsum(inputs.exponential_f64(50, 4, nreq, 20000.0) * 1e9).astype(np.int64)
    table = pyc.RequestTable(nreq)
    plan, outs = [], {}
    for k in range(nreq):
        dt = ["f32", "bf16", "i32"][min(2, int(u_dt[k] * 3))]
        n = int(sizes[k])
        off = int(u_off[k] * (P - n + 1))
        a, b = dev[dt]
        es = a.element_size()
        ptrs = [a.data_ptr() + off * es, b.data_ptr() + off * es]
        check = n <= (1 << 16) or k % 100 == 0
        if u_kind[k] < 0.6:
            table.set(k, pyc.PYC_REQ_REDUCE, stock.create(reds[dt]), n, ptrs)
            plan.append((pyc.PYC_REQ_REDUCE, dt, n, off, check))
        else:
            if check:
                outs[k] = torch.empty(n, dtype=tdt[dt], device="cuda")
                z = outs[k].data_ptr()
            else:
                z = sink[dt].data_ptr() + off * es  # same alignment as the inputs
            table.set(k, pyc.PYC_REQ_MAP, stock.create(maps[dt]), n, ptrs + [z], scal[dt])
            plan.append((pyc.PYC_REQ_MAP, dt, n, off, check))
    srv = pyc.pyc_server_create(40 << 30)
    try:
        res = pyc.pyc_server_replay(srv, table, arrival, pyc.PYC_REPLAY_SERVER)
        torch.cuda.synchronize()
        assert all(r.status == pyc.PYC_OK for r in res)
        assert max(r.batch_size for r in res) > 1  # requests really shared launches
        st = pyc.pyc_server_get_stats(srv)
        assert st["peak_admitted_bytes"] <= 40 << 30 and st["admitted_bytes"] == 0
    finally:
        pyc.pyc_server_destroy(srv)
    checked = {"map": 0, "reduce": 0, "elements": 0, "bf16_maps": 0, "big": 0}
    for k, (kind, dt, n, off, check) in enumerate(plan):
        if not check:
            continue
        a, b = host[dt][0][off:off + n], host[dt][1][off:off + n]
        checked["elements"] += n
        checked["big"] += n > (1 << 16)
        if kind == pyc.PYC_REQ_MAP:
            checked["map"] += 1
            if dt == "i32":
                want = (3 * a.astype(np.int64) - 2 * b.astype(np.int64)).astype(np.int32)
                got = outs[k].cpu().numpy()
            else:
                want = oracle.map_lin_comb_f32ops(A, a, B, b, out_bf16=(dt == "bf16"))
                got = outs[k].float().cpu().numpy()
                checked["bf16_maps"] += dt == "bf16"
            assert np.array_equal(got, want), (k, dt, n, off)
        else:
            checked["reduce"] += 1
            raw = bytes(res[k].value)
            if dt == "i32":
                assert np.frombuffer(raw[:8], np.int64)[0] == oracle.dot_i32_i64(a, b), (k, n)
            else:
                ref, ab = oracle.dot_f32(a, b)
                v = float(np.frombuffer(raw[:4], np.float32)[0])
                assert abs(v - ref) <= plain_sum_bound(ab), (k, dt, n, v, ref)
    print("serving mix: checked", checked)
    assert checked["map"] > 200 and checked["reduce"] > 300 and checked["bf16_maps"] > 50
    assert checked["big"] >= 10


def test_chunking_edges_alone():
    """Requests whose lengths sit on the edges of the server's chunking -- one warp
    (at most 2048 elements) or one CTA chunk, the least chunk (4096), where about
    256 chunks stop being the least chunk (2^20), where the chunk reaches its cap
    (2^24), ragged tails and misaligned starts -- each served alone: int32 dot
    products into int64 and int32 maps bit-exact, binary32 dots within the plain
    sum's bound."""
    N = (1 << 25) + 64
    xi, yi = inputs.int_uniform_i32(32, 0, N), inputs.int_uniform_i32(32, 1, N)
    x, y = inputs.uniform_f32(32, 2, N, -1.0, 1.0), inputs.uniform_f32(32, 3, N, -1.0, 1.0)
    dxi, dyi = torch.from_numpy(xi).cuda(), torch.from_numpy(yi).cuda()
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    dz = torch.empty(N, dtype=torch.int32, device="cuda")
    hdi, hdf, hm = stock.create("dot_i32_i64"), stock.create("dot_f32"), stock.create("lin_comb_i32")
    sc = pyc.pack_scalars(hm, [3, -2])
    sizes = [2048, 2049, 4095, 4096, 4097, 65537, (1 << 20) - 1, 1 << 20, (1 << 20) + 1,
             (1 << 22) + 3, (1 << 24) - 1, (1 << 24) + 4097, (1 << 25) - 5]
    srv = pyc.pyc_server_create(8 << 30)
    try:
        for n in sizes:
            for off in (0, 3):
                a, b = xi[off:off + n], yi[off:off + n]
                rid, r = _run_one(srv, pyc.make_request(
                    pyc.PYC_REQ_REDUCE, hdi, n, [dxi.data_ptr() + 4 * off, dyi.data_ptr() + 4 * off]))
                pyc.pyc_server_release(srv, rid)
                got = np.frombuffer(bytes(r.value)[:8], np.int64)[0]
                assert got == oracle.dot_i32_i64(a, b), ("dot i32", n, off)
                rid, r = _run_one(srv, pyc.make_request(
                    pyc.PYC_REQ_REDUCE, hdf, n, [dx.data_ptr() + 4 * off, dy.data_ptr() + 4 * off]))
                pyc.pyc_server_release(srv, rid)
                ref, ab = oracle.dot_f32(x[off:off + n], y[off:off + n])
                v = float(np.frombuffer(bytes(r.value)[:4], np.float32)[0])
                assert abs(v - ref) <= plain_sum_bound(ab), ("dot f32", n, off, v, ref)
                rid, r = _run_one(srv, pyc.make_request(
                    pyc.PYC_REQ_MAP, hm, n, [dxi.data_ptr() + 4 * off, dyi.data_ptr() + 4 * off,
                                             dz.data_ptr() + 4 * off], sc))
                pyc.pyc_server_release(srv, rid)
                want = (3 * a.astype(np.int64) - 2 * b.astype(np.int64)).astype(np.int32)
                assert np.array_equal(dz[off:off + n].cpu().numpy(), want), ("map i32", n, off)
    finally:
        pyc.pyc_server_destroy(srv)
