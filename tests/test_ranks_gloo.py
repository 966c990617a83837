"""The benchmark's multi-rank path on CPU (gloo, world size 2): every rank gets
the slowest rank's step time, the whole-job value counts every rank's bytes,
and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = [2.0, 3.5][rank]  # rank 1 is the slower replica
        ms = bench.max_over_ranks(step_ms, dist)
        out[rank] = (ms, bench.whole_job_gbs(1e9, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 3.5
    # 2 ranks x 1 GB in 3.5 ms
    assert res[0][1] == pytest.approx(2 * 1e9 / 3.5e-3 / 1e9)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_gbs(2e9, 1, 1.0) == pytest.approx(2000.0)


def test_reference_arm_prints_on_rank0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 1})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


# ---------------------------------------------------------------- sharded map-reduce
# The host side of paper_1304_5553_gb300.shard.ShardedReduce among gloo ranks on
# CPU: shard bounds, the exchange of 16-byte records in rank order, and the
# combine.  The two GPU steps (pyc_reduce_shard / pyc_reduce_combine) are
# replaced by the oracle's per-shard partial and in-order combine, packed into
# records of the same 16 bytes.

_KINDS = ("sum_i32_i64", "argmin_f32", "argmax_f32", "max_f32", "sum_f32", "dot_f32")


def _pack(kind, p):
    import struct
    if kind == "sum_i32_i64":
        return struct.pack("<qq", p, 0)
    if kind == "max_f32":
        return struct.pack("<fiq", p, 0, 0)
    if kind in ("argmin_f32", "argmax_f32"):
        return struct.pack("<fiq", p[0], 0, p[1])
    return struct.pack("<dd", p[0], p[1])


def _unpack(kind, b):
    import struct
    if kind == "sum_i32_i64":
        return struct.unpack("<qq", b)[0]
    if kind == "max_f32":
        return struct.unpack("<fiq", b)[0]
    if kind in ("argmin_f32", "argmax_f32"):
        v, _, i = struct.unpack("<fiq", b)
        return v, i
    return struct.unpack("<dd", b)


def _shard_inputs(kind, n, world):
    import numpy as np
    from paper_1304_5553_gb300 import inputs
    from paper_1304_5553_gb300.shard import shard_bounds
    if kind == "sum_i32_i64":
        return [inputs.int_uniform_i32(41, 0, n)]
    if kind == "dot_f32":
        return [inputs.uniform_f32(41, s, n, -1.0, 1.0) for s in range(2)]
    if kind == "sum_f32":
        return [inputs.lognormal_signed_f32(41, 0, n)]
    x = inputs.uniform_f32(41, 0, n, -2.0, 2.0)
    ext = np.float32(-3.0 if kind == "argmin_f32" else 3.0)
    b = shard_bounds(n, world)
    for r in range(1, world):  # ties of the extremum straddling every cut
        if not 0 < b[r] < n:
            continue
        x[b[r] - 1] = ext
        x[b[r]] = ext
    return [x]


def _shard_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import oracle
    from paper_1304_5553_gb300.shard import ShardedReduce
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for kind in _KINDS:
            for n in (0, 5, 100003):
                arrays = _shard_inputs(kind, n, world)
                sr = ShardedReduce(None, n, rank, world)
                mine = [a[sr.i0:sr.i0 + sr.n] for a in arrays]
                rec = torch.from_numpy(np.frombuffer(
                    _pack(kind, oracle.shard_partial(kind, mine, sr.i0)), np.uint8).copy())
                recs = sr.exchange(rec)
                assert tuple(recs.shape) == (world, 16)
                parts = [_unpack(kind, bytes(recs[r].numpy())) for r in range(world)]
                res[(kind, n)] = (sr.i0, sr.n, oracle.combine_partials(kind, parts))
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_reduce_exchange_and_combine(world):
    sys.path.insert(0, ROOT)
    import oracle
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = {r: dict(v) for r, v in out.items()}
    for kind in _KINDS:
        for n in (0, 5, 100003):
            # the shards tile [0, n) in rank order
            spans = [res[r][(kind, n)][:2] for r in range(world)]
            assert spans[0][0] == 0 and sum(s[1] for s in spans) == n
            assert all(spans[r][0] + spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            got = [res[r][(kind, n)][2] for r in range(world)]
            assert all(g == got[0] for g in got)  # every rank holds the same result
            arrays = _shard_inputs(kind, n, world)
            if kind == "sum_i32_i64":
                assert got[0] == oracle.sum_i32_i64(arrays[0])
            elif kind in ("argmin_f32", "argmax_f32", "max_f32"):
                whole = getattr(oracle, kind)(arrays[0])
                assert got[0] == (tuple(whole) if kind != "max_f32" else whole)
                if n > 5 and kind != "max_f32":  # the first of the straddling ties
                    from paper_1304_5553_gb300.shard import shard_bounds
                    assert got[0][1] == shard_bounds(n, world)[1] - 1
            else:
                ref, ab = (oracle.sum_f32(arrays[0]) if kind == "sum_f32"
                           else oracle.dot_f32(*arrays))
                assert abs(got[0][0] - ref) <= 2.0 ** -50 * ab + 1e-300


def test_shard_bounds_partition():
    sys.path.insert(0, ROOT)
    from paper_1304_5553_gb300.shard import shard_bounds
    for n in (0, 1, 7, 2 ** 28 + 3):
        for world in (1, 2, 3, 8):
            b = shard_bounds(n, world)
            assert b[0] == 0 and b[-1] == n and len(b) == world + 1
            lens = [b[r + 1] - b[r] for r in range(world)]
            assert min(lens) >= 0 and max(lens) - min(lens) <= 1
    with pytest.raises(ValueError):
        shard_bounds(5, 0)


def test_segment_bounds_balance_and_cover():
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1304_5553_gb300 import inputs
    from paper_1304_5553_gb300.shard import segment_bounds
    lens = inputs.segment_lengths()  # the 20,000-segment table
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    for world in (1, 2, 3, 8):
        b = segment_bounds(off, world)
        assert b[0] == 0 and b[-1] == lens.size and all(b[r] <= b[r + 1] for r in range(world))
        per = [int(off[b[r + 1]] - off[b[r]]) for r in range(world)]
        assert sum(per) == int(off[-1])
        # each cut is within one segment (at most 2^20 elements) of its target
        assert max(per) - min(per) <= 2 * (1 << 20)
    assert segment_bounds(np.array([0, 5]), 3) in ([0, 0, 1, 1], [0, 1, 1, 1], [0, 0, 0, 1])
    assert segment_bounds(np.array([7]), 2) == [0, 0, 0]


def _segment_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import oracle
    from paper_1304_5553_gb300 import inputs
    from paper_1304_5553_gb300.shard import segment_bounds
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lens = inputs.segment_lengths(nseg=300, seed=44, max_log2=12)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        x = inputs.uniform_f32(44, 0, int(off[-1]), -1.0, 1.0)
        y = inputs.uniform_f32(44, 1, int(off[-1]), -1.0, 1.0)
        b = segment_bounds(off, world)
        s0, s1 = b[rank], b[rank + 1]
        # this rank's part of the table and arrays (what it would hold on its GPU);
        # the oracle stands in for pyc_reduce_batched
        mine = off[s0:s1 + 1] - off[s0]
        lo, hi = int(off[s0]), int(off[s1])
        vals, _ = oracle.dot_segments_f32(mine, x[lo:hi], y[lo:hi])
        out[rank] = (s0, s1, vals.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_segmented_batch_shards_without_exchange():
    """Each rank reduces its own whole segments; together the ranks' results are
    the unsharded table's, segment for segment (world size 3)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_1304_5553_gb300 import inputs
    world = 3
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_segment_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    lens = inputs.segment_lengths(nseg=300, seed=44, max_log2=12)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    x = inputs.uniform_f32(44, 0, int(off[-1]), -1.0, 1.0)
    y = inputs.uniform_f32(44, 1, int(off[-1]), -1.0, 1.0)
    whole, _ = oracle.dot_segments_f32(off, x, y)
    got = np.concatenate([np.array(res[r][2]) for r in range(world)])
    assert [res[r][0] for r in range(world)] == sorted(res[r][0] for r in range(world))
    assert got.size == lens.size and np.array_equal(got, whole)
