"""Sharded map-reduce on the GPU: pyc_reduce_shard + pyc_reduce_combine.

Several "virtual ranks" run on one GPU one after another: each folds its shard
of one device array (a pointer to the shard's first element) into a 16-byte
record, the records are placed side by side as an all-gather would leave them,
and pyc_reduce_combine folds them.  Sec. 3.2.5's reduction of the whole range
is the reference: integer sums, max and argmin / argmax must match the oracle
bit for bit whatever the cuts (ties of the minimum straddling a cut, cuts inside
a vector tile, empty shards, shards at odd element offsets), floating-point
sums within the stated bounds; each record must also be the oracle's partial of
its own shard (global indices included).
"""
import numpy as np
import pytest
import torch

import oracle
from bounds import compensated_sum_bound, plain_sum_bound
from paper_1304_5553_gb300 import inputs, pyc, stock

pytestmark = pytest.mark.gpu

N = (1 << 20) + 77
CUTS = [
    [0, N],                          # one shard
    [0, 4097, N],                    # a cut inside a vector tile
    [0, 0, N],                       # an empty first shard
    [0, N, N],                       # an empty last shard
    [0, 1, 2, 3, N],                 # shards of one element at odd offsets
    [0, 123457, 500001, 777777, N],  # five uneven shards
]


def _s():
    return torch.cuda.current_stream().cuda_stream


def _sharded(name, arrays, cuts, scalars=None):
    """(records as bytes per shard, combined result as raw bytes)."""
    h = stock.create(name) if isinstance(name, str) else name
    k = len(cuts) - 1
    recs = torch.zeros(k, 16, dtype=torch.uint8, device="cuda")
    for r in range(k):
        ptrs = [a.data_ptr() + cuts[r] * a.element_size() for a in arrays]
        pyc.pyc_reduce_shard(h, cuts[-1], cuts[r], cuts[r + 1] - cuts[r], ptrs, scalars,
                             recs[r].data_ptr(), _s())
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    pyc.pyc_reduce_combine(h, k, recs.data_ptr(), out.data_ptr(), _s())
    torch.cuda.synchronize()
    return [bytes(recs[r].cpu().numpy()) for r in range(k)], out.cpu().numpy().view(np.uint8)


def _f32(b):
    return float(np.frombuffer(bytes(b[:4]), np.float32)[0])


def _i64(b, off=0):
    return int(np.frombuffer(bytes(b[off:off + 8]), np.int64)[0])


def _f64(b, off=0):
    return float(np.frombuffer(bytes(b[off:off + 8]), np.float64)[0])


@pytest.fixture(scope="module")
def data():
    x = inputs.lognormal_signed_f32(31, 0, N)
    y = inputs.uniform_f32(31, 1, N, -1.0, 1.0)
    xi = inputs.int_uniform_i32(31, 2, N)
    xu = inputs.uniform_f32(31, 3, N, -2.0, 2.0)
    d = {k: torch.from_numpy(v).cuda() for k, v in dict(x=x, y=y, xi=xi).items()}
    return dict(x=x, y=y, xi=xi, xu=xu, d=d)


def _extremes(base, cuts, v, last_only=False):
    """base with the value v (beyond base's range) at both sides of every inner
    cut, or only at the first element of the last shard."""
    x = base.copy()
    inner = [c for c in cuts[1:-1] if 0 < c < x.size]
    if last_only:
        if inner:
            x[inner[-1]] = v
        return x
    for c in inner:
        x[c - 1] = v
        x[c] = v
    return x


@pytest.mark.parametrize("cuts", CUTS, ids=lambda c: "x".join(str(v) for v in c))
def test_exact_reductions_match_the_whole(data, cuts):
    d = data["d"]
    recs, out = _sharded("sum_i32_i64", [d["xi"]], cuts)
    assert _i64(out) == oracle.sum_i32_i64(data["xi"])
    for r, rec in enumerate(recs):  # each record is its shard's own sum
        assert _i64(rec) == oracle.shard_partial("sum_i32_i64",
                                                 [data["xi"][cuts[r]:cuts[r + 1]]], cuts[r])
        assert rec[8:] == bytes(8)
    for name, v in (("argmin_f32", -2.5), ("argmax_f32", 2.5)):
        for last_only in (False, True):
            xa = _extremes(data["xu"], cuts, v, last_only)
            recs, out = _sharded(name, [torch.from_numpy(xa).cuda()], cuts)
            assert (_f32(out), _i64(out, 8)) == getattr(oracle, name)(xa)
            for r, rec in enumerate(recs):
                want = oracle.shard_partial(name, [xa[cuts[r]:cuts[r + 1]]], cuts[r])
                assert (_f32(rec), _i64(rec, 8)) == want
    recs, out = _sharded("max_f32", [d["x"]], cuts)
    assert _f32(out) == oracle.max_f32(data["x"])


@pytest.mark.parametrize("cuts", CUTS, ids=lambda c: "x".join(str(v) for v in c))
def test_float_sums_within_bounds(data, cuts):
    d, x, y = data["d"], data["x"], data["y"]
    recs, out = _sharded("sum_f32", [d["x"]], cuts)
    ref, ab = oracle.sum_f32(x)
    assert abs(_f32(out) - ref) <= plain_sum_bound(ab)
    recs, out = _sharded("dot_f32", [d["x"], d["y"]], cuts)
    ref, ab = oracle.dot_f32(x, y)
    assert abs(_f32(out) - ref) <= plain_sum_bound(ab)
    # compensated: binary64 (hi, lo) records, one rounding at the end
    recs, out = _sharded("sum_f32_comp", [d["x"]], cuts)
    ex = oracle.exact_sum_f32(x)
    assert abs(_f32(out) - ex) <= compensated_sum_bound(ex, oracle.sum_f32(x)[1])
    for r, rec in enumerate(recs):
        part = x[cuts[r]:cuts[r + 1]]
        ex_r, ab_r = oracle.exact_sum_f32(part), oracle.sum_f32(part)[1]
        # the record (hi + lo, before the final rounding) is within the
        # compensated tolerance of its shard's exact sum
        assert abs((_f64(rec) + _f64(rec, 8)) - ex_r) <= compensated_sum_bound(ex_r, ab_r)


def test_bf16_dot_records_keep_binary32_accumulators(data):
    cuts = [0, 333333, 333334, N]
    xb = torch.from_numpy(data["x"]).to(torch.bfloat16)
    yb = torch.from_numpy(data["y"]).to(torch.bfloat16)
    recs, out = _sharded("dot_bf16", [xb.cuda(), yb.cuda()], cuts)
    ref, ab = oracle.dot_f32(xb.float().numpy(), yb.float().numpy())
    assert abs(_f32(out) - ref) <= plain_sum_bound(ab)
    for r, rec in enumerate(recs):
        ref_r, ab_r = oracle.dot_f32(xb[cuts[r]:cuts[r + 1]].float().numpy(),
                                     yb[cuts[r]:cuts[r + 1]].float().numpy())
        assert abs(_f32(rec) - ref_r) <= plain_sum_bound(ab_r) and rec[4:] == bytes(12)


def test_map_expression_sees_the_global_index(data):
    # sum of i * x[i] (exact in 64-bit integers): i must be the global index
    h = pyc.pyc_reduce_create(pyc.PYC_I64, "0", "a+b", "i * (long long)x[i]", "int *x")
    xi = data["xi"]
    want = int(np.dot(np.arange(N, dtype=np.int64), xi.astype(np.int64)))
    for cuts in CUTS:
        _, out = _sharded(h, [data["d"]["xi"]], cuts)
        assert _i64(out) == want
    # n in the expression is the whole range's length
    hn = pyc.pyc_reduce_create(pyc.PYC_I64, "0", "a+b", "(i < n / 2) ? (long long)x[i] : 0LL",
                               "int *x")
    _, out = _sharded(hn, [data["d"]["xi"]], [0, 1000, 600000, N])
    assert _i64(out) == int(xi[:N // 2].astype(np.int64).sum())
    pyc.pyc_reduce_destroy(h)
    pyc.pyc_reduce_destroy(hn)


def test_combine_of_zero_records_is_the_neutral_element():
    for name, check in (("sum_i32_i64", lambda o: _i64(o) == 0),
                        ("argmin_f32", lambda o: _f32(o) == np.inf and _i64(o, 8) == 2 ** 63 - 1),
                        ("sum_f32_comp", lambda o: _f32(o) == 0.0)):
        h = stock.create(name)
        out = torch.full((2,), 7, dtype=torch.int64, device="cuda")
        pyc.pyc_reduce_combine(h, 0, 0, out.data_ptr(), _s())
        torch.cuda.synchronize()
        assert check(out.cpu().numpy().view(np.uint8))


def test_full_size_two_shards():
    """n = 2^28 (the reductions' size) cut in two inside a tile, in the
    configuration the tuner picks for a shard of that size."""
    n = 1 << 28
    cut = (n >> 1) + 4099
    xi = inputs.int_uniform_i32(0, 0, n)
    xa = inputs.argmin_with_minima(0, n)
    h_sum, h_arg = stock.create("sum_i32_i64"), stock.create("argmin_f32")
    for h in (h_sum, h_arg):
        pyc.pyc_reduce_autotune(h, n >> 1, _s())
    d = torch.from_numpy(xi).cuda()
    _, out = _sharded(h_sum, [d], [0, cut, n])
    assert _i64(out) == oracle.sum_i32_i64(xi)
    del d
    d = torch.from_numpy(xa).cuda()
    _, out = _sharded(h_arg, [d], [0, cut, n])
    assert (_f32(out), _i64(out, 8)) == oracle.argmin_f32(xa)


def test_a_thousand_shards(data):
    """1,000 uneven shards (some empty): the combine folds more records than it
    has threads (256), still exactly for integer sums and argmin, and within the
    compensated bound for the compensated sum."""
    rng = np.random.default_rng(77)
    cuts = [0] + sorted(int(c) for c in rng.integers(0, N + 1, 999)) + [N]
    d = data["d"]
    _, out = _sharded("sum_i32_i64", [d["xi"]], cuts)
    assert _i64(out) == oracle.sum_i32_i64(data["xi"])
    xa = _extremes(data["xu"], cuts, -2.5)
    _, out = _sharded("argmin_f32", [torch.from_numpy(xa).cuda()], cuts)
    assert (_f32(out), _i64(out, 8)) == oracle.argmin_f32(xa)
    _, out = _sharded("sum_f32_comp", [d["x"]], cuts)
    ex = oracle.exact_sum_f32(data["x"])
    assert abs(_f32(out) - ex) <= compensated_sum_bound(ex, oracle.sum_f32(data["x"])[1])


def test_shards_beyond_2e31_elements():
    """n = 2^31 + 100003: shards that start and end on either side of 2^31.
    An argmin's record carries the global index (above 2^31, first of two
    equal minima), an int32 sum's record its shard's int64 sum; the combine
    gives the whole range's.  Inputs are constant except at a few planted
    elements, so every record is known exactly."""
    n = (1 << 31) + 100003
    cuts = [0, (1 << 31) - 1, (1 << 31) + 500, n]
    x = torch.ones(n, dtype=torch.float32, device="cuda")
    for i, v in ((5, -2.0), ((1 << 31) + 777, -3.0), ((1 << 31) + 90000, -3.0)):
        x[i] = v
    recs, out = _sharded("argmin_f32", [x], cuts)
    assert [(_f32(r), _i64(r, 8)) for r in recs] == \
        [(-2.0, 5), (1.0, (1 << 31) - 1), (-3.0, (1 << 31) + 777)]
    assert (_f32(out), _i64(out, 8)) == (-3.0, (1 << 31) + 777)
    del x
    xi = torch.ones(n, dtype=torch.int32, device="cuda")
    planted = {7: -5, (1 << 31) - 2: 1 << 30, (1 << 31): -(1 << 30), n - 1: 12345}
    for i, v in planted.items():
        xi[i] = v

    def shard_sum(a, b):
        return (b - a) + sum(v - 1 for i, v in planted.items() if a <= i < b)

    recs, out = _sharded("sum_i32_i64", [xi], cuts)
    assert [_i64(r) for r in recs] == [shard_sum(a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert _i64(out) == shard_sum(0, n)
    del xi
    torch.cuda.empty_cache()
