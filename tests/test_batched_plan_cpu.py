"""The segmented reducer's work plan, checked on the host (no GPU): every segment
becomes exactly one task, every chunk of a long task and every short task is
one work item's work exactly once, partial slots do not overlap, and each
task's vector head follows its arrays' alignment.  pyc_reduce_batched launches
the plan pyc_reduce_batched_plan returns."""
import numpy as np
import pytest

from paper_1304_5553_gb300 import inputs, pyc

SMALL = 2048  # segments up to this length are reduced by one warp
BASE_X, BASE_Y = 1 << 32, 3 << 32  # stand-in array addresses (never dereferenced)


@pytest.fixture(scope="module")
def dot():
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y")
    yield h
    pyc.pyc_reduce_destroy(h)


def _lengths():
    lens = inputs.segment_lengths(nseg=3000).astype(np.int64)
    # edge lengths: empty, one element, the one-warp limit and one past it, equal ties
    extra = np.array([0, 1, SMALL, SMALL + 1, 0, 70000, 70000, 1 << 20], np.int64)
    return np.concatenate([lens[:1500], extra, lens[1500:]])


def _plan(h, lens, shift_x=0, shift_y=0):
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ptrs = [BASE_X + 4 * shift_x, BASE_Y + 4 * shift_y]
    info, items, slots = pyc.batched_plan(h, off, ptrs)
    return off, info, items, slots


def test_tasks_are_a_permutation_short_first_then_longest_first(dot):
    lens = _lengths()
    _, info, _, _ = _plan(dot, lens)
    seg = info[:, 0]
    assert sorted(seg.tolist()) == list(range(lens.size))
    assert np.array_equal(info[:, 1], lens[seg])
    short = lens <= SMALL
    ns = int(short.sum())
    assert np.array_equal(seg[:ns], np.flatnonzero(short))  # input order
    long_seg = seg[ns:]
    long_len = lens[long_seg]
    assert np.all(np.diff(long_len) <= 0)  # longest first
    for v in np.unique(long_len):  # ties keep input order
        s = long_seg[long_len == v]
        assert np.all(np.diff(s) > 0)
    assert np.all(info[:ns, 4] == 0)


def test_items_cover_each_chunk_and_short_task_once(dot):
    lens = _lengths()
    _, info, items, _ = _plan(dot, lens, 3, 3)
    ns = int((lens <= SMALL).sum())
    block = pyc.batched_config(dot)[2]
    chunks = items[items[:, 1] >= 0]
    bundles = items[items[:, 1] < 0]
    # one-warp tasks: bundles of at most block/32 tasks partition [0, ns)
    assert np.all(bundles[:, 2] >= 1) and np.all(bundles[:, 2] <= block // 32)
    covered = np.zeros(ns, np.int64)
    for t, _, c, _ in bundles:
        covered[t:t + c] += 1
    assert np.all(covered == 1)
    # long tasks: chunks 0 .. nchunks-1 each exactly once, and they span the body
    assert np.all(chunks[:, 2] == 1)
    got = sorted(map(tuple, chunks[:, :2].tolist()))
    want = sorted((t, c) for t in range(ns, lens.size) for c in range(int(info[t, 4])))
    assert got == want
    for t in range(ns, lens.size):
        n, head, chunk, nch = (int(v) for v in info[t, 1:5])
        body = n - head if head >= 0 else n
        assert chunk > 0 and nch == -(-body // chunk)
        assert sum(min(chunk, body - c * chunk) for c in range(nch)) == body


def test_partial_slots_do_not_overlap(dot):
    lens = _lengths()
    _, info, _, slots = _plan(dot, lens)
    used = np.zeros(slots, np.int64)
    for t in range(lens.size):
        nch, s0 = int(info[t, 4]), int(info[t, 5])
        if nch > 1:
            used[s0:s0 + nch] += 1
    assert np.all(used == 1)
    assert slots == int(info[info[:, 4] > 1, 4].sum())


@pytest.mark.parametrize("shift_x,shift_y", [(0, 0), (1, 1), (5, 5), (0, 1), (2, 7)])
def test_head_follows_the_arrays_alignment(dot, shift_x, shift_y):
    lens = _lengths()
    off, info, _, _ = _plan(dot, lens, shift_x, shift_y)
    vec = pyc.batched_config(dot)[0]
    span = vec // 4
    for seg, n, head in info[:, :3]:
        ax = BASE_X + 4 * (shift_x + int(off[seg]))
        ay = BASE_Y + 4 * (shift_y + int(off[seg]))
        want = -1
        for k in range(span):  # the first shift that aligns both arrays
            if (ax + 4 * k) % vec == 0 and (ay + 4 * k) % vec == 0:
                want = k if k < n else -1
                break
        assert head == want, (seg, n, head, want)


def test_empty_table_and_argument_errors(dot):
    info, items, slots = pyc.batched_plan(dot, np.array([0], np.int64), [BASE_X, BASE_Y])
    assert info.shape == (0, 6) and items.shape == (0, 4) and slots == 0
    with pytest.raises(pyc.PycError) as e:
        pyc.batched_plan(dot, np.array([0, 5, 3], np.int64), [BASE_X, BASE_Y])
    assert e.value.status == pyc.PYC_E_ARG
    with pytest.raises(pyc.PycError) as e:
        pyc.batched_plan(dot, np.array([0, 5], np.int64), [0, BASE_Y])
    assert e.value.status == pyc.PYC_E_ARG
    # too small an item buffer is an error, not an overflow
    off = np.array([0, 100000], np.int64)
    assert pyc.load().pyc_reduce_batched_plan(
        dot, 1, off.ctypes.data, pyc._ptr_array([BASE_X, BASE_Y]), None, None,
        np.zeros(4, np.int32).ctypes.data, 0, None, None) == pyc.PYC_E_ARG
