"""Pins of the oracle's sharded reduction (shard_partial / combine_partials).

What fixes the answer independently of the oracle: the reduction of the whole
range (Sec. 3.2.5) -- each partition must reproduce it -- and plain numpy /
Python brute force on the whole array (np.argmin's first occurrence, Python's
exact int sum, math.fsum).  Planted mistakes (a shard index left local, ties
resolved towards the later shard, a dropped shard, a sum combined without
compensation) each fail one of the pins.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1304_5553_gb300 import inputs


def _arrays(kind, n, seed):
    if kind == "sum_i32_i64":
        return [inputs.int_uniform_i32(seed, 0, n)]
    if kind == "dot_f32":
        return [inputs.uniform_f32(seed, s, n, -1.0, 1.0) for s in range(2)]
    if kind in ("argmin_f32", "argmax_f32"):
        x = inputs.uniform_f32(seed, 0, n, -2.0, 2.0)
        # few distinct values, so that the extremum repeats across shards
        return [np.round(x * 2.0).astype(np.float32)]
    return [inputs.lognormal_signed_f32(seed, 0, n)]


def _brute(kind, arrays):
    x = arrays[0]
    if kind == "sum_i32_i64":
        return int(sum(int(v) for v in x))
    if kind == "max_f32":
        return float(np.max(x))
    if kind == "argmin_f32":
        i = int(np.argmin(x))
        return float(x[i]), i
    if kind == "argmax_f32":
        i = int(np.argmax(x))
        return float(x[i]), i
    if kind == "sum_f32":
        return math.fsum(float(v) for v in x)
    return math.fsum(float(a) * float(b) for a, b in zip(arrays[0], arrays[1]))


def _cuts(n, k, rng):
    c = sorted(int(v) for v in rng.integers(0, n + 1, size=k - 1))
    return [0] + c + [n]


def _sharded(kind, arrays, cuts, partial=oracle.shard_partial,
             combine=oracle.combine_partials):
    parts = [partial(kind, [a[cuts[r]:cuts[r + 1]] for a in arrays], cuts[r])
             for r in range(len(cuts) - 1)]
    return combine(kind, parts)


def _agrees(kind, got, arrays):
    want = _brute(kind, arrays)
    if kind in ("sum_f32", "dot_f32"):
        ab = sum(abs(float(a) * (float(arrays[1][j]) if kind == "dot_f32" else 1.0))
                 for j, a in enumerate(arrays[0]))
        return abs(got[0] - want) <= 2.0 ** -50 * ab + 1e-300
    return got == want


def _pins_pass(partial=oracle.shard_partial, combine=oracle.combine_partials):
    """All pins below as one predicate (used to check the planted mistakes)."""
    rng = np.random.default_rng(7)
    for kind in oracle.SHARD_KINDS:
        arrays = _arrays(kind, 3001, 11)
        for k in (1, 2, 3, 5):
            for _ in range(4):
                got = _sharded(kind, arrays, _cuts(3001, k, rng), partial, combine)
                if not _agrees(kind, got, arrays):
                    return False
    # a tie of the minimum on both sides of a cut: the first index wins
    x = np.array([3, 2, 1, 1, 2], np.float32)
    for kind, want in (("argmin_f32", (1.0, 2)), ("argmax_f32", (3.0, 0))):
        if _sharded(kind, [x], [0, 3, 5], partial, combine) != want:
            return False
    if _sharded("argmin_f32", [np.array([2, 2, 1, 1], np.float32)], [0, 3, 4], partial,
                combine) != (1.0, 2):
        return False
    return True


@pytest.mark.parametrize("kind", oracle.SHARD_KINDS)
def test_every_partition_reproduces_the_whole(kind):
    rng = np.random.default_rng(3)
    for n in (0, 1, 17, 3001):
        arrays = _arrays(kind, n, 5)
        whole = _brute(kind, arrays) if n else None
        for k in (1, 2, 3, 4, 7):
            for _ in range(6):
                got = _sharded(kind, arrays, _cuts(n, k, rng))
                if n == 0:
                    neutral = {"sum_i32_i64": 0, "max_f32": -math.inf,
                               "argmin_f32": (math.inf, 2 ** 63 - 1),
                               "argmax_f32": (-math.inf, 2 ** 63 - 1)}.get(kind, (0.0, 0.0))
                    assert got == neutral
                else:
                    assert _agrees(kind, got, arrays), (kind, n, k, got, whole)


def test_ties_straddling_a_cut_take_the_first_index():
    x = np.full(1000, 5.0, np.float32)
    x[[499, 500, 900]] = -1.0  # minima on both sides of the cut at 500
    assert _sharded("argmin_f32", [x], [0, 500, 1000]) == (-1.0, 499)
    assert _sharded("argmin_f32", [x], [0, 499, 1000]) == (-1.0, 499)
    assert _sharded("argmin_f32", [x], [0, 250, 500, 750, 1000]) == (-1.0, 499)
    y = np.full(1000, 5.0, np.float32)
    y[[600, 601]] = -1.0  # only in a later shard: its global index
    assert _sharded("argmin_f32", [y], [0, 500, 1000]) == (-1.0, 600)
    assert _sharded("argmin_f32", [y], [0, 0, 1000]) == (-1.0, 600)


def test_integer_sum_is_exact_past_2_to_31():
    x = np.full(5000, 2 ** 20, np.int32)
    assert _sharded("sum_i32_i64", [x], [0, 1234, 1234, 5000]) == 5000 * 2 ** 20


def test_sum_matches_exact_superaccumulator():
    x = inputs.lognormal_signed_f32(9, 0, 20000)
    s, ab = _sharded("sum_f32", [x], [0, 7000, 7001, 20000])
    assert abs(s - oracle.exact_sum_f32(x)) <= 2.0 ** -50 * ab


def test_pins_hold_for_the_oracle():
    assert _pins_pass()


def test_planted_mistakes_are_caught():
    def local_index(kind, arrays, i0):  # forgot to shift by i0
        return oracle.shard_partial(kind, arrays, 0)

    def later_wins_ties(kind, parts):
        if kind in ("argmin_f32", "argmax_f32"):
            sign = 1.0 if kind == "argmin_f32" else -1.0
            best = (sign * math.inf, 2 ** 63 - 1)
            for v, i in parts:
                if sign * v <= sign * best[0]:
                    best = (v, i)
            return best
        return oracle.combine_partials(kind, parts)

    def drops_last(kind, parts):
        return oracle.combine_partials(kind, parts[:-1] if len(parts) > 1 else parts)

    def plain_float_sum(kind, parts):
        if kind in ("sum_f32", "dot_f32"):
            s = np.float32(0)
            for p in parts:
                s = np.float32(s + np.float32(p[0]))
            return float(s), sum(p[1] for p in parts)
        return oracle.combine_partials(kind, parts)

    assert not _pins_pass(partial=local_index)
    assert not _pins_pass(combine=later_wins_ties)
    assert not _pins_pass(combine=drops_last)
    assert not _pins_pass(combine=plain_float_sum)
