"""Memory pool bookkeeping (Sec. 3.2.6), on the host pool kind (no GPU needed):
size classes, reuse, limits, statistics and thread safety."""
import threading

import numpy as np
import pytest

from paper_1304_5553_gb300 import pyc


def test_size_classes():
    assert pyc.pyc_pool_block_size(1) == 512 and pyc.pyc_pool_block_size(512) == 512
    prev = 512
    for b in list(range(513, 5000, 7)) + [2 ** k + d for k in range(12, 40) for d in (-1, 0, 1)]:
        c = pyc.pyc_pool_block_size(b)
        assert c >= b and (c - b) * 8 <= c, b          # at most 1/8 unused
        assert c >= prev or b < prev                    # monotone in the request
        e = (b - 1).bit_length() - 1
        assert c % (1 << (e - 3)) == 0                  # 8 classes per octave
        prev = c
    # the classes of one octave: 2^e * (1 + k/8)
    assert sorted({pyc.pyc_pool_block_size(b) for b in range(4097, 8193)}) == \
        [4096 + 512 * k for k in range(1, 9)]


def test_reuse_is_lifo_within_a_class():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_HOST)
    try:
        a, b, c = (pyc.pyc_pool_alloc(p, 3000) for _ in range(3))
        assert len({a, b, c}) == 3 and all(q % 256 == 0 for q in (a, b, c))
        pyc.pyc_pool_free(p, a)
        pyc.pyc_pool_free(p, b)
        assert pyc.pyc_pool_alloc(p, 2900) == b         # same class, most recent first
        assert pyc.pyc_pool_alloc(p, 3072) == a
        assert pyc.pyc_pool_alloc(p, 5000) not in (a, b, c)   # another class: new block
        st = pyc.pyc_pool_get_stats(p)
        assert st["hits"] == 2 and st["misses"] == 4 and st["retained_blocks"] == 0
    finally:
        pyc.pyc_pool_destroy(p)


def test_random_sequence_invariants():
    """A seeded random alloc/free sequence: live blocks never overlap, stats add up,
    and every request of a class that has a retained block reuses it."""
    rng = np.random.default_rng(70)
    p = pyc.pyc_pool_create(pyc.PYC_POOL_HOST)
    live = {}
    retained_by_class = {}
    try:
        for step in range(3000):
            if live and rng.random() < 0.45:
                q = list(live)[rng.integers(len(live))]
                size = live.pop(q)
                pyc.pyc_pool_free(p, q)
                retained_by_class.setdefault(size, 0)
                retained_by_class[size] += 1
            else:
                b = int(rng.choice([100, 700, 3000, 3100, 70000, 1 << 20]) * rng.uniform(0.9, 1.1))
                cls = pyc.pyc_pool_block_size(b)
                before = pyc.pyc_pool_get_stats(p)["hits"]
                q = pyc.pyc_pool_alloc(p, b)
                hit = pyc.pyc_pool_get_stats(p)["hits"] == before + 1
                assert hit == (retained_by_class.get(cls, 0) > 0)
                if hit:
                    retained_by_class[cls] -= 1
                live[q] = cls
            spans = sorted((q, q + s) for q, s in live.items())
            assert all(spans[k][1] <= spans[k + 1][0] for k in range(len(spans) - 1))
            st = pyc.pyc_pool_get_stats(p)
            assert st["live_blocks"] == len(live) and st["live_bytes"] == sum(live.values())
            assert st["system_bytes"] == st["live_bytes"] + st["retained_bytes"]
            assert st["hits"] + st["misses"] == st["system_allocs"] + st["hits"]
        pyc.pyc_pool_trim(p)
        st = pyc.pyc_pool_get_stats(p)
        assert st["retained_blocks"] == 0 and st["system_bytes"] == st["live_bytes"]
        assert st["system_allocs"] - st["system_frees"] == len(live)
    finally:
        pyc.pyc_pool_destroy(p)


def test_limits():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_HOST, max_bytes=10 * 4096, max_retained=2 * 4096)
    try:
        blocks = [pyc.pyc_pool_alloc(p, 4096) for _ in range(10)]
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_pool_alloc(p, 4096)
        assert e.value.status == pyc.PYC_E_NOMEM
        for q in blocks[:5]:
            pyc.pyc_pool_free(p, q)
        st = pyc.pyc_pool_get_stats(p)
        assert st["retained_bytes"] == 2 * 4096 and st["system_frees"] == 3   # max_retained
        # a request of another class: retained blocks are released to fit max_bytes
        q = pyc.pyc_pool_alloc(p, 8192)
        st = pyc.pyc_pool_get_stats(p)
        assert st["system_bytes"] <= 10 * 4096 and q not in blocks
    finally:
        pyc.pyc_pool_destroy(p)


def test_errors():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_HOST)
    try:
        for bad in (0, -5):
            with pytest.raises(pyc.PycError):
                pyc.pyc_pool_alloc(p, bad)
        q = pyc.pyc_pool_alloc(p, 10)
        pyc.pyc_pool_free(p, q)
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_pool_free(p, q)
        assert e.value.status == pyc.PYC_E_ARG
        pyc.pyc_pool_free(p, None)  # no-op
    finally:
        pyc.pyc_pool_destroy(p)
    with pytest.raises(pyc.PycError):
        pyc.pyc_pool_create(pyc.PYC_POOL_HOST, max_bytes=-1)


def test_threads():
    p = pyc.pyc_pool_create(pyc.PYC_POOL_HOST)
    errors = []

    def worker(seed):
        rng = np.random.default_rng(seed)
        mine = []
        try:
            for _ in range(2000):
                if mine and rng.random() < 0.5:
                    q, size = mine.pop(rng.integers(len(mine)))
                    pyc.pyc_pool_free(p, q)
                else:
                    size = int(rng.integers(1, 20000))
                    mine.append((pyc.pyc_pool_alloc(p, size), size))
            for q, _ in mine:
                pyc.pyc_pool_free(p, q)
        except Exception as ex:  # surfaced by the assertion below
            errors.append(ex)

    ts = [threading.Thread(target=worker, args=(s,)) for s in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    try:
        assert not errors
        st = pyc.pyc_pool_get_stats(p)
        assert st["live_blocks"] == 0 and st["retained_bytes"] == st["system_bytes"]
    finally:
        pyc.pyc_pool_destroy(p)
