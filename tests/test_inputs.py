"""Pins for the seeded input generator (shared by oracle checks and the bench)."""
import os

import numpy as np

from paper_1304_5553_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_sequence():
    want = [int(l) for l in open(os.path.join(GOLD, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert inputs.splitmix64_sequence(1234567, 5) == want


def test_counter_based_slices_agree():
    full = inputs.uniform_f32(1, 2, 300000, -2.0, 2.0)
    part = inputs.uniform_f32(1, 2, 1000, -2.0, 2.0, offset=123456)
    assert np.array_equal(full[123456:124456], part)
    ln = inputs.lognormal_signed_f32(1, 3, 200000)
    assert np.array_equal(ln[5000:6000], inputs.lognormal_signed_f32(1, 3, 1000, offset=5000))
    assert not np.array_equal(full[:1000], inputs.uniform_f32(1, 3, 1000, -2.0, 2.0))
    assert not np.array_equal(full[:1000], inputs.uniform_f32(2, 2, 1000, -2.0, 2.0))


def test_uniform_exact_grid_and_range():
    x = inputs.uniform_f32(0, 0, 1 << 18, -2.0, 2.0)
    assert x.min() >= -2.0 and x.max() < 2.0
    k = (x.astype(np.float64) + 2.0) * 2.0 ** 22  # 4*u - 2 with u = k * 2^-24
    assert np.array_equal(k, np.round(k))
    y = inputs.uniform_f32(0, 1, 1 << 18, -1.0, 1.0)
    assert y.min() >= -1.0 and y.max() < 1.0
    assert abs(float(y.mean())) < 0.01 and abs(float(y.var()) - 1 / 3) < 0.01


def test_lognormal_moments():
    x = inputs.lognormal_signed_f32(4, 0, 1 << 18, sigma=3.0)
    l = np.log(np.abs(x.astype(np.float64)))
    assert abs(l.mean()) < 0.05 and abs(l.std() - 3.0) < 0.05
    assert abs(float((x > 0).mean()) - 0.5) < 0.01


def test_int_and_lengths():
    v = inputs.int_uniform_i32(5, 0, 1 << 18)
    assert v.min() >= -(1 << 20) and v.max() <= (1 << 20)
    assert v.min() < -(1 << 20) + 100 and v.max() > (1 << 20) - 100
    lens = inputs.segment_lengths()
    assert lens.size == 20000 and lens.min() >= 1 and lens.max() <= 1 << 20
    assert 0.45 < float((lens <= 1024).mean()) < 0.55  # median near 2^10
    gaps = inputs.exponential_f64(6, 0, 100000, 20000.0)
    assert abs(gaps.mean() * 20000.0 - 1.0) < 0.02


def test_f16_values_round_to_nearest_even():
    # binary16 format facts: ties to even at 1 + 2^-11 and at 2^-25 (half the
    # smallest subnormal), the largest finite value 65504, overflow from 65520
    v = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -25, 3 * 2.0 ** -25, 65519.0, 65520.0],
                 np.float32)
    got = inputs.to_f16_values(v).astype(np.float64).tolist()
    assert got == [1.0, 1 + 2.0 ** -9, 0.0, 2.0 ** -23, 65504.0, float("inf")]
    x = inputs.uniform_f32(20, 0, 1000, -2.0, 2.0)
    h = inputs.to_f16_values(x)
    assert h.dtype == np.float16
    assert np.all(np.abs(h.astype(np.float64) - x) <= 2.0 ** -11 * np.abs(x) + 2.0 ** -25)
