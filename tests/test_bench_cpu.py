"""Host-side pieces of bench.py that need no GPU: the clock / throttle summary,
the peak lookup, and that the committed DRAM-traffic figure belongs to the
dominant kernel's current generated source."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return s


def test_clock_summary_median_and_reasons(tmp_path):
    rows = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1965, 2070, 1398.2, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = _sampler_with(tmp_path, rows).summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    rows.append("0, 1500, 2070, 800.0, 0x8, Active, Not Active, Active, Not Active")
    out = _sampler_with(tmp_path, rows).summary()
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(tmp_path):
    out = _sampler_with(tmp_path, ["garbage"]).summary()
    assert out["reasons"] == ["unavailable"] and out["sm_mhz"] is None


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6793.4}))
    assert bench.peaks() == (6793.4, "measured")


def test_committed_traffic_matches_the_current_kernel_source():
    # bench.py reports roofline.traffic only for the kernel source the ncu
    # capture was taken from; the committed figure must match today's source
    from paper_1304_5553_gb300 import pyc, stock
    dom = max(bench.MAP_BYTES, key=bench.MAP_BYTES.get)  # the 20-byte map dominates the step
    src = pyc.pyc_map_source(stock.create(dom))
    digest = hashlib.sha256(src.encode()).hexdigest()[:16]
    rows = [ln.split() for ln in open(os.path.join(ROOT, "profiles", "dram_traffic.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert any(r[0].startswith("pyc_map_%s_" % dom) and r[1] == digest for r in rows), \
        "profiles/dram_traffic.txt holds no capture of the current %s source" % dom
