"""Automatic tuning at first launch (environment variable PYC_AUTOTUNE=1, Sec.
3.3.1's automated tuning): a launch at an untuned size bucket tunes it after
running, the tuned configuration is persisted and used by the launches that
follow (in this process and, through the tuning cache, in the next), results
stay correct, and nothing is tuned inside a stream capture."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, os, sys
sys.path.insert(0, %r)
import numpy as np, torch
import oracle
from paper_1304_5553_gb300 import inputs, pyc
torch.cuda.set_device(0)
s = torch.cuda.current_stream().cuda_stream
tune = os.path.join(os.environ["PYC_CACHE_DIR"], "tune.jsonl")
lines = lambda: open(tune).read().splitlines() if os.path.exists(tune) else []
n = (1 << 20) + 5
x = inputs.uniform_f32(90, 0, n, -1.0, 1.0); y = inputs.uniform_f32(90, 1, n, -1.0, 1.0)
dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
out = {}
# a map-reduce: the first launch tunes its bucket
r = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i] + 0.25f", "float *x, float *y")
res = torch.zeros(1, dtype=torch.float32, device="cuda")
out["before"] = list(pyc.launch_config(r, n, reduce=True))
pyc.pyc_reduce_launch(r, n, [dx.data_ptr(), dy.data_ptr()], None, res.data_ptr(), s)
torch.cuda.synchronize()
out["records_after_first"] = len(lines())
out["after"] = list(pyc.launch_config(r, n, reduce=True))
pyc.pyc_reduce_launch(r, n, [dx.data_ptr(), dy.data_ptr()], None, res.data_ptr(), s)
torch.cuda.synchronize()
ref, ab = oracle.dot_f32(x, y)
out["err"] = abs(float(res.item()) - (ref + 0.25 * n)) / (ab + 0.25 * n)
out["records_after_second"] = len(lines())
# a map launched only inside a capture: nothing is tuned
m = pyc.pyc_map_create("float *x, float *y", "y[i] = x[i] * 1.5f - 2.0f")
gs = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=gs):
    pyc.pyc_map_launch(m, n, [dx.data_ptr(), dy.data_ptr()], None, gs.cuda_stream)
g.replay(); torch.cuda.synchronize()
out["map_ok"] = bool(torch.equal(dy, dx * 1.5 - 2.0))
out["records_after_capture"] = len(lines())
print(json.dumps(out))
"""


def _run(tmp_path, env_extra):
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path), **env_extra)
    p = subprocess.run([sys.executable, "-c", _CHILD % ROOT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_first_launch_tunes_the_bucket(tmp_path):
    r = _run(tmp_path, {"PYC_AUTOTUNE": "1"})
    assert r["records_after_first"] == 1            # the reduction's bucket, once
    assert r["records_after_second"] == 1           # tuned already: no second tuning
    assert r["err"] <= 8 * 2.0 ** -24
    assert r["map_ok"] and r["records_after_capture"] == 1  # no tuning inside a capture
    # a second process finds the tuned configuration in the cache and tunes nothing
    r2 = _run(tmp_path, {"PYC_AUTOTUNE": "1"})
    assert r2["before"] == r["after"] and r2["records_after_second"] == 1


def test_without_the_variable_nothing_is_tuned(tmp_path):
    r = _run(tmp_path, {"PYC_AUTOTUNE": "0"})
    assert r["records_after_second"] == 0 and r["before"] == r["after"]
