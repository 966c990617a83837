"""Benchmark of the map / map-reduce path on GB300.

One step = the three elementwise maps at n = 2^28 (the headline workload):
  z = a*x + b*y in binary32, the same in bfloat16 storage, and the four-input
  z = x*exp(-y*y) + sin(u)*w in binary32; a = 2.5, b = -0.75, inputs
  uniform[-2, 2) from the seeded generator.
value = algorithmic HBM bytes of a step / device time of a step (GB/s); each
input is 0.5-1 GiB, far above the 129 MB L2, so no flush is needed.

Also measured (in "details"): the n = 2^28 reductions, the n = 2^20 dot
latency, and the 20,000-segment batched dot against per-segment launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs the same workload on its own GPU (independent
replicas, weak scaling); rank 0 prints one JSON line.  --impl reference times
the CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "achieved HBM GB/s (% of GB300 peak) for map/map-reduce; batched reqs/s with p50/p99 latency"
N_MAP = 1 << 28  # may be lowered by --n-log2 (profiling captures only)
A, B = 2.5, -0.75
MAP_BYTES = {"lin_comb_f32": 12, "lin_comb_bf16": 6, "gauss_sin_f32": 20}  # per element
WORKLOAD = ("maps n=2^28: z=a*x+b*y f32 + z=a*x+b*y bf16 storage + "
            "z=x*exp(-y*y)+sin(u)*w f32; a=2.5 b=-0.75; inputs uniform[-2,2) seeded")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm

def make_map_inputs(torch, dev, only=None, offset=0):
    """The maps' inputs: elements [offset, offset + N_MAP) of the seeded arrays
    (one rank's shard of arrays of world * N_MAP elements under torchrun)."""
    from paper_1304_5553_gb300 import inputs
    n = N_MAP
    want = set(only.split(",")) if only else set(MAP_BYTES)
    host = {}
    if want & {"lin_comb_f32", "lin_comb_bf16"}:
        x = inputs.uniform_f32(0, 0, n, -2.0, 2.0, offset=offset)
        y = inputs.uniform_f32(0, 1, n, -2.0, 2.0, offset=offset)
        if "lin_comb_f32" in want:
            host["lin_comb_f32"] = [x, y]
        if "lin_comb_bf16" in want:
            host["lin_comb_bf16"] = [inputs.to_bf16_values(x), inputs.to_bf16_values(y)]
    if "gauss_sin_f32" in want:
        host["gauss_sin_f32"] = [inputs.uniform_f32(1, s, n, -2.0, 2.0, offset=offset)
                                 for s in range(4)]
    d = {}
    for k, arrs in host.items():
        dt = torch.bfloat16 if k.endswith("bf16") else torch.float32
        ins = [torch.from_numpy(a).to(dt).to(dev) for a in arrs]
        d[k] = ins + [torch.empty(n, dtype=dt, device=dev)]
    return host, d


def map_launchers(torch, pyc, stock, d, stream):
    """name -> zero-argument launch of that map through the C ABI."""
    out = {}
    for k, bufs in d.items():
        h = stock.create(k)
        sc = pyc.pack_scalars(h, [A, B]) if k.startswith("lin_comb") else None
        ptrs = [b.data_ptr() for b in bufs]
        out[k] = (lambda h=h, ptrs=ptrs, sc=sc: pyc.pyc_map_launch(h, N_MAP, ptrs, sc, stream))
    return out


def time_steps(torch, launchers, names, steps, warmup, barrier):
    """Time `steps` steps (each: every named launch once), recording an event pair
    around every launch on the launching stream."""
    for _ in range(warmup):
        for k in names:
            launchers[k]()
    torch.cuda.synchronize()
    ev = {k: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)] for k in names}
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t0.record()
    for s in range(steps):
        for k in names:
            ev[k][s][0].record()
            launchers[k]()
            ev[k][s][1].record()
    t1.record()
    torch.cuda.synchronize()
    barrier()
    total_ms = t0.elapsed_time(t1)
    per = {k: [a.elapsed_time(b) for a, b in ev[k]] for k in names}
    return total_ms, per


def bench_e2e(torch, pyc, stock, host, dev, steps=3, warmup=1):
    """Same step through the C ABI with HOST buffers: pyc_map_launch_host on
    page-locked host arrays, inside the timed region.  The arrays are mapped into
    the device's address space, so each kernel loads its inputs from host memory
    and stores its output there over the chip-to-chip link (pageable arrays would
    be staged through device buffers instead); it returns when the output is in
    host memory."""
    pinned = {k: [torch.from_numpy(a).to(torch.bfloat16 if k.endswith("bf16") else torch.float32)
                  .pin_memory() for a in arrs] for k, arrs in host.items()}
    outs_h = {k: torch.empty(N_MAP, dtype=pinned[k][0].dtype).pin_memory() for k in pinned}
    handles = {k: stock.create(k) for k in pinned}
    scal = {k: pyc.pack_scalars(handles[k], [A, B]) if k.startswith("lin_comb") else None
            for k in pinned}
    ptrs = {k: [t.data_ptr() for t in pinned[k]] + [outs_h[k].data_ptr()] for k in pinned}
    h2d = sum(t.numel() * t.element_size() for p in pinned.values() for t in p)
    d2h = sum(t.numel() * t.element_size() for t in outs_h.values())

    def step():
        for k in pinned:
            pyc.pyc_map_launch_host(handles[k], N_MAP, ptrs[k], scal[k])

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    alg = sum(MAP_BYTES[k] for k in pinned) * N_MAP
    del pinned, outs_h
    return {"value": round(alg / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ms, 3),
            "steps": steps}


def bench_reductions(torch, pyc, stock, dev, reps=20):
    """n = 2^28 reductions and the n = 2^20 dot: mean device time over reps."""
    from paper_1304_5553_gb300 import inputs
    n = N_MAP
    res = {}
    s = torch.cuda.current_stream().cuda_stream
    ln = torch.from_numpy(inputs.lognormal_signed_f32(0, 0, n)).to(dev)
    xi = torch.from_numpy(inputs.int_uniform_i32(0, 0, n)).to(dev)
    xa = torch.from_numpy(inputs.argmin_with_minima(0, n)).to(dev)
    out = torch.zeros(2, dtype=torch.int64, device=dev)
    cases = [("sum_f32", ln, 4), ("sum_f32_comp", ln, 4), ("sum_i32_i64", xi, 4),
             ("max_f32", ln, 4), ("argmin_f32", xa, 4)]
    for name, arr, bpe in cases:
        h = stock.create(name)
        pyc.pyc_reduce_autotune(h, n, s)
        f = (lambda h=h, arr=arr: pyc.pyc_reduce_launch(h, n, [arr.data_ptr()], None,
                                                         out.data_ptr(), s))
        ms = _time_fn(torch, f, reps)
        res[name] = {"n": n, "us": round(ms * 1e3, 2), "GB/s": round(bpe * n / (ms * 1e-3) / 1e9, 1),
                     "config": "vec%d_u%d_b%d" % pyc.launch_config(h, n, reduce=True)}
    del ln, xi, xa
    # small dot: latency-bound (8 MiB fits in L2: warm timing)
    m = 1 << 20
    x = torch.from_numpy(inputs.uniform_f32(0, 0, m, -1.0, 1.0)).to(dev)
    y = torch.from_numpy(inputs.uniform_f32(0, 1, m, -1.0, 1.0)).to(dev)
    h = stock.create("dot_f32")
    pyc.pyc_reduce_autotune(h, m, s)
    f = lambda: pyc.pyc_reduce_launch(h, m, [x.data_ptr(), y.data_ptr()], None, out.data_ptr(), s)
    ms = _time_fn(torch, f, 200)
    # the same launch replayed from a CUDA graph of 100 launches (no per-launch
    # stream submission cost): the kernel's own latency
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gs):
        for _ in range(3):
            pyc.pyc_reduce_launch(h, m, [x.data_ptr(), y.data_ptr()], None, out.data_ptr(),
                                  gs.cuda_stream)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=gs):
        for _ in range(100):
            pyc.pyc_reduce_launch(h, m, [x.data_ptr(), y.data_ptr()], None, out.data_ptr(),
                                  gs.cuda_stream)
    ms_g = _time_fn(torch, g.replay, 20) / 100
    # cold: before each launch a 512 MiB write evicts x and y from L2 (and leaves
    # L2 full of dirty lines that the dot's misses must write back); the events
    # bracket the dot launch alone (median of 20).  Beside it, cold after a
    # 512 MiB read (L2 holds only clean lines of other data).
    # Beside them, the same measurement of a one-CTA map over 32 elements: what
    # any launch costs right after the flush (its code and launch state come
    # from DRAM too), the floor under the dot's cold time.
    flush = torch.empty(1 << 27, dtype=torch.float32, device=dev)
    tiny = pyc.pyc_map_create("float *x", "x[i] = 1.0f")
    tz = torch.empty(32, dtype=torch.float32, device=dev)
    ft = lambda: pyc.pyc_map_launch(tiny, 32, [tz.data_ptr()], None, s)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cold, clean, floor = [], [], []
    for r in range(69):
        k = r % 3
        if k == 1:
            flush.sum()
        else:
            flush.fill_(float(r))
        a.record()
        (ft if k == 2 else f)()
        b.record()
        torch.cuda.synchronize()
        if r >= 9:
            (cold, clean, floor)[k].append(a.elapsed_time(b))
    ms_c = statistics.median(cold)
    ms_cc = statistics.median(clean)
    ms_floor = statistics.median(floor)
    pyc.pyc_map_destroy(tiny)
    res["dot_f32_n2^20"] = {"n": m, "us": round(ms * 1e3, 2),
                            "GB/s": round(8 * m / (ms * 1e-3) / 1e9, 1), "cache": "warm (fits L2)",
                            "launches_per_s": round(1e3 / ms, 1),
                            "graph_us": round(ms_g * 1e3, 2),
                            "cold_us": round(ms_c * 1e3, 2),
                            "cold_GB/s": round(8 * m / (ms_c * 1e-3) / 1e9, 1),
                            "cold_after_read_flush_us": round(ms_cc * 1e3, 2),
                            "cold_launch_floor_us": round(ms_floor * 1e3, 2),
                            "config": "vec%d_u%d_b%d" % pyc.launch_config(h, m, reduce=True)}
    del g, flush
    return res


def bench_sharded_sum(torch, pyc, stock, dev, rank, world, dist, reps=10):
    """Compensated binary32 sum over world * 2^28 elements, each rank holding a
    2^28-element shard: shard record -> all-gather of 16-byte records (NCCL) ->
    combine.  Time of the whole step (max over ranks)."""
    from paper_1304_5553_gb300 import inputs
    from paper_1304_5553_gb300.shard import ShardedReduce
    n = N_MAP
    x = torch.from_numpy(inputs.lognormal_signed_f32(0, 0, n, offset=rank * n)).to(dev)
    out = torch.zeros(1, dtype=torch.float32, device=dev)
    h = stock.create("sum_f32_comp")
    sr = ShardedReduce(h, world * n, rank, world)
    assert (sr.i0, sr.n) == (rank * n, n)
    f = lambda: sr([x.data_ptr()], None, out.data_ptr())
    for _ in range(3):
        f()
    torch.cuda.synchronize()
    dist.barrier()
    ms = max_over_ranks(_time_fn(torch, f, reps), dist, dev)
    vals = [torch.zeros_like(out) for _ in range(world)]
    dist.all_gather(vals, out)
    same = all(float(v.item()) == float(out.item()) for v in vals)
    del x
    return {"n_total": world * n, "us": round(ms * 1e3, 2),
            "GB/s": round(4 * world * n / (ms * 1e-3) / 1e9, 1),
            "exchange": "all-gather of %d x 16 B" % world, "same_on_every_rank": same}


def bench_scans(torch, pyc, stock, dev, reps=10):
    """n = 2^28 prefix scans (Sec. 3.2.6), one single-pass launch each.  GB/s
    counts the algorithmic bytes: input read once, output written once (the
    kernel's second read of a tile is served by L2)."""
    from paper_1304_5553_gb300 import inputs
    n = N_MAP
    res = {}
    s = torch.cuda.current_stream().cuda_stream
    xf = torch.from_numpy(inputs.uniform_f32(0, 0, n, -1.0, 1.0)).to(dev)
    xi = torch.from_numpy(inputs.int_uniform_i32(0, 0, n)).to(dev)
    yf = torch.empty(n, dtype=torch.float32, device=dev)
    yi = torch.empty(n, dtype=torch.int64, device=dev)
    cases = [("cumsum_f32", xf, yf, 8), ("cummax_f32", xf, yf, 8),
             ("cumsum_excl_i32_i64", xi, yi, 12)]
    # the map with the same reads and writes per element and no dependence between
    # elements (a copy for the 4-byte scans, a widening copy for int32 -> int64):
    # the bandwidth this read/write mix reaches at all, beside the scan's
    mix = {}
    for spec in ("float *x, float *y", "int *x, long long *y"):
        hm = pyc.pyc_map_create(spec, "y[i] = x[i]")
        x, y = (xf, yf) if spec.startswith("float") else (xi, yi)
        pyc.pyc_map_autotune(hm, n, s)
        mix[spec] = _time_fn(torch, lambda hm=hm, x=x, y=y: pyc.pyc_map_launch(
            hm, n, [x.data_ptr(), y.data_ptr()], None, s), reps)
        pyc.pyc_map_destroy(hm)
    peak, kind = peaks()
    for name, x, y, bpe in cases:
        h = stock.create(name)
        pyc.pyc_scan_autotune(h, n, s)
        f = (lambda h=h, x=x, y=y: pyc.pyc_scan_launch(h, n, [x.data_ptr(), y.data_ptr()], None, s))
        ms = _time_fn(torch, f, reps)
        gbs = bpe * n / (ms * 1e-3) / 1e9
        mix_ms = mix["int *x, long long *y" if bpe == 12 else "float *x, float *y"]
        res[name] = {"n": n, "us": round(ms * 1e3, 2), "GB/s": round(gbs, 1),
                     "frac_of_%s_peak" % kind: round(gbs / peak, 4),
                     "bytes_per_elem": bpe,
                     "config": "vec%d_u%d_b%d" % pyc.launch_config(h, n, reduce="scan"),
                     "same_mix_map_us": round(mix_ms * 1e3, 2),
                     "frac_of_same_mix_map": round(mix_ms / ms, 4)}
    del xf, xi, yf, yi
    torch.cuda.empty_cache()
    return res


def bench_fused(torch, dev, reps=10):
    """GPUArray-style expressions at n = 2^28 (Sec. 3.2.4): fused into one kernel
    vs evaluated operator by operator (one kernel and one temporary per node).
    GB/s counts the fused pass's algorithmic bytes for both."""
    from paper_1304_5553_gb300 import gpuarray as ga
    from paper_1304_5553_gb300 import inputs
    n = N_MAP
    res = {}
    arrs = [torch.from_numpy(inputs.uniform_f32(1, s, n, -2.0, 2.0)).to(dev) for s in range(4)]
    X, Y, U, W = (ga.GArray(a) for a in arrs)
    out = ga.GArray(torch.empty(n, dtype=torch.float32, device=dev))
    cases = [("x*exp(-y*y)+sin(u)*w", lambda: X * ga.exp(-(Y * Y)) + ga.sin(U) * W, 20),
             ("2.5*x-0.75*y", lambda: 2.5 * X - 0.75 * Y, 12)]
    for name, build, bpe in cases:
        e = build()
        ga.autotune(e)
        ms_f = _time_fn(torch, lambda: ga.evaluate(e, out=out), reps)
        kernels = [0]

        def eager():
            r, k = ga.evaluate_eager(e)
            kernels[0] = k
        ms_e = _time_fn(torch, eager, 3, warmup=1)
        torch.cuda.empty_cache()
        res[name] = {"n": n, "fused_us": round(ms_f * 1e3, 1), "eager_us": round(ms_e * 1e3, 1),
                     "speedup": round(ms_e / ms_f, 2), "kernels_fused": 1,
                     "kernels_eager": kernels[0],
                     "fused_GB/s": round(bpe * n / (ms_f * 1e-3) / 1e9, 1)}
    del arrs, X, Y, U, W, out
    torch.cuda.empty_cache()
    return res


def bench_compile(pyc):
    """Spec to kernel (Sec. 2, Fig. 1; Sec. 3.3.2): host time of pyc_*_create for
    a spec never seen before (parse, generate, NVRTC compile for sm_103a, write
    the disk cache, load the module), for the same spec again in this process
    (parse, generate, hash, in-process hit), and in a fresh process whose
    context is already up (disk-cache hit)."""
    import subprocess
    import time
    import uuid
    tag = uuid.uuid4().int % 1000003  # a constant no earlier run compiled
    cases = {
        "map": ("pyc_map_create", "pyc_map_destroy",
                ("float a, float *x, float b, float *y, float *z",
                 "z[i] = a*x[i] + b*y[i] + %d.0f" % tag)),
        "reduce": ("pyc_reduce_create", "pyc_reduce_destroy",
                   (pyc.PYC_F32, "0", "a+b", "x[i]*y[i] + %d.0f" % tag, "float *x, float *y")),
    }
    res = {}
    for name, (fn, fd, args) in cases.items():
        f, destroy = getattr(pyc, fn), getattr(pyc, fd)
        t0 = time.perf_counter()
        h = f(*args)
        cold = time.perf_counter() - t0
        destroy(h)
        reps = 200
        warm = 0.0
        for _ in range(reps):
            t0 = time.perf_counter()
            h = f(*args)
            warm += time.perf_counter() - t0
            destroy(h)
        warm /= reps
        code = ("import sys, time; sys.path.insert(0, %r)\n"
                "from paper_1304_5553_gb300 import pyc\n"
                "pyc.pyc_map_create('float *x, float *y', 'y[i] = x[i]')\n"
                "t0 = time.perf_counter(); pyc.%s(*%r)\n"
                "print(time.perf_counter() - t0)\n" % (ROOT, fn, args))
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             timeout=600)
        disk = float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
        res[name] = {"cold_ms": round(cold * 1e3, 1), "warm_us": round(warm * 1e6, 1),
                     "disk_hit_ms": round(disk * 1e3, 2) if disk is not None else None}
    return res


def bench_pool(torch, pyc, dev):
    """Memory pools (Sec. 3.2.6): host time of one allocate + free pair served by
    a pool (reuse) vs by the driver (a pool that retains nothing) vs torch's own
    caching allocator; and operator-at-a-time evaluation of a 4-node expression
    at n = 2^20 with its temporaries from each."""
    import time
    from paper_1304_5553_gb300 import gpuarray as ga
    from paper_1304_5553_gb300 import inputs
    s = torch.cuda.current_stream().cuda_stream
    pool = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE)
    nopool = pyc.pyc_pool_create(pyc.PYC_POOL_DEVICE, max_retained=1)
    res = {}
    try:
        for label, nbytes in (("1MiB", 1 << 20), ("64MiB", 1 << 26)):
            row = {}
            for name, p in (("pool", pool), ("driver", nopool)):
                q = pyc.pyc_pool_alloc(p, nbytes, s)
                pyc.pyc_pool_free(p, q, s)
                reps = 2000 if name == "pool" else 200
                t0 = time.perf_counter()
                for _ in range(reps):
                    q = pyc.pyc_pool_alloc(p, nbytes, s)
                    pyc.pyc_pool_free(p, q, s)
                row[name + "_us"] = round((time.perf_counter() - t0) / reps * 1e6, 2)
            t0 = time.perf_counter()
            for _ in range(2000):
                t = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
                del t
            row["torch_us"] = round((time.perf_counter() - t0) / 2000 * 1e6, 2)
            res["alloc_free_" + label] = row
        n = 1 << 20
        x, y = (torch.from_numpy(inputs.uniform_f32(7, k, n)).to(dev) for k in range(2))
        X, Y = ga.GArray(x), ga.GArray(y)
        e = (X * Y + 2.5) * (X - Y)
        row = {}
        for name, p in (("pool", pool), ("driver", nopool), ("torch", None)):
            ga.set_pool(p)
            row[name + "_us"] = round(_time_fn(torch, lambda: ga.evaluate_eager(e), 50) * 1e3, 1)
        ga.set_pool(None)
        row["fused_us"] = round(_time_fn(torch, lambda: ga.evaluate(e), 50) * 1e3, 1)
        res["eager_4_kernels_n2^20"] = row
    finally:
        ga.set_pool(None)
        torch.cuda.synchronize()
        pyc.pyc_pool_destroy(pool)
        pyc.pyc_pool_destroy(nopool)
    return res


def bench_cg(torch, pyc, dev, nx=2048, iters=100):
    """Sparse (Sec. 3.2.6): the 5-point Laplacian on an nx x nx grid (4.19 M
    unknowns, 21 M nonzeros at nx = 2048).  SpMV GB/s over its algorithmic bytes
    (values + column indices + row pointers + x once + y); CG time per step over
    `iters` steps (rtol = 0), whose algorithmic bytes are one SpMV (p.q folded
    in) plus 9 vector passes (x and r update with r.r folded in: 6, p update: 3)."""
    from paper_1304_5553_gb300 import inputs
    s = torch.cuda.current_stream().cuda_stream
    res = {}
    n = nx * nx
    for name, vt, npdt, tdt in (("f32", pyc.PYC_F32, np.float32, torch.float32),
                                ("f64", pyc.PYC_F64, np.float64, torch.float64)):
        rp, c, v = inputs.poisson2d(nx, nx, npdt)
        d = [torch.from_numpy(a).to(dev) for a in (rp, c, v)]
        a = pyc.pyc_csr_create(n, n, c.size, *(t.data_ptr() for t in d), vt)
        try:
            vb = np.dtype(npdt).itemsize
            x = torch.from_numpy(np.random.default_rng(9).uniform(-1, 1, n).astype(npdt)).to(dev)
            y = torch.empty(n, dtype=tdt, device=dev)
            pyc.pyc_spmv_autotune(a, x.data_ptr(), y.data_ptr(), s)
            ms = _time_fn(torch, lambda: pyc.pyc_spmv(a, x.data_ptr(), y.data_ptr(), s), 20)
            spmv_bytes = c.size * (vb + 4) + (n + 1) * 8 + 2 * n * vb
            b = torch.ones(n, dtype=tdt, device=dev)
            xs = torch.zeros(n, dtype=tdt, device=dev)
            pyc.pyc_cg_solve(a, b.data_ptr(), xs.data_ptr(), 0.0, 8, s)   # warm-up
            xs.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = pyc.pyc_cg_solve(a, b.data_ptr(), xs.data_ptr(), 0.0, iters, s)
            e1.record()
            torch.cuda.synchronize()
            ms_cg = e0.elapsed_time(e1) / info["iterations"]
            step_bytes = spmv_bytes + 9 * n * vb
            res[name] = {"n": n, "nnz": int(c.size), "spmv_us": round(ms * 1e3, 1),
                         "spmv_GB/s": round(spmv_bytes / (ms * 1e-3) / 1e9, 1),
                         "lanes_per_row": pyc.pyc_csr_width(a),
                         "cg_steps": info["iterations"], "cg_us_per_step": round(ms_cg * 1e3, 1),
                         "cg_GB/s": round(step_bytes / (ms_cg * 1e-3) / 1e9, 1),
                         "cg_residual": info["residual"]}
        finally:
            torch.cuda.synchronize()
            pyc.pyc_csr_destroy(a)
        del d, x, y, b, xs
        torch.cuda.empty_cache()
    return res


def _time_fn(torch, f, reps, warmup=3):
    for _ in range(warmup):
        f()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        f()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def bench_batched(torch, pyc, stock, dev, reps=5):
    """20,000 segments, lengths log-uniform in [1, 2^20], dot per segment: one
    persistent launch (graph replay) vs one launch per segment."""
    from paper_1304_5553_gb300 import inputs
    lens = inputs.segment_lengths()
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(off[-1])
    res = {"segments": int(lens.size), "elements": total}
    s = torch.cuda.current_stream().cuda_stream
    for name, dt, bpe in (("dot_f32", torch.float32, 8), ("dot_bf16", torch.bfloat16, 4)):
        x = torch.from_numpy(inputs.uniform_f32(2, 0, total, -1.0, 1.0)).to(dt).to(dev)
        y = torch.from_numpy(inputs.uniform_f32(2, 1, total, -1.0, 1.0)).to(dt).to(dev)
        out = torch.zeros(lens.size, dtype=torch.float32, device=dev)
        h = stock.create(name)
        ptrs = [x.data_ptr(), y.data_ptr()]
        pyc.pyc_reduce_batched_autotune(h, lens.size, off, ptrs, None, out.data_ptr(), s)
        fb = lambda: pyc.pyc_reduce_batched(h, lens.size, off, ptrs, None, out.data_ptr(), s)
        ms_b = _time_fn(torch, fb, reps)

        def per_seg():
            es = x.element_size()
            for k in range(lens.size):
                pyc.pyc_reduce_launch(h, int(lens[k]), [x.data_ptr() + int(off[k]) * es,
                                                       y.data_ptr() + int(off[k]) * es],
                                      None, out.data_ptr() + 4 * k, s)
        ms_p = _time_fn(torch, per_seg, 1, warmup=1)
        res[name] = {"config": pyc.batched_config_name(h),
                     "batched_ms": round(ms_b, 3), "per_segment_launches_ms": round(ms_p, 3),
                     "speedup": round(ms_p / ms_b, 2),
                     "batched_GB/s": round(bpe * total / (ms_b * 1e-3) / 1e9, 1),
                     "reqs/s": round(lens.size / (ms_b * 1e-3), 1)}
        del x, y
        torch.cuda.empty_cache()
    return res


def serving_trace(torch, pyc, stock, dev, nreq=50000, rate=20000.0):
    """The request trace: Poisson arrivals (mean `rate`/s), 60% map-reduce (dot) /
    40% map (a*x+b*y), dtype uniform over {f32, bf16, i32}, sizes log-uniform in
    [2^10, 2^26], inputs at random offsets of resident pools.  Returns (table,
    arrival times in ns, algorithmic bytes, pools)."""
    from paper_1304_5553_gb300 import inputs
    P = 1 << 26
    x = inputs.uniform_f32(4, 0, P, -1.0, 1.0)
    y = inputs.uniform_f32(4, 1, P, -1.0, 1.0)
    pools = {
        "f32": (torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)),
        "bf16": (torch.from_numpy(x).to(torch.bfloat16).to(dev),
                 torch.from_numpy(y).to(torch.bfloat16).to(dev)),
        "i32": (torch.from_numpy(inputs.int_uniform_i32(4, 2, P)).to(dev),
                torch.from_numpy(inputs.int_uniform_i32(4, 3, P)).to(dev)),
    }
    del x, y
    maps = {"f32": "lin_comb_f32", "bf16": "lin_comb_bf16", "i32": "lin_comb_i32"}
    reds = {"f32": "dot_f32", "bf16": "dot_bf16", "i32": "dot_i32_i64"}
    scal = {k: bytes(pyc.pack_scalars(stock.create(v), [3, -2] if k == "i32" else [2.5, -0.75]))
            for k, v in maps.items()}
    u_kind = inputs.unit_f64(5, 0, nreq)
    u_dt = inputs.unit_f64(5, 1, nreq)
    sizes = inputs.loguniform_i64(5, 2, nreq, 10.0, 16.0, 1 << 10, 1 << 26)
    u_off = inputs.unit_f64(5, 3, nreq)
    arrival = np.cumsum(inputs.exponential_f64(5, 4, nreq, rate) * 1e9).astype(np.int64)
    table = pyc.RequestTable(nreq)
    dts = ["f32", "bf16", "i32"]
    total_bytes = 0
    for k in range(nreq):
        dt = dts[min(2, int(u_dt[k] * 3))]
        n = int(sizes[k])
        off = int(u_off[k] * (P - n + 1))
        a, b = pools[dt]
        es = a.element_size()
        ptrs = [a.data_ptr() + off * es, b.data_ptr() + off * es]
        if u_kind[k] < 0.6:
            table.set(k, pyc.PYC_REQ_REDUCE, stock.create(reds[dt]), n, ptrs)
            total_bytes += 2 * es * n
        else:
            table.set(k, pyc.PYC_REQ_MAP, stock.create(maps[dt]), n, ptrs + [0], scal[dt])
            total_bytes += 3 * es * n
    return table, arrival, total_bytes, pools


def bench_serving(torch, pyc, stock, dev, nreq=50000, rate=20000.0, budget=40 << 30):
    """The request trace (`serving_trace`) with a 40 GB admission cap.  Open loop
    (arrivals as drawn) and closed loop (all queued at t=0), through the serving
    loop and as one plain launch per request."""
    table, arrival, total_bytes, pools = serving_trace(torch, pyc, stock, dev, nreq, rate)
    srv = pyc.pyc_server_create(budget)
    out = {"requests": nreq, "rate_per_s": rate, "budget_bytes": budget,
           "algorithmic_bytes": total_bytes}
    try:
        # warm: every handle's batched and single kernels loaded
        pyc.pyc_server_replay(srv, table, None, pyc.PYC_REPLAY_SERVER)
        for label, arr in (("open_loop", arrival), ("closed_loop", None)):
            for mode, mname in ((pyc.PYC_REPLAY_SERVER, "server"), (pyc.PYC_REPLAY_DIRECT, "direct")):
                res = pyc.pyc_server_replay(srv, table, arr, mode)
                ok = sum(1 for r in res if r.status == pyc.PYC_OK)
                sub_t = np.array([r.t_submit_ns for r in res], np.int64)
                done_t = np.array([r.t_done_ns for r in res], np.int64)
                lat = (done_t - sub_t) / 1e3
                span = (done_t.max() - sub_t.min()) / 1e9
                bs = np.array([r.batch_size for r in res])
                out["%s_%s" % (label, mname)] = {
                    "ok": ok, "p50_us": round(float(np.percentile(lat, 50)), 1),
                    "p99_us": round(float(np.percentile(lat, 99)), 1),
                    "reqs_per_s": round(nreq / span, 1),
                    "GB/s": round(total_bytes / span / 1e9, 1),
                    "mean_batch": round(float(bs.mean()), 2)}
                if mode == pyc.PYC_REPLAY_SERVER and arr is not None:
                    # where an open-loop request's time goes (medians): arrival ->
                    # admitted, admitted -> its batch enqueued (work list, launch),
                    # enqueued -> completion seen by the scheduler
                    adm_t = np.array([r.t_admit_ns for r in res], np.int64)
                    lau_t = np.array([r.t_launch_ns for r in res], np.int64)
                    med = lambda v: round(float(np.percentile(v / 1e3, 50)), 1)
                    out["%s_%s" % (label, mname)]["stages_p50_us"] = {
                        "queued": med(adm_t - sub_t), "batched_and_launched": med(lau_t - adm_t),
                        "on_device_until_seen": med(done_t - lau_t)}
        st = pyc.pyc_server_get_stats(srv)
        out["peak_admitted_bytes"] = st["peak_admitted_bytes"]
        c = out["closed_loop_server"]["reqs_per_s"] / out["closed_loop_direct"]["reqs_per_s"]
        out["closed_loop_throughput_vs_direct"] = round(c, 2)
    finally:
        pyc.pyc_server_destroy(srv)
    del pools
    torch.cuda.empty_cache()
    return out


def oracle_map_step(n_sample):
    """The three maps' inputs over n_sample elements, generated once, and a
    function that runs the oracle (single-threaded C) over them once and returns
    the seconds it took."""
    import oracle
    from paper_1304_5553_gb300 import inputs
    x = inputs.uniform_f32(0, 0, n_sample, -2.0, 2.0)
    y = inputs.uniform_f32(0, 1, n_sample, -2.0, 2.0)
    bx, by = inputs.to_bf16_values(x), inputs.to_bf16_values(y)
    g = [inputs.uniform_f32(1, s, n_sample, -2.0, 2.0) for s in range(4)]
    oracle.map_lin_comb(A, x[:16], B, y[:16])  # load the library outside the timing

    def step():
        t = time.perf_counter()
        oracle.map_lin_comb(A, x, B, y)
        oracle.map_lin_comb(A, bx, B, by, out_bf16=True)
        oracle.map_gauss_sin(*g)
        return time.perf_counter() - t
    return step


def cpu_oracle_maps(n_sample, steps=1):
    """The oracle on the three maps over n_sample elements: (GB/s, seconds per pass)."""
    step = oracle_map_step(n_sample)
    sec = sum(step() for _ in range(steps)) / steps
    alg = sum(MAP_BYTES.values()) * n_sample
    return alg / sec / 1e9, sec


def max_over_ranks(value, dist=None, device=None):
    """The largest value over all ranks (the slowest replica's step time); the
    value itself without a process group."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(step_bytes_per_rank, world, ms_step):
    """Whole-job throughput: every rank's bytes over the slowest rank's step time."""
    return world * step_bytes_per_rank / (ms_step * 1e-3) / 1e9


def kernel_name(pyc, stock, name):
    h = stock.create(name)
    v, u, b = pyc.launch_config(h, N_MAP)
    return "pyc_map_%s_v%d_u%d" % (name, v, u)


def measured_traffic(pyc, stock, name, n):
    """DRAM bytes (read + write) per launch of this kernel from the committed ncu
    summary profiles/dram_traffic.txt, scaled to n elements; None when no
    capture exists for the kernel as currently generated (source digest)."""
    import hashlib
    kname = kernel_name(pyc, stock, name)
    digest = hashlib.sha256(pyc.pyc_map_source(stock.create(name)).encode()).hexdigest()[:16]
    try:
        for line in open(os.path.join(ROOT, "profiles", "dram_traffic.txt")):
            f = line.split("#")[0].split()
            if len(f) >= 3 and f[0] == kname and f[1] == digest:
                return round(float(f[2]) * n)
    except OSError:
        pass
    return None


def profile_reduce(args):
    """Profiling driver (not a bench line): one stock reduction at n = 2^n_log2,
    warm-up then `steps` launches, for ncu captures of a single kernel."""
    import torch
    from paper_1304_5553_gb300 import inputs, pyc, stock
    torch.cuda.set_device(0)
    n = N_MAP
    name = args.profile_reduce
    if name.startswith("sum_i32"):
        arr = [inputs.int_uniform_i32(0, 0, n)]
    elif name.startswith("argmin"):
        arr = [inputs.argmin_with_minima(0, n)]
    elif name.startswith("dot"):
        arr = [inputs.uniform_f32(0, s, n, -1.0, 1.0) for s in range(2)]
        if name.endswith("bf16"):
            arr = [torch.from_numpy(a).to(torch.bfloat16) for a in arr]
    else:
        arr = [inputs.lognormal_signed_f32(0, 0, n)]
    d = [(a if isinstance(a, torch.Tensor) else torch.from_numpy(a)).cuda() for a in arr]
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    h = stock.create(name)
    s = torch.cuda.current_stream().cuda_stream
    if args.autotune == "on":
        pyc.pyc_reduce_autotune(h, n, s)
    print("config vec%d_u%d_b%d" % pyc.launch_config(h, n, reduce=True), file=sys.stderr)
    f = lambda: pyc.pyc_reduce_launch(h, n, [t.data_ptr() for t in d], None, out.data_ptr(), s)
    ms = _time_fn(torch, f, args.steps, warmup=args.warmup)
    print(json.dumps({"profile_reduce": name, "n": n, "us": round(ms * 1e3, 2),
                      "note": "profiling driver, not a bench value"}))


def profile_scan(args):
    """Profiling driver (not a bench line): one stock scan at n = 2^n_log2,
    warm-up then `steps` launches, for ncu captures of a single kernel."""
    import torch
    from paper_1304_5553_gb300 import inputs, pyc, stock
    torch.cuda.set_device(0)
    n = N_MAP
    name = args.profile_scan
    if "i32" in name:
        x = torch.from_numpy(inputs.int_uniform_i32(0, 0, n)).cuda()
        y = torch.empty(n, dtype=torch.int64, device="cuda")
    else:
        x = torch.from_numpy(inputs.uniform_f32(0, 0, n, -1.0, 1.0)).cuda()
        y = torch.empty(n, dtype=torch.float32, device="cuda")
    opts = {}
    if args.config:  # vecV_uU_bB: a fixed launch configuration (no tuning launches)
        v, u, b = (int(q[1:] if q[0] in "ub" else q[3:]) for q in args.config.split("_"))
        opts = dict(vec_bytes=v, items_per_thread=u, block=b)
    if args.scan_op:  # the stock spec with its operation written another way
        dt, neu, _, inp, out, spec = stock.SCANS[name]
        h = pyc.pyc_scan_create(dt, neu, args.scan_op, inp, out, spec, opts or None)
    else:
        h = stock.create(name, **opts)
    s = torch.cuda.current_stream().cuda_stream
    if args.autotune == "on" and not opts:
        pyc.pyc_scan_autotune(h, n, s)
    print("config vec%d_u%d_b%d" % pyc.launch_config(h, n, reduce="scan"), file=sys.stderr)
    f = lambda: pyc.pyc_scan_launch(h, n, [x.data_ptr(), y.data_ptr()], None, s)
    ms = _time_fn(torch, f, args.steps, warmup=args.warmup)
    pyc.pyc_scan_sync(h, s)
    print(json.dumps({"profile_scan": name, "n": n, "us": round(ms * 1e3, 2),
                      "note": "profiling driver, not a bench value"}))


def profile_batched(args):
    """Profiling driver (not a bench line): the segmented dot product over the
    first `segments` segments of the bench's segment table (lengths log-uniform in
    [1, 2^20]), warm-up then `steps` batched launches, for ncu captures of the
    persistent segmented kernel."""
    import torch
    from paper_1304_5553_gb300 import inputs, pyc, stock
    torch.cuda.set_device(0)
    name = args.profile_batched
    dt = torch.bfloat16 if name.endswith("bf16") else torch.float32
    lens = inputs.segment_lengths(nseg=args.segments)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(off[-1])
    x = torch.from_numpy(inputs.uniform_f32(2, 0, total, -1.0, 1.0)).to(dt).cuda()
    y = torch.from_numpy(inputs.uniform_f32(2, 1, total, -1.0, 1.0)).to(dt).cuda()
    out = torch.zeros(lens.size, dtype=torch.float32, device="cuda")
    opts = {}
    if args.config:  # vecV_uU_bB: a fixed launch configuration (no tuning launches)
        v, u, b = (int(q[1:] if q[0] in "ub" else q[3:]) for q in args.config.split("_"))
        opts = dict(vec_bytes=v, items_per_thread=u, block=b)
    h = stock.create(name, **opts)
    s = torch.cuda.current_stream().cuda_stream
    ptrs = [x.data_ptr(), y.data_ptr()]
    if args.autotune == "on" and not opts:
        pyc.pyc_reduce_batched_autotune(h, lens.size, off, ptrs, None, out.data_ptr(), s)
    print("config " + pyc.batched_config_name(h), file=sys.stderr)
    f = lambda: pyc.pyc_reduce_batched(h, lens.size, off, ptrs, None, out.data_ptr(), s)
    ms = _time_fn(torch, f, args.steps, warmup=args.warmup)
    bpe = x.element_size() * 2
    print(json.dumps({"profile_batched": name, "segments": int(lens.size), "elements": total,
                      "us": round(ms * 1e3, 2), "GB/s": round(bpe * total / (ms * 1e-3) / 1e9, 1),
                      "note": "profiling driver, not a bench value"}))


def profile_serving(args):
    """Profiling driver (not a bench line): the first `requests` requests of the
    serving trace, replayed closed loop (all queued at t = 0) through the serving
    loop: one warm-up replay, then `steps` replays, for an ncu launch list."""
    import torch
    from paper_1304_5553_gb300 import pyc, stock
    torch.cuda.set_device(0)
    dev = torch.device("cuda")
    table, _, total_bytes, pools = serving_trace(torch, pyc, stock, dev, args.requests)
    srv = pyc.pyc_server_create(40 << 30)
    try:
        pyc.pyc_server_replay(srv, table, None, pyc.PYC_REPLAY_SERVER)
        spans = []
        for _ in range(args.steps):
            res = pyc.pyc_server_replay(srv, table, None, pyc.PYC_REPLAY_SERVER)
            assert all(r.status == pyc.PYC_OK for r in res)
            spans.append((max(r.t_done_ns for r in res) - min(r.t_submit_ns for r in res)) / 1e9)
    finally:
        pyc.pyc_server_destroy(srv)
    span = statistics.median(spans)
    print(json.dumps({"profile_serving": args.requests, "closed_loop_reqs_per_s":
                      round(args.requests / span, 1), "GB/s": round(total_bytes / span / 1e9, 1),
                      "note": "profiling driver, not a bench value"}))
    del pools


def profile_cg(args):
    """Profiling driver (not a bench line): CG on the 5-point Laplacian of an
    nx x nx grid (binary32), a warm-up solve of 8 steps, then `steps` steps."""
    import torch
    from paper_1304_5553_gb300 import inputs, pyc
    torch.cuda.set_device(0)
    nx = 1 << (args.n_log2 // 2)
    n = nx * nx
    rp, c, v = inputs.poisson2d(nx, nx, np.float32)
    d = [torch.from_numpy(a).cuda() for a in (rp, c, v)]
    a = pyc.pyc_csr_create(n, n, c.size, *(t.data_ptr() for t in d), pyc.PYC_F32)
    s = torch.cuda.current_stream().cuda_stream
    b = torch.ones(n, dtype=torch.float32, device="cuda")
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    if args.lanes is not None:  # a fixed width (no tuning launches)
        pyc.pyc_csr_set_width(a, args.lanes)
    elif args.autotune == "on":  # as the bench: time the lanes per row first
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        pyc.pyc_spmv_autotune(a, b.data_ptr(), y.data_ptr(), s)
    pyc.pyc_cg_solve(a, b.data_ptr(), x.data_ptr(), 0.0, 8, s)
    x.zero_()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    info = pyc.pyc_cg_solve(a, b.data_ptr(), x.data_ptr(), 0.0, args.steps, s)
    t1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_cg": "poisson2d %dx%d f32" % (nx, nx), "nnz": int(c.size),
                      "lanes_per_row": pyc.pyc_csr_width(a), "steps": info["iterations"],
                      "us_per_step": round(t0.elapsed_time(t1) * 1e3 / max(1, info["iterations"]), 1),
                      "note": "profiling driver, not a bench value"}))
    pyc.pyc_csr_destroy(a)


def run_gpu(args):
    import torch
    from paper_1304_5553_gb300 import pyc, stock

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(args.dist_backend)
    # one GPU per rank; ranks beyond the visible GPUs share them (a smoke run of
    # the multi-rank path with --dist-backend gloo: no kernel waits on another rank)
    local %= torch.cuda.device_count()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()

    stock.compile_all()
    # each rank holds its own shard of the maps' arrays (world * 2^28 elements)
    host, d = make_map_inputs(torch, dev, args.only, offset=rank * N_MAP)
    stream = torch.cuda.current_stream().cuda_stream
    launch = map_launchers(torch, pyc, stock, d, stream)
    if args.autotune == "on":
        for k in launch:
            pyc.pyc_map_autotune(stock.create(k), N_MAP, stream)
    torch.cuda.synchronize()

    # CPU baseline first (rank 0, N = 1 only): the oracle on a bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_s = N_MAP
        gbs, sec = cpu_oracle_maps(n_s, steps=2)
        cpu = {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "the three maps over the same 2^%d-element inputs, twice "
                         "(%.1f s per pass on one host core)" % (n_s.bit_length() - 1, sec)}

    names = [k for k in MAP_BYTES if not args.only or k in args.only.split(",")]
    with ClockSampler(local) as clk:
        total_ms, per = time_steps(torch, launch, names, args.steps, args.warmup, barrier)
    clocks = clk.summary()
    ms_step = max_over_ranks(total_ms / args.steps, dist, dev)
    step_bytes = sum(MAP_BYTES[k] for k in names) * N_MAP
    if args.n_log2 != 28 or args.only:
        print("note: reduced profiling configuration, not a bench value", file=sys.stderr)
    value = whole_job_gbs(step_bytes, world, ms_step)
    peak, peak_kind = peaks()
    avg = {k: statistics.mean(v) for k, v in per.items()}
    dom = max(avg, key=lambda k: avg[k])
    ach = MAP_BYTES[dom] * N_MAP / (avg[dom] * 1e-3) / 1e9
    kernels = {k: {"avg_us": round(avg[k] * 1e3, 2),
                   "GB/s": round(MAP_BYTES[k] * N_MAP / (avg[k] * 1e-3) / 1e9, 1),
                   "frac_of_%s_peak" % peak_kind: round(MAP_BYTES[k] * N_MAP / (avg[k] * 1e-3) / 1e9 / peak, 4)}
               for k in names}

    details = {"maps": kernels}
    if world > 1:
        details["sharded_sum"] = bench_sharded_sum(torch, pyc, stock, dev, rank, world, dist)
    e2e = None
    if rank == 0 and not args.quick:
        details["reductions"] = bench_reductions(torch, pyc, stock, dev)
        details["scans"] = bench_scans(torch, pyc, stock, dev)
        details["fused"] = bench_fused(torch, dev)
        details["pool"] = bench_pool(torch, pyc, dev)
        details["compile"] = bench_compile(pyc)
        details["cg"] = bench_cg(torch, pyc, dev)
        details["batched"] = bench_batched(torch, pyc, stock, dev)
        details["serving"] = bench_serving(torch, pyc, stock, dev)
    if not args.quick:
        del d, launch
        torch.cuda.empty_cache()
        e2e = bench_e2e(torch, pyc, stock, host, dev)
        e2e["value"] = round(e2e["value"] * world, 2)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic (seeded uniform[-2,2))",
            "config": {"workload": WORKLOAD, "n": N_MAP, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": ("sharded: rank r holds elements [r n, (r + 1) n) of "
                                       "arrays of %d n" % world) if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4),
                         "traffic": measured_traffic(pyc, stock, dom, N_MAP),
                         "kernel": "%s (%s)" % (kernel_name(pyc, stock, dom), dom),
                         "peak_kind": peak_kind},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": len(names) * args.steps,
            "clocks": clocks, "details": details,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm

def run_reference(args, budget_s=170.0):
    """The reference arm: the oracle on the host cores (rank 0 only) over the same
    three maps.  Warm-up steps run at 2^20 elements; the timed steps run at the
    bench's 2^28 whenever `steps` of them fit in about budget_s seconds (the
    per-element cost measured in the warm-up), else at the largest power of two
    that does."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    warm = oracle_map_step(1 << 20)
    per_elem = min(warm() for _ in range(max(1, args.warmup))) / (1 << 20)
    n_s = N_MAP
    while n_s > (1 << 20) and per_elem * n_s * args.steps > budget_s:
        n_s //= 2
    step = oracle_map_step(n_s)
    t = time.perf_counter()
    secs = [step() for _ in range(args.steps)]
    total = sum(secs)
    alg = sum(MAP_BYTES.values()) * n_s
    value = alg * args.steps / total / 1e9
    full = n_s == N_MAP
    config = {"workload": WORKLOAD, "n": N_MAP, "l2": "inputs larger than L2 (no flush)",
              "parallelism": "single GPU"}
    if not full:
        config["sample_per_step"] = n_s
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded uniform[-2,2))",
        "config": config,
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "each timed step: the three maps over 2^%d elements of the "
                                   "same inputs (%s; binary64 oracle, one host core; warm-up "
                                   "steps at 2^20)" % (n_s.bit_length() - 1,
                                                       "the full workload" if full else
                                                       "a sample, to bound the run")},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - t, 2),
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pyc", choices=["pyc", "reference"])
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="process group of a torchrun launch (gloo: several ranks may "
                         "share one GPU, for a smoke run of the multi-rank path)")
    ap.add_argument("--quick", action="store_true", help="maps only (no details, no e2e)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--only", default="", help="comma-separated subset of the maps (profiling)")
    ap.add_argument("--n-log2", type=int, default=28, help="map size (profiling captures only)")
    ap.add_argument("--profile-reduce", default="",
                    help="profiling driver: time one stock reduction only (not a bench line)")
    ap.add_argument("--profile-scan", default="",
                    help="profiling driver: time one stock scan only (not a bench line)")
    ap.add_argument("--scan-op", default="",
                    help="with --profile-scan: the stock scan with this operation instead")
    ap.add_argument("--profile-batched", default="",
                    help="profiling driver: the segmented dot (dot_f32 / dot_bf16) only")
    ap.add_argument("--segments", type=int, default=20000,
                    help="with --profile-batched: the first K segments of the segment table")
    ap.add_argument("--profile-serving", action="store_true",
                    help="profiling driver: closed-loop replays of the serving trace's first requests")
    ap.add_argument("--requests", type=int, default=50000,
                    help="with --profile-serving: the first K requests of the trace")
    ap.add_argument("--profile-cg", action="store_true",
                    help="profiling driver: CG steps on a Poisson matrix of 2^n_log2 rows")
    ap.add_argument("--lanes", type=int, default=None,
                    help="with --profile-cg: fixed width (0: rows in chunks of 32; "
                         "else lanes per row 1, 2, ..., 32)")
    ap.add_argument("--config", default="",
                    help="with --profile-scan: fixed launch configuration, e.g. vec32_u4_b512")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="off: use the tuning cache / defaults without timing candidates")
    args = ap.parse_args()
    global N_MAP
    N_MAP = 1 << args.n_log2
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_reduce:
        profile_reduce(args)
    elif args.profile_scan:
        profile_scan(args)
    elif args.profile_batched:
        profile_batched(args)
    elif args.profile_serving:
        profile_serving(args)
    elif args.profile_cg:
        profile_cg(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
