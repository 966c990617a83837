"""C-ABI checks that need no GPU: the library loads and exports every symbol
include/pyc.h declares; arg-spec parsing, statement analysis, run-time
compilation (NVRTC needs no GPU), the kernel cache and argument validation."""
import ctypes
import json
import os
import re
import subprocess
import sys

import pytest

from paper_1304_5553_gb300 import pyc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_exports_match_header():
    hdr = open(os.path.join(ROOT, "include", "pyc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(pyc_[a-z_0-9]+)\s*\(", hdr))
    lib = pyc.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pyc.EXPORTED)
    assert pyc.pyc_version().startswith("pyc ")


@pytest.mark.parametrize("spec", [
    "", "float", "float *", "char *x", "float **x", "float *x, float *x", "float i",
    "float n", "float pyc_x", "float x;", "float *x) { } __global__ void evil(float *y",
    "struct foo *x", "float *x,", "unsigned mystery x", "float *restrict", "float *__x",
    "float # x", "float *x, int",
])
def test_bad_argspec(spec):
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_map_create(spec, "1")
    assert e.value.status == pyc.PYC_E_PARSE, (spec, str(e.value))


@pytest.mark.parametrize("stmt", [
    "z[i] = 1; #include <stdio.h>", "z[i] = (1", "z[i] = 1)", "return", "goto out",
    "z[i] = 1; /* open", "z[i] = 'a", "z[i] = pyc_r_z[0]", "z[i] = 1 }", "z[i] = `1`",
    "asm(\"trap;\")",
])
def test_bad_statement(stmt):
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_map_create("float *z", stmt)
    assert e.value.status == pyc.PYC_E_PARSE, (stmt, str(e.value))


def test_compile_error_carries_log():
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_map_create("float *x", "x[i] = undefined_name * 2")
    assert e.value.status == pyc.PYC_E_COMPILE
    assert "undefined_name" in e.value.message and "error" in e.value.message


def _info(spec, stmt):
    h = pyc.pyc_map_create(spec, stmt)
    try:
        return {p["name"]: p for p in pyc.params(h)}, pyc.pyc_map_source(h)
    finally:
        pyc.pyc_map_destroy(h)


def test_statement_analysis():
    p, src = _info("float a, float *x, float b, float *y, float *z", "z[i] = a*x[i] + b*y[i]")
    assert p["x"]["lifted"] and p["x"]["read"] and not p["x"]["written"]
    assert p["z"]["lifted"] and p["z"]["written"] and not p["z"]["read"]
    assert not p["a"]["is_pointer"] and p["a"]["scalar_offset"] == 0 and p["b"]["scalar_offset"] == 4
    assert [p[k]["pointer_slot"] for k in "xyz"] == [0, 1, 2]
    # in-place compound assignment (Listing 1): read and written
    p, _ = _info("float *a", "a[i] *= 2")
    assert p["a"]["lifted"] and p["a"]["read"] and p["a"]["written"]
    # a conditional write must keep unwritten elements: the array is loaded too
    p, _ = _info("float *x, float *z", "if (x[i] > 0) z[i] = 1")
    assert p["z"]["read"] and p["z"]["written"]
    p, _ = _info("float *x, float *z", "float t = x[i]; z[i] = t * t")
    assert not p["z"]["read"] and p["z"]["written"]
    # other index expressions or address-of keep the raw pointer
    p, _ = _info("float *x, float *z", "z[i] = i + 1 < n ? x[i+1] : 0")
    assert not p["x"]["lifted"] and p["z"]["lifted"]
    p, _ = _info("float *x, float *z", "const float *q = &x[i]; z[i] = *q")
    assert not p["x"]["lifted"]
    # a binary '&' after an operand is not address-of
    p, _ = _info("int *x, int *z", "z[i] = 3 & x[i]")
    assert p["x"]["lifted"]
    # member-like names are not the parameter
    p, _ = _info("float *x, float *z", "float2 v; v.x = 1.f; z[i] = v.x + x[i]")
    assert p["x"]["lifted"]


def test_scalar_layout_and_source():
    h = pyc.pyc_map_create("double a, float b, int *x, short c, __nv_bfloat16 d, float *z",
                           "z[i] = a*x[i] + b + c + d")
    try:
        p = {q["name"]: q for q in pyc.params(h)}
        assert (p["a"]["scalar_offset"], p["b"]["scalar_offset"], p["c"]["scalar_offset"],
                p["d"]["scalar_offset"]) == (0, 8, 12, 14)
        assert pyc.load().pyc_map_scalar_bytes(h) == 16
        assert p["d"]["dtype"] == pyc.PYC_BF16 and p["x"]["dtype"] == pyc.PYC_I32
        src = pyc.pyc_map_source(h)
        for v in ("v16_u1", "v16_u2", "v16_u4", "v32_u1", "v32_u2", "v32_u4"):
            assert re.search(r"pyc_map_m[0-9a-f]{8}_" + v + r"\b", src)
            assert re.search(r"pyc_mbatch_m[0-9a-f]{8}_" + v + r"\b", src)
        assert "ld.global.L1::no_allocate.v4.u32" in src and "ld.global.L1::no_allocate.v8.u32" in src
        assert re.search(r"pyc_r_x\s*\[\s*pyc_k\s*\]", src)
        assert re.search(r"pyc_r_z\s*\[\s*pyc_k\s*\]", src)
    finally:
        pyc.pyc_map_destroy(h)


def test_reduce_create_validation():
    cases = [
        (pyc.PYC_F32, "-INFINITY", "a > b ? a : b", None, "float *x", {"compensated": 1}),
        (pyc.PYC_F64, "0", "a+b", None, "double *x", {"compensated": 1}),
        (pyc.PYC_ARGMIN_F32, "0", None, None, "float *x", {}),
        (pyc.PYC_F32, "0", "a+b", None, "float *x, float *y", {}),
        (pyc.PYC_U8, "0", "a+b", None, "unsigned char *x", {}),
        (pyc.PYC_F32, None, "a+b", None, "float *x", {}),
        (pyc.PYC_F32, "0", "a+b", None, "float *x", {"block": 100}),
        (pyc.PYC_F32, "0", "a+b", None, "float *x", {"items_per_thread": 3}),
        (pyc.PYC_F32, "0", "a+b; }", None, "float *x", {}),
    ]
    for dt, neu, red, m, spec, o in cases:
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_reduce_create(dt, neu, red, m, spec, o or None)
        assert e.value.status in (pyc.PYC_E_ARG, pyc.PYC_E_PARSE), (dt, neu, red, spec, o)
    h = pyc.pyc_reduce_create(pyc.PYC_ARGMIN_F32, None, None, None, "float *x")
    assert pyc.pyc_reduce_out_bytes(h) == 16
    pyc.pyc_reduce_destroy(h)
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", None, "float *x", {"compensated": 1})
    assert "pyc_two_sum" in pyc.pyc_reduce_source(h) and pyc.pyc_reduce_out_bytes(h) == 4
    pyc.pyc_reduce_destroy(h)


def test_batched_validation_before_any_gpu_work():
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y")
    try:
        with pytest.raises(pyc.PycError) as e:  # decreasing offsets
            pyc.pyc_reduce_batched(h, 2, [0, 5, 3], [1 << 20, 1 << 21], None, 1 << 22)
        assert e.value.status == pyc.PYC_E_ARG
        pyc.pyc_reduce_batched(h, 0, [0], [1 << 20, 1 << 21], None, 1 << 22)  # no-op
    finally:
        pyc.pyc_reduce_destroy(h)


def test_batched_null_arrays_and_scalars_are_argument_errors():
    """A NULL ptrs (or scalar block) for a spec that declares arrays (scalars)
    is PYC_E_ARG from the segmented calls and the plan call alike, before any
    read of the missing table (the plan's cache key copies ptrs[])."""
    import numpy as np
    lib = pyc.load()
    off = np.array([0, 7, 100], np.int64)
    offp = off.ctypes.data_as(pyc.ctypes.POINTER(pyc.ctypes.c_int64))
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y")
    hs = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "a*x[i]", "float a, float *x")
    try:
        for fn in (lib.pyc_reduce_batched, lib.pyc_reduce_batched_autotune):
            assert fn(h, 2, offp, None, None, 1 << 22, None) == pyc.PYC_E_ARG
            assert "ptrs is NULL" in pyc.pyc_last_error()
            assert fn(hs, 2, offp, pyc._ptr_array([1 << 20]), None, 1 << 22, None) == pyc.PYC_E_ARG
            assert "scalars is NULL" in pyc.pyc_last_error()
        assert lib.pyc_reduce_batched_plan(h, 2, off.ctypes.data, None, None, None, None, 0,
                                           None, None) == pyc.PYC_E_ARG
        assert lib.pyc_reduce_batched_plan(hs, 2, off.ctypes.data, pyc._ptr_array([1 << 20]),
                                           None, None, None, 0, None, None) == pyc.PYC_E_ARG
    finally:
        pyc.pyc_reduce_destroy(h)
        pyc.pyc_reduce_destroy(hs)


@pytest.mark.skipif(_has_gpu(), reason="checks the no-driver error path")
def test_launch_without_driver_is_an_error():
    h = pyc.pyc_map_create("float *x", "x[i] = 1")
    try:
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_map_launch(h, 10, [1 << 20])
        assert e.value.status == pyc.PYC_E_CUDA
    finally:
        pyc.pyc_map_destroy(h)


_CACHE_CHILD = r"""
import json, sys
sys.path.insert(0, %r)
from paper_1304_5553_gb300 import pyc
h = pyc.pyc_map_create("float *x, float *z", sys.argv[1])
h2 = pyc.pyc_map_create("float *x, float *z", sys.argv[1])
print(json.dumps(pyc.pyc_cache_stats()))
"""


def test_kernel_cache_memory_and_disk(tmp_path):
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    code = _CACHE_CHILD % ROOT

    def run(stmt):
        out = subprocess.run([sys.executable, "-c", code, stmt], env=env, capture_output=True,
                             text=True, check=True).stdout
        return json.loads(out.strip().splitlines()[-1])

    a = run("z[i] = 3 * x[i]")
    assert a == {"compiled": 1, "disk_hits": 0, "mem_hits": 1}
    b = run("z[i] = 3 * x[i]")  # new process: loaded from disk, no compile
    assert b == {"compiled": 0, "disk_hits": 1, "mem_hits": 1}
    c = run("z[i] = 4 * x[i]")  # a changed kernel recompiles
    assert c["compiled"] == 1
    # a corrupted cache file is ignored and rewritten
    for f in os.listdir(tmp_path):
        if f.endswith(".pyck"):
            open(os.path.join(tmp_path, f), "wb").write(b"garbage")
    d = run("z[i] = 3 * x[i]")
    assert d["compiled"] == 1 and d["disk_hits"] == 0


def test_kernel_cache_checks_the_full_key(tmp_path):
    # a cache file stored under one spec's hash but holding another spec's key
    # text (what a hash collision would look like) is not loaded: the spec recompiles
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    code = _CACHE_CHILD % ROOT

    def run(stmt):
        out = subprocess.run([sys.executable, "-c", code, stmt], env=env, capture_output=True,
                             text=True, check=True).stdout
        return json.loads(out.strip().splitlines()[-1])

    run("z[i] = 5 * x[i]")
    first = set(f for f in os.listdir(tmp_path) if f.endswith(".pyck"))
    run("z[i] = 6 * x[i]")
    second = set(f for f in os.listdir(tmp_path) if f.endswith(".pyck")) - first
    assert len(first) == 1 and len(second) == 1
    (a,), (b,) = first, second
    data = open(os.path.join(tmp_path, a), "rb").read()
    open(os.path.join(tmp_path, b), "wb").write(data)
    r = run("z[i] = 6 * x[i]")
    assert r["compiled"] == 1 and r["disk_hits"] == 0
    # the other spec still loads its own file
    assert run("z[i] = 5 * x[i]")["disk_hits"] == 1


def test_kernel_cache_units(tmp_path):
    """A generated source is split into one NVRTC unit per kernel (compiled in
    parallel); its cache record holds one binary per unit, and a record cut
    short inside a unit is ignored and rewritten."""
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    code = _CACHE_CHILD % ROOT

    def run(stmt):
        out = subprocess.run([sys.executable, "-c", code, stmt], env=env, capture_output=True,
                             text=True, check=True).stdout
        return json.loads(out.strip().splitlines()[-1])

    assert run("z[i] = 7 * x[i]")["compiled"] == 1
    (f,) = [g for g in os.listdir(tmp_path) if g.endswith(".pyck")]
    path = os.path.join(tmp_path, f)
    data = open(path, "rb").read()
    assert data.startswith(b"PYCK2\n")
    p = 6
    nl = data.index(b"\n", p)
    klen = int(data[p:nl])
    key = data[nl + 1:nl + 1 + klen]
    p = nl + 1 + klen
    nl = data.index(b"\n", p)
    units = int(data[p:nl])
    # six variants, each a single map and a batched map kernel
    assert units == 12 and key.count(b"\n//@@pyc-unit\n") == 12
    p = nl + 1
    for _ in range(units):
        nl = data.index(b"\n", p)
        p = nl + 1 + int(data[p:nl])
    assert p == len(data)
    open(path, "wb").write(data[:-100])
    r = run("z[i] = 7 * x[i]")
    assert r["compiled"] == 1 and r["disk_hits"] == 0
    assert run("z[i] = 7 * x[i]")["disk_hits"] == 1


def test_front_end_params():
    k = pyc.ElementwiseKernel("float a, float *x, float b, float *y, float *z",
                              "z[i] = a*x[i] + b*y[i]", "linear_combination")
    assert [p["name"] for p in k._params] == ["a", "x", "b", "y", "z"]
    buf = pyc.pack_scalars(k._h, [5, 6])  # Listing 3a passes ints for float params
    import struct
    assert struct.unpack_from("ff", buf, 0) == (5.0, 6.0)


@pytest.mark.skipif(_has_gpu(), reason="checks the no-driver error path")
def test_server_without_driver_is_an_error():
    with pytest.raises(pyc.PycError) as e:
        pyc.pyc_server_create(1 << 20)
    assert e.value.status == pyc.PYC_E_CUDA


def test_server_config_validation():
    for bad in (dict(mem_budget_bytes=0), dict(mem_budget_bytes=1 << 20, num_streams=100)):
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_server_create(**bad)
        assert e.value.status == pyc.PYC_E_ARG


def test_scan_create_validation():
    h = pyc.pyc_scan_create(pyc.PYC_F32, "0", "a+b", "x[i]", "y[i] = item", "float *x, float *y")
    p = {q["name"]: q for q in pyc.params(h, "scan")}
    assert p["x"]["lifted"] and p["x"]["read"] and not p["x"]["written"]
    assert p["y"]["lifted"] and p["y"]["written"] and not p["y"]["read"]
    src = pyc.pyc_scan_source(h)
    assert "pyc_scan_s" in src and "pyc_lookback" in src
    pyc.pyc_scan_destroy(h)
    bad = [
        (pyc.PYC_BF16, "0", "a+b", "x[i]", "y[i] = item", "float *x, float *y"),
        (pyc.PYC_F32, "0", "a+b", "x[i]", "y[i] = item", "float *x, float *item"),
        (pyc.PYC_F32, "0", "a+b; }", "x[i]", "y[i] = item", "float *x, float *y"),
    ]
    for args in bad:
        with pytest.raises(pyc.PycError) as e:
            pyc.pyc_scan_create(*args)
        assert e.value.status in (pyc.PYC_E_ARG, pyc.PYC_E_PARSE)


def test_batched_config_default_and_fixed_options():
    # no tuning has run for these handles: the default batched configuration
    # (16-byte vectors, unroll 1, 256 threads), with fixed options taking over
    spec = "float *x, float *y"
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]+0.0f*%d" % os.getpid(), spec)
    assert pyc.batched_config(h) == (16, 1, 256)
    g = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", spec,
                              {"vec_bytes": 32, "items_per_thread": 2, "block": 128})
    assert pyc.batched_config(g) == (32, 2, 128)
    assert pyc.load().pyc_reduce_batched_config(None, None, None, None, None) == pyc.PYC_E_ARG
    pyc.pyc_reduce_destroy(h)
    pyc.pyc_reduce_destroy(g)


def test_no_alloc_tests_are_collected_last():
    # the allocation-free entry point's GPU test file runs after every other
    # GPU test, so a run that stops at the first failure has run the rest first
    out = subprocess.run([sys.executable, "-m", "pytest", "--collect-only", "-q", "-m", "gpu",
                          "-p", "no:cacheprovider", os.path.join(ROOT, "tests")],
                         capture_output=True, text=True, cwd=ROOT).stdout
    ids = [ln for ln in out.splitlines() if "::" in ln]
    files = [ln.split("::")[0] for ln in ids]
    assert files and files[-1].endswith("test_zz_no_alloc.py")
    first = files.index(files[-1])
    assert all(f.endswith("test_zz_no_alloc.py") for f in files[first:])


_FUZZ_CHILD = r'''
import json, random, sys
sys.path.insert(0, %r)
from paper_1304_5553_gb300 import pyc
rng = random.Random(1304)
spec_tok = ["float", "int", "double", "__half", "unsigned", "long", "char", "const", "struct",
            "__restrict__", "*", "**", ",", ";", "(", ")", "[", "]", "#", "x", "y", "i", "n",
            "0", "a", "pyc_q", "void", "float *x", "int k"]
stmt_tok = ["x[i]", "z[i]", "=", "+", "*", "/", "k", "i", "(", ")", ";", "[", "]", "1",
            "2.5f", "if", "else", "{", "}", "#", "/*", "*/", "\"", "'", "?", ":", "return",
            "->", ".", "x", "z", "+=", "<<", "sin(", "exp(", "n", "__syncthreads()", "\\"]
counts = {}
for _ in range(400):
    s = " ".join(rng.choice(spec_tok) for _ in range(rng.randint(1, 6)))
    try:
        h = pyc.pyc_map_create(s, "0")
        pyc.pyc_map_destroy(h)
        st = 0
    except pyc.PycError as e:
        st = e.status
    counts["spec%%d" %% st] = counts.get("spec%%d" %% st, 0) + 1
for _ in range(120):
    s = " ".join(rng.choice(stmt_tok) for _ in range(rng.randint(1, 8)))
    try:
        h = pyc.pyc_map_create("float *x, float *z, int k", s)
        pyc.pyc_map_destroy(h)
        st = 0
    except pyc.PycError as e:
        st = e.status
    counts["stmt%%d" %% st] = counts.get("stmt%%d" %% st, 0) + 1
red_tok = ["a", "b", "+", "*", "?", ":", ">", "<", "(", ")", "0", "1", "INFINITY", "x[i]",
           "y[i]", ";", "{", "#", "a>b", "i", "/*", "\"", "min(", "fmaxf(a,b)", ","]
for _ in range(120):
    parts = [" ".join(rng.choice(red_tok) for _ in range(rng.randint(1, 5))) for _ in range(3)]
    try:
        h = pyc.pyc_reduce_create(rng.choice([pyc.PYC_F32, pyc.PYC_I64, pyc.PYC_F64]), parts[0],
                                  parts[1], parts[2], "float *x, float *y")
        pyc.pyc_reduce_destroy(h)
        st = 0
    except pyc.PycError as e:
        st = e.status
    counts["red%%d" %% st] = counts.get("red%%d" %% st, 0) + 1
for _ in range(60):
    parts = [" ".join(rng.choice(red_tok + ["item", "prev_item", "y[i] ="])
                      for _ in range(rng.randint(1, 5))) for _ in range(4)]
    try:
        h = pyc.pyc_scan_create(pyc.PYC_F32, parts[0], parts[1], parts[2], parts[3],
                                "float *x, float *y")
        pyc.pyc_scan_destroy(h)
        st = 0
    except pyc.PycError as e:
        st = e.status
    counts["scan%%d" %% st] = counts.get("scan%%d" %% st, 0) + 1
expr_tok = ["(", ")", "(+", "(*", "(-", "(/", "(sin", "(exp", "(where", "(pow", "(f32", "(i64",
            "(<", "(min", "$0", "$1", "$2", "%%2", "%%0", "$9", "1.5", "2", "-3", "1e400", "(neg",
            "(floor", "(bogus", "))", "$", "%%", "(rsqrt"]
for _ in range(150):
    e = " ".join(rng.choice(expr_tok) for _ in range(rng.randint(1, 9)))
    try:
        h = pyc.pyc_expr_map_create(e, [pyc.PYC_F32, pyc.PYC_I32, pyc.PYC_F32], [1, 1, 0],
                                    pyc.PYC_F32)
        pyc.pyc_map_destroy(h)
        st = 0
    except pyc.PycError as err:
        st = err.status
    counts["expr%%d" %% st] = counts.get("expr%%d" %% st, 0) + 1
print(json.dumps(counts))
'''


def test_random_specs_and_statements_never_crash(tmp_path):
    # seeded random token soup for argument specs, map statements, map-reduce and
    # scan expressions and fused array expressions: every create returns a status
    # (accepted, parse, argument or compile error); none crashes
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    p = subprocess.run([sys.executable, "-c", _FUZZ_CHILD % ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    counts = json.loads(p.stdout.strip().splitlines()[-1])
    allowed = {pyc.PYC_OK, pyc.PYC_E_PARSE, pyc.PYC_E_COMPILE, pyc.PYC_E_ARG}
    for k in counts:
        assert int(re.sub(r"\D", "", k)) in allowed, counts
    assert sum(v for k, v in counts.items() if k.startswith("spec")) == 400
    assert sum(v for k, v in counts.items() if k.startswith("stmt")) == 120
    assert sum(v for k, v in counts.items() if k.startswith("red")) == 120
    assert sum(v for k, v in counts.items() if k.startswith("scan")) == 60
    assert sum(v for k, v in counts.items() if k.startswith("expr")) == 150


def test_plain_c_program_uses_the_header_and_library(tmp_path):
    # the boundary is a C ABI: a C11 program compiles against include/pyc.h with
    # strict warnings, links libpyc.so and makes the calls that need no GPU
    from paper_1304_5553_gb300 import buildlib
    src = os.path.join(ROOT, "tests", "c_abi", "abi_consumer.c")
    lib = buildlib.pyc_lib_path()
    pyc.load()
    exe = str(tmp_path / "abi_consumer")
    cc = os.environ.get("CC", "gcc")
    p = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), src, "-o", exe,
                        "-L", os.path.dirname(lib), "-lpyc",
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path / "cache"))
    out = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    assert lines[0].startswith("version pyc ")
    assert "map params 5 scalar_bytes 8" in lines
    assert "param a ptr 0 dtype %d off 0 slot -1" % pyc.PYC_F32 in lines
    assert "param x ptr 1 dtype %d off -1 slot 0" % pyc.PYC_F32 in lines
    assert "param z ptr 1 dtype %d off -1 slot 2" % pyc.PYC_F32 in lines
    assert "source has kernel 1" in lines
    assert "reduce_create 0 out_bytes 4" in lines
    assert "bad spec %d null 1 msg 1" % pyc.PYC_E_PARSE in lines


_THREADS_CHILD = r'''
import json, sys, threading
sys.path.insert(0, %r)
from paper_1304_5553_gb300 import pyc
specs = [("float *x, float *z", "z[i] = %%d * x[i] + 1" %% k) for k in range(6)]
results, errors = {}, []

def worker(t):
    try:
        for j in range(len(specs)):
            spec, stmt = specs[(j + t) %% len(specs)]
            h = pyc.pyc_map_create(spec, stmt)
            results.setdefault(stmt, set()).add(pyc.pyc_map_source(h))
            pyc.pyc_map_destroy(h)
            r = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", stmt.split("= ")[1], spec)
            pyc.pyc_reduce_destroy(r)
        try:  # a spec that fails to compile: every thread gets the compile error
            pyc.pyc_map_create("float *x, float *z", "z[i] = no_such_function(x[i])")
            errors.append("compiled a bad spec")
        except pyc.PycError as e:
            if e.status != pyc.PYC_E_COMPILE or "no_such_function" not in str(e):
                errors.append("wrong error: %%d %%s" %% (e.status, e))
    except Exception as e:  # reported to the parent
        errors.append(repr(e))

ts = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
[t.start() for t in ts]
[t.join() for t in ts]
print(json.dumps({"errors": errors, "distinct_sources": {k: len(v) for k, v in results.items()},
                  "stats": pyc.pyc_cache_stats()}))
'''


def test_concurrent_creates_from_eight_threads(tmp_path):
    # eight host threads create the same six map and six map-reduce specs in
    # different orders (the C calls run without the interpreter lock): no errors,
    # one generated source per spec, and each of the twelve kernels compiled once
    # (a thread that asks while another compiles the same source waits for it)
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    p = subprocess.run([sys.executable, "-c", _THREADS_CHILD % ROOT], env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    res = json.loads(p.stdout.strip().splitlines()[-1])
    assert res["errors"] == []
    assert len(res["distinct_sources"]) == 6
    assert all(v == 1 for v in res["distinct_sources"].values())
    assert res["stats"]["compiled"] == 12
    # the twelve good kernels: 84 hits; the failing spec: a thread that asked while
    # another compiled it counts a hit, one that asked later compiles (and fails) again
    assert 8 * 12 - 12 <= res["stats"]["mem_hits"] <= 8 * 12 - 12 + 7


def test_shard_and_combine_argument_errors_need_no_gpu():
    """pyc_reduce_shard / pyc_reduce_combine reject bad ranges, NULL or
    misaligned records and non-elementwise arrays before any GPU work."""
    lib = pyc.load()
    E = pyc.PYC_E_ARG
    h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y")
    hs = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i+1]-x[i]", "float *x")
    hk = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "k*x[i]*y[i]", "float k, float *x, float *y")
    p = pyc._ptr_array([1 << 20, 1 << 21])
    rec = 1 << 22
    try:
        for n_total, i0, n in ((-1, 0, 0), (10, -1, 1), (10, 0, -1), (10, 8, 3), (10, 11, 0),
                               (2 ** 62, 2 ** 62, 2 ** 62)):
            assert lib.pyc_reduce_shard(h, n_total, i0, n, p, None, rec, None) == E
            assert "exceeds" in pyc.pyc_last_error() or ">= 0" in pyc.pyc_last_error()
        assert lib.pyc_reduce_shard(h, 10, 0, 10, p, None, None, None) == E
        assert lib.pyc_reduce_shard(h, 10, 0, 10, p, None, rec + 4, None) == E
        assert lib.pyc_reduce_shard(hs, 10, 0, 10, p, None, rec, None) == E
        assert "a shard holds only its own elements" in pyc.pyc_last_error()
        assert lib.pyc_reduce_shard(h, 10, 0, 10, pyc._ptr_array([0, 1 << 21]), None, rec,
                                    None) == E
        assert lib.pyc_reduce_shard(None, 10, 0, 10, p, None, rec, None) == E
        # NULL arrays or scalars for a spec that declares them: argument errors
        # before the pointers are read
        assert lib.pyc_reduce_shard(h, 10, 0, 10, None, None, rec, None) == E
        assert "ptrs is NULL" in pyc.pyc_last_error()
        assert lib.pyc_reduce_shard(hk, 10, 0, 10, p, None, rec, None) == E
        assert "scalars is NULL" in pyc.pyc_last_error()
        assert lib.pyc_reduce_combine(h, -1, rec, rec, None) == E
        assert lib.pyc_reduce_combine(h, 2, None, rec, None) == E
        assert lib.pyc_reduce_combine(h, 2, rec + 4, rec, None) == E
        assert lib.pyc_reduce_combine(h, 2, rec, None, None) == E
        assert lib.pyc_reduce_combine(h, 2, rec, rec + 2, None) == E
        assert lib.pyc_reduce_combine(None, 2, rec, rec, None) == E
    finally:
        pyc.pyc_reduce_destroy(h)
        pyc.pyc_reduce_destroy(hs)
        pyc.pyc_reduce_destroy(hk)


def test_shard_and_combine_kernels_are_generated():
    """A map-reduce's main module holds the single and batched reductions; the
    shard kernels (six variants), the record combine and the register-lean
    batched builds are in its extra module, compiled on first use."""
    for out, kw in ((pyc.PYC_F32, {}), (pyc.PYC_F32, {"compensated": 1}),
                    (pyc.PYC_ARGMIN_F32, {}), (pyc.PYC_I64, {}), (pyc.PYC_BF16, {})):
        if out == pyc.PYC_ARGMIN_F32:
            h = pyc.pyc_reduce_create(out, None, None, "x[i]", "float *x")
        elif out == pyc.PYC_I64:
            h = pyc.pyc_reduce_create(out, "0", "a+b", "(long long)x[i]", "int *x")
        else:
            h = pyc.pyc_reduce_create(out, "0", "a+b", "x[i]", "float *x", kw)
        src = pyc.pyc_reduce_source(h)
        assert src.count("__global__ void __launch_bounds__(512) pyc_reduce_") == 6
        assert src.count("__global__ void __launch_bounds__(512) pyc_rbatch_") == 6
        assert "pyc_rshard_" not in src.split("pyc_shard_body")[-1] and "_r80(" not in src
        assert 'static_assert(sizeof(pyc_record) == 16, "record size")' in src
        pyc.pyc_reduce_destroy(h)


_EXT_CHILD = r"""
import json, sys
sys.path.insert(0, %r)
from paper_1304_5553_gb300 import pyc
lib = pyc.load()
h = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i]*y[i] + 0.5f", "float *x, float *y")
c0 = pyc.pyc_cache_stats()["compiled"]
st = []
for _ in range(2):
    st.append(lib.pyc_reduce_shard(h, 100, 0, 100, pyc._ptr_array([1 << 20, 1 << 21]), None,
                                   1 << 22, None))
c1 = pyc.pyc_cache_stats()["compiled"]
print(json.dumps({"c0": c0, "c1": c1, "st": st}))
"""


@pytest.mark.skipif(_has_gpu(), reason="checks the compile-then-no-driver path")
def test_extra_module_is_compiled_on_first_use(tmp_path):
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    out = subprocess.run([sys.executable, "-c", _EXT_CHILD % ROOT], env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["c0"] == 1            # creation compiled the main module only
    assert r["c1"] == 2            # the first shard call compiled the extra module, once
    assert r["st"] == [pyc.PYC_E_CUDA, pyc.PYC_E_CUDA]  # then needed a GPU


def test_sparse_null_and_misaligned_arrays_are_argument_errors():
    """The sparse calls reject NULL vectors and arrays not aligned to their
    element size (a kernel given one would fault) before any GPU work."""
    lib = pyc.load()
    E = pyc.PYC_E_ARG
    V = ctypes.c_void_p
    h = ctypes.c_void_p()
    for vt, vb in ((pyc.PYC_F32, 4), (pyc.PYC_F64, 8)):
        for rp, ci, va in ((1 << 20, 1 << 21, (1 << 22) + vb // 2), ((1 << 20) + 4, 1 << 21, 1 << 22),
                           (1 << 20, (1 << 21) + 2, 1 << 22)):
            assert lib.pyc_csr_create(4, 4, 8, V(rp), V(ci), V(va), vt, ctypes.byref(h)) == E
            assert "aligned" in pyc.pyc_last_error()
        a = pyc.pyc_csr_create(4, 4, 8, 1 << 20, 1 << 21, 1 << 22, vt)
        try:
            good, odd = 1 << 23, (1 << 23) + vb // 2
            for x, y in ((None, good), (good, None), (odd, good), (good, odd)):
                assert lib.pyc_spmv(a, V(x), V(y), None) == E
                assert lib.pyc_spmv_autotune(a, V(x), V(y), None) == E
            info = pyc.pyc_cg_info()
            for b, x in ((None, good), (good, None), (odd, good), (good, odd)):
                assert lib.pyc_cg_solve(a, V(b), V(x), ctypes.c_double(1e-6), 10, None,
                                        ctypes.byref(info)) == E
        finally:
            pyc.pyc_csr_destroy(a)


def test_every_array_is_checked_before_a_launch():
    """NULL or misaligned arrays are PYC_E_ARG before any GPU work, also those
    a statement indexes other than as name[i] (not on the vector path)."""
    lib = pyc.load()
    m = pyc.pyc_map_create("float *x, float *y", "y[i] = x[i + 1] - x[i]")
    r = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "x[i + 1] * y[i]", "float *x, float *y")
    try:
        for xp, what in ((0, "is NULL"), ((1 << 20) + 2, "not aligned")):
            assert lib.pyc_map_launch(m, 10, pyc._ptr_array([xp, 1 << 21]), None,
                                      None) == pyc.PYC_E_ARG
            assert what in pyc.pyc_last_error()
            assert lib.pyc_reduce_launch(r, 10, pyc._ptr_array([xp, 1 << 21]), None, 1 << 22,
                                         None) == pyc.PYC_E_ARG
            assert what in pyc.pyc_last_error()
        # n = 0 launches nothing: a NULL array is allowed there
        assert lib.pyc_map_launch(m, 0, pyc._ptr_array([0, 0]), None, None) == pyc.PYC_OK
    finally:
        pyc.pyc_map_destroy(m)
        pyc.pyc_reduce_destroy(r)


def test_expression_casts_need_no_prior_evaluation():
    """Expr.astype builds a cast node on its own (no evaluation has to come
    first) and refuses a dtype the expression language has no cast for."""
    import torch

    from paper_1304_5553_gb300 import gpuarray as ga
    leaf = ga.Expr("leaf")
    for dt, op in ((torch.float32, "f32"), (torch.float64, "f64"), (torch.int32, "i32"),
                   (torch.int64, "i64")):
        e = leaf.astype(dt)
        assert e.op == op and e.args == (leaf,)
    with pytest.raises(TypeError):
        leaf.astype(torch.bfloat16)


def test_introspection_of_reduce_and_scan_handles():
    """Parameter records, scalar block sizes and launch configurations of
    map-reduce and scan handles (no GPU needed)."""
    lib = pyc.load()
    r = pyc.pyc_reduce_create(pyc.PYC_F32, "0", "a+b", "k*x[i]*y[i]",
                              "float k, const float *x, float *y")
    s = pyc.pyc_scan_create(pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "y[i] = prev_item",
                            "int *x, long long *y")
    try:
        assert lib.pyc_reduce_num_params(r) == 3 and lib.pyc_reduce_scalar_bytes(r) == 4
        assert lib.pyc_scan_num_params(s) == 2 and lib.pyc_scan_scalar_bytes(s) == 0
        info = pyc.pyc_param_info()
        want = [(b"k", 0, pyc.PYC_F32, 4, 0, -1, 0), (b"x", 1, pyc.PYC_F32, 4, -1, 0, 1),
                (b"y", 1, pyc.PYC_F32, 4, -1, 1, 1)]
        for i, w in enumerate(want):
            assert lib.pyc_reduce_param(r, i, ctypes.byref(info)) == pyc.PYC_OK
            got = (info.name, info.is_pointer, info.dtype, info.elem_bytes, info.scalar_offset,
                   info.pointer_slot, info.read)
            assert got == w, (i, got)
            assert info.written == 0  # a map expression only reads
        assert lib.pyc_reduce_param(r, 3, ctypes.byref(info)) == pyc.PYC_E_ARG
        assert lib.pyc_scan_param(s, 1, ctypes.byref(info)) == pyc.PYC_OK
        assert (info.name, info.dtype, info.read, info.written) == (b"y", pyc.PYC_I64, 0, 1)
        assert lib.pyc_scan_param(s, -1, ctypes.byref(info)) == pyc.PYC_E_ARG
        v, u, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        for fn, h in ((lib.pyc_reduce_config, r), (lib.pyc_scan_config, s)):
            assert fn(h, ctypes.c_int64(1 << 20), ctypes.byref(v), ctypes.byref(u),
                      ctypes.byref(b)) == pyc.PYC_OK
            assert v.value in (16, 32) and u.value in (1, 2, 4) and b.value % 32 == 0
    finally:
        pyc.pyc_reduce_destroy(r)
        pyc.pyc_scan_destroy(s)


def test_expression_typing_matches_the_typed_oracle():
    """pyc_expr_type (the library's typing of fused expressions) gives, for every
    operator and pair of operand types, the type the expression oracle's typed
    evaluation computes in."""
    import numpy as np

    from oracle import expr as ox
    dts = {pyc.PYC_I32: np.int32, pyc.PYC_I64: np.int64, pyc.PYC_F32: np.float32,
           pyc.PYC_F64: np.float64}
    back = {v: k for k, v in dts.items()}
    for a in dts:
        for op in ("neg", "abs", "sqrt", "f32", "f64", "i32", "i64"):
            got = pyc.pyc_expr_type("(%s $0)" % op, [a], [1])
            assert got == back[ox.result_type(op, [dts[a]])], (op, a, got)
        for b in dts:
            for op in ("+", "-", "*", "/", "min", "max"):
                got = pyc.pyc_expr_type("(%s $0 $1)" % op, [a, b], [1, 1])
                assert got == back[ox.result_type(op, [dts[a], dts[b]])], (op, a, b, got)
            assert pyc.pyc_expr_type("(< $0 $1)", [a, b], [1, 1]) == pyc.PYC_I32
            # a scalar argument carries its own type like an array
            got = pyc.pyc_expr_type("(* $0 %1)", [a, b], [1, 0])
            assert got == back[ox.result_type("*", [dts[a], dts[b]])], (a, b, got)
    # bfloat16 and binary16 arrays are read as binary32
    for h in (pyc.PYC_BF16, pyc.PYC_F16):
        assert pyc.pyc_expr_type("(+ $0 $1)", [h, pyc.PYC_I64], [1, 1]) == pyc.PYC_F32


def test_partial_overlap_with_a_written_array_is_an_argument_error():
    """A written array that overlaps another array in part is undefined behaviour
    (only exact aliasing is allowed, as in Listing 1's in-place a[i] *= 2); for
    arrays indexed as name[i] the host rejects it before any GPU work: maps, scans
    and host-array maps."""
    lib = pyc.load()
    m = pyc.pyc_map_create("float *x, float *y", "y[i] = 2*x[i]")
    s = pyc.pyc_scan_create(pyc.PYC_I64, "0", "a+b", "(long long)x[i]", "y[i] = item",
                            "int *x, long long *y")
    base = 1 << 20
    try:
        for xp, yp in ((base, base + 400), (base + 400, base), (base, base + 3996)):
            assert lib.pyc_map_launch(m, 1000, pyc._ptr_array([xp, yp]), None,
                                      None) == pyc.PYC_E_ARG
            assert "overlap in part" in pyc.pyc_last_error()
            assert lib.pyc_map_launch_host(m, 1000, pyc._ptr_array([xp, yp]),
                                           None) == pyc.PYC_E_ARG
            assert "overlap in part" in pyc.pyc_last_error()
        # int32 input and int64 output at the same address differ in element size:
        # y[i] would overwrite x[2i] and x[2i + 1] before they are read
        assert lib.pyc_scan_launch(s, 1000, pyc._ptr_array([base, base]), None,
                                   None) == pyc.PYC_E_ARG
        assert "overlap in part" in pyc.pyc_last_error()
        # disjoint ranges and exact aliasing pass the check and go on to launch, which
        # needs the driver: only where there is none (the pointers here are not real)
        if not _has_gpu():
            for xp, yp in ((base, base + 4000), (base + 4000, base), (base, base)):
                lib.pyc_map_launch(m, 1000, pyc._ptr_array([xp, yp]), None, None)
                assert "overlap" not in pyc.pyc_last_error()
        # n = 0 touches nothing
        assert lib.pyc_map_launch(m, 0, pyc._ptr_array([base, base + 4]), None,
                                  None) == pyc.PYC_OK
    finally:
        pyc.pyc_map_destroy(m)
        pyc.pyc_scan_destroy(s)


_TUNE_CHILD = r"""
import json, os, sys
sys.path.insert(0, %r)
from paper_1304_5553_gb300 import pyc

def digest(data):
    # the library's source digest (two 64-bit FNV-style lanes), the tuning cache's key
    h1, h2, m = 1469598103934665603, 0x9E3779B97F4A7C15, (1 << 64) - 1
    for c in data:
        h1 = ((h1 ^ c) * 1099511628211) & m
        h2 = (((h2 ^ c) * 0x100000001B3) + 0x632BE59BD9B4E019) & m
        h2 ^= h2 >> 29
    return "%%016x%%016x" %% (h1, h2)

spec, stmt = "float *x, float *y", "y[i] = 3.0f * x[i]"
h0 = pyc.pyc_map_create(spec, stmt)
key = digest(pyc.pyc_map_source(h0).encode())
# records as the library writes them (compact), and with spaces as json.dumps writes them
rec = lambda **k: json.dumps(dict({"key": key, "kind": "map", "us": 1.0}, **k),
                             separators=(",", ":") if k.get("bucket", 0) %% 2 else None)
lines = [rec(bucket=10, vec_bytes=32, unroll=2, block=128),
         rec(bucket=10, vec_bytes=16, unroll=1, block=512),        # a later line wins
         rec(bucket=11, vec_bytes=32, unroll=4, block=64, kind="reduce"),  # another kind
         json.dumps({"key": "0" * 32, "kind": "map", "bucket": 11, "vec_bytes": 32,
                     "unroll": 4, "block": 64}),                   # another spec
         rec(bucket=12, vec_bytes=8, unroll=2, block=128),         # not a valid variant
         rec(bucket=13, vec_bytes=32, unroll=4, block=96)]
with open(os.path.join(os.environ["PYC_CACHE_DIR"], "tune.jsonl"), "a") as f:
    f.write("\n".join(lines) + "\n")
h = pyc.pyc_map_create(spec, stmt)                                 # loads the cache
out = {}
for n in (2 ** 19 - 1, 2 ** 19, 2 ** 21 - 1, 2 ** 21, 2 ** 23, 2 ** 25, 2 ** 27 - 1, 2 ** 27):
    out[n] = list(pyc.launch_config(h, n))
fixed = pyc.pyc_map_create(spec, stmt, None, {"block": 256})      # options win over tuning
out["fixed"] = list(pyc.launch_config(fixed, 2 ** 19))
print(json.dumps(out))
"""


def test_tuning_cache_buckets(tmp_path):
    """Tuned configurations persist per (source digest, kind, size bucket), the
    bucket of n being half the bit length of n (two powers of two per bucket);
    records of another kind or spec, or with an invalid variant, are ignored, a
    later record of a bucket wins, and configuration options override."""
    env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path))
    out = subprocess.run([sys.executable, "-c", _TUNE_CHILD % ROOT], env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    r = json.loads(out.stdout.strip().splitlines()[-1])
    default = [16, 4, 256]
    want = {2 ** 19 - 1: default, 2 ** 19: [16, 1, 512], 2 ** 21 - 1: [16, 1, 512],
            2 ** 21: default, 2 ** 23: default, 2 ** 25: [32, 4, 96], 2 ** 27 - 1: [32, 4, 96],
            2 ** 27: default}
    for n, cfg in want.items():
        assert r[str(n)] == cfg, (n, r[str(n)])
    assert r["fixed"] == [16, 1, 256]


_LOG_CHILD = r"""
import sys
sys.path.insert(0, %r)
from paper_1304_5553_gb300 import pyc
h = pyc.pyc_map_create("float *x, float *y", "y[i] = x[i] * 9.0f - 1.0f")
s = pyc.pyc_server_create_host(lambda req, value: 0, 1 << 20)
pyc.pyc_server_destroy(s)
"""


def test_event_log(tmp_path):
    """PYC_LOG=1: one stderr line per compilation (and, in a later process, per
    disk-cache load) and per server creation and destruction; nothing without."""
    def run(log):
        env = dict(os.environ, PYC_CACHE_DIR=str(tmp_path), PYC_LOG=log)
        p = subprocess.run([sys.executable, "-c", _LOG_CHILD % ROOT], env=env,
                           capture_output=True, text=True, timeout=600)
        assert p.returncode == 0, p.stderr
        return [l for l in p.stderr.splitlines() if l.startswith("pyc: ")]
    first = run("1")
    assert any(re.match(r"pyc: compiled \d+ kernel units with NVRTC in \d+ ms", l) for l in first)
    assert any(l.startswith("pyc: server created with host-executed batches") for l in first)
    assert any(l.startswith("pyc: server destroyed: 0 requests completed") for l in first)
    second = run("1")
    assert any(l.startswith("pyc: loaded") and "from the disk cache" in l for l in second)
    assert not any("compiled" in l for l in second)
    assert run("0") == []
