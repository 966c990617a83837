"""Build steps for the native parts of the package.

* ``libpyc.so``    -- the C-ABI library (C++ host code: spec parser, code
  generator, NVRTC driver + kernel cache, launches, batched reducer,
  autotuner; plus one nvcc-compiled sm_103a unit with the library's own
  device objects, linked with the static CUDA runtime).  Device code is generated per spec and compiled by
  NVRTC for sm_103a at run time; :func:`check_templates` compiles the stock
  templates ahead of time so that a template error fails the build.
* ``libpycgen.so`` -- the seeded input generator (plain C).

Everything is built in-tree under ``paper_1304_5553_gb300/_build`` with plain
compiler invocations (no cmake), so the same step works on x86_64 and aarch64.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(PKG_DIR, "_build")
CSRC = os.path.join(PKG_DIR, "csrc")
REPO_DIR = os.path.dirname(PKG_DIR)
INCLUDE_DIR = os.path.join(REPO_DIR, "include")
ARCH = "sm_103a"


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.isdir(os.path.join(cand, "include")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("CUDA toolkit not found (set CUDA_HOME)")


def pyc_lib_path() -> str:
    return os.path.join(BUILD_DIR, "libpyc.so")


def gen_lib_path() -> str:
    return os.path.join(BUILD_DIR, "libpycgen.so")


def _run(cmd):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s\n%s" % (" ".join(cmd), p.stdout, p.stderr))
    return p


def _newer(target, sources) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(s) <= t for s in sources)


def gen_cmd():
    src = os.path.join(PKG_DIR, "inputs", "gen.c")
    return [os.environ.get("CC", "gcc"), "-O2", "-std=c11", "-fPIC", "-shared", "-o",
            gen_lib_path(), src, "-lm", "-lpthread"], [src]


def _pyc_sources():
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.h"))) + \
        sorted(glob.glob(os.path.join(CSRC, "*.inc"))) + \
        sorted(glob.glob(os.path.join(INCLUDE_DIR, "*.h")))
    return srcs, hdrs


def _obj_path(src):
    return os.path.join(BUILD_DIR, "obj", os.path.basename(src) + ".o")


def _cu_sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def nvcc_path():
    p = os.path.join(cuda_home(), "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def pyc_compile_cmds():
    """One compile command per translation unit (run in parallel).  The .cpp
    files are host code (g++); the .cu files hold device objects of the library
    itself and are compiled by nvcc for sm_103a."""
    srcs, hdrs = _pyc_sources()
    inc = ["-I", INCLUDE_DIR, "-I", os.path.join(cuda_home(), "include")]
    base = [os.environ.get("CXX", "g++"), "-O2", "-std=c++17", "-fPIC",
            "-Wall", "-Wno-unused-function", "-fvisibility=hidden"] + inc
    cmds = [(_obj_path(s), base + ["-c", s, "-o", _obj_path(s)], [s] + hdrs) for s in srcs]
    for cu in _cu_sources():
        cmds.append((_obj_path(cu),
                     [nvcc_path(), "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
                      "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden"] + inc +
                     ["-I", CSRC, "-c", cu, "-o", _obj_path(cu)], [cu] + hdrs))
    return cmds


def pyc_link_cmd():
    srcs, _ = _pyc_sources()
    objs = [_obj_path(s) for s in srcs + _cu_sources()]
    libdir = os.path.join(cuda_home(), "lib64")
    return [os.environ.get("CXX", "g++"), "-shared", "-o", pyc_lib_path()] + objs + \
        ["-L", libdir, "-lcudart_static", "-ldl", "-lpthread", "-lrt"], objs


def build_gen(force=False):
    os.makedirs(BUILD_DIR, exist_ok=True)
    cmd, deps = gen_cmd()
    if force or not _newer(gen_lib_path(), deps):
        _run(cmd)
    return gen_lib_path()


def _run_parallel(steps, force):
    procs = []
    for target, cmd, deps in steps:
        if force or not _newer(target, deps):
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.PIPE, text=True)))
    errors = []
    for cmd, p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            errors.append("build step failed: %s\n%s\n%s" % (" ".join(cmd), out, err))
    if errors:
        raise RuntimeError("\n".join(errors))


def build_pyc(force=False):
    os.makedirs(os.path.join(BUILD_DIR, "obj"), exist_ok=True)
    _run_parallel(pyc_compile_cmds(), force)
    cmd, objs = pyc_link_cmd()
    if force or not _newer(pyc_lib_path(), objs):
        _run(cmd)
    return pyc_lib_path()


def build_all(force=False):
    """Compile every native library; translation units build in parallel."""
    os.makedirs(os.path.join(BUILD_DIR, "obj"), exist_ok=True)
    _run_parallel([(gen_lib_path(),) + gen_cmd()] + pyc_compile_cmds(), force)
    cmd, objs = pyc_link_cmd()
    if force or not _newer(pyc_lib_path(), objs):
        _run(cmd)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print("built", pyc_lib_path(), gen_lib_path())
