"""Race detection for the library's host-side concurrency (no GPU needed).

compute-sanitizer's racecheck is not available to these tests, and the
serving loop's shared state lives on the host anyway.  This test builds the
library's host code with ThreadSanitizer into a temporary directory, builds the
plain C driver tests/c_abi/server_threads.c against it, and runs it: eight
client threads submit, poll, check and release requests on one serving loop
whose batches run on the host (pyc_server_create_host), while another thread
reads its statistics.  The run must finish with every result correct and no
ThreadSanitizer report."""
import os
import shutil
import subprocess

import pytest

from paper_1304_5553_gb300 import buildlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tsan_works(tmp):
    src = os.path.join(tmp, "t.c")
    with open(src, "w") as f:
        f.write("int main(void) { return 0; }\n")
    p = subprocess.run(["gcc", "-fsanitize=thread", src, "-o", os.path.join(tmp, "t")],
                       capture_output=True)
    return p.returncode == 0 and subprocess.run([os.path.join(tmp, "t")]).returncode == 0


_RACY = r"""
#include <pthread.h>
static int counter;
static void* bump(void* a) { (void)a; for (int k = 0; k < 100000; ++k) ++counter; return 0; }
int main(void) {
  pthread_t t[2];
  for (int k = 0; k < 2; ++k) pthread_create(&t[k], 0, bump, 0);
  for (int k = 0; k < 2; ++k) pthread_join(t[k], 0);
  return 0;
}
"""


def test_thread_sanitizer_reports_a_planted_race(tmp_path):
    """Positive control: ThreadSanitizer, built as below, reports an unsynchronised
    counter shared by two threads."""
    tmp = str(tmp_path)
    if shutil.which("gcc") is None or not _tsan_works(tmp):
        pytest.skip("ThreadSanitizer is not available")
    src, exe = os.path.join(tmp, "racy.c"), os.path.join(tmp, "racy")
    with open(src, "w") as f:
        f.write(_RACY)
    p = subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fsanitize=thread", src, "-o", exe,
                        "-lpthread"], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120,
                         env=dict(os.environ, TSAN_OPTIONS="exitcode=66"))
    assert "WARNING: ThreadSanitizer: data race" in out.stderr
    assert out.returncode == 66


def test_serving_loop_under_thread_sanitizer(tmp_path):
    tmp = str(tmp_path)
    if shutil.which("gcc") is None or shutil.which("g++") is None or not _tsan_works(tmp):
        pytest.skip("ThreadSanitizer is not available")
    # the library's translation units: host code instrumented, the one .cu as usual
    objs, procs = [], []
    for obj, cmd, _ in buildlib.pyc_compile_cmds():
        out = os.path.join(tmp, os.path.basename(obj))
        cmd = [out if c == obj else c for c in cmd]
        if os.path.basename(cmd[0]).startswith(("g++", "c++", "clang")):
            cmd = cmd[:1] + ["-fsanitize=thread", "-g"] + [c for c in cmd[1:] if c != "-O2"] + \
                ["-O1"]
        objs.append(out)
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    for p in procs:
        _, err = p.communicate()
        assert p.returncode == 0, err[-3000:]
    lib = os.path.join(tmp, "libpyc.so")
    link, _ = buildlib.pyc_link_cmd()
    link = [link[0], "-shared", "-fsanitize=thread", "-o", lib] + objs + \
        [c for c in link[4 + len(objs):]]
    p = subprocess.run(link, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr[-3000:]
    exe = os.path.join(tmp, "server_threads")
    p = subprocess.run(["gcc", "-std=gnu11", "-O1", "-g", "-ffp-contract=off", "-fsanitize=thread",
                        "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi", "server_threads.c"), "-o", exe,
                        "-L", tmp, "-lpyc", "-lpthread", "-Wl,-rpath," + tmp],
                       capture_output=True, text=True)
    assert p.returncode == 0, p.stderr[-3000:]
    env = dict(os.environ, PYC_CACHE_DIR=os.path.join(tmp, "cache"),
               TSAN_OPTIONS="halt_on_error=1 exitcode=66 second_deadlock_stack=1")
    out = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=900)
    assert "ThreadSanitizer" not in out.stderr, out.stderr[-6000:]
    assert out.returncode == 0, out.stdout + out.stderr[-3000:]
    done, batches = (int(v) for v in out.stdout.split()[1:3])
    assert done == 8 * 300 and batches < done
