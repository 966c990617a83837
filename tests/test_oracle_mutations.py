"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case plants one mistake in a copy of oracle/oracle.c (a dropped term, a
wrong sign, a transposed operand, a wrong rounding or tie rule, a wrong index),
builds it, and runs the pin tests against it (ORACLE_LIB): they must fail.  The
unmodified copy must pass, so a failure is the mistake's doing.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = [
    # (name, original text, mutated text)
    ("lin_comb drops b*y", "double v = p + q;", "double v = p;"),
    ("lin_comb sign", "double q = b * (double)y[i];", "double q = -b * (double)y[i];"),
    ("lin_comb transposed", "double p = a * (double)x[i];", "double p = a * (double)y[i];"),
    ("gauss_sin drops sin term", "    double v = a + b;\n    if (z64) z64[i] = v;\n    if (t1)",
     "    double v = a;\n    if (z64) z64[i] = v;\n    if (t1)"),
    ("gauss_sin exp sign", "double a = (double)x[i] * exp(-(yy * yy));\n    double b = sin((double)u[i]) * (double)w[i];\n    double v = a + b;\n    if (z64)",
     "double a = (double)x[i] * exp(yy * yy);\n    double b = sin((double)u[i]) * (double)w[i];\n    double v = a + b;\n    if (z64)"),
    ("bf16 rounds with 9 bits", "q = ldexp(nearbyint(ldexp(m, 8)), e - 8);",
     "q = ldexp(nearbyint(ldexp(m, 9)), e - 9);"),
    ("bf16 truncates", "q = ldexp(nearbyint(ldexp(m, 8)), e - 8);",
     "q = ldexp(floor(ldexp(m, 8)), e - 8);"),
    ("neumaier drops compensation", "  return s + c;\n}\n\n/* Listing 3b: map x[i]*y[i]",
     "  return s;\n}\n\n/* Listing 3b: map x[i]*y[i]"),
    ("dot squares x", "double t = (double)x[i] * (double)y[i];\n    neumaier_add(&s, &c, t);",
     "double t = (double)x[i] * (double)x[i];\n    neumaier_add(&s, &c, t);"),
    ("int sum skips first", "for (int64_t i = 0; i < n; ++i) s += (uint64_t)(int64_t)x[i];",
     "for (int64_t i = 1; i < n; ++i) s += (uint64_t)(int64_t)x[i];"),
    ("argmin last index on ties", "if (x[i] < bv || (x[i] == bv && i < bi)) { bv = x[i]; bi = i; }",
     "if (x[i] <= bv) { bv = x[i]; bi = i; }"),
    ("max uses >=", "    if (x[i] > m) m = x[i];\n  return m;\n}\n\nfloat orc_min_f32",
     "    if (x[i] < m) m = x[i];\n  return m;\n}\n\nfloat orc_min_f32"),
    ("superacc ties away from zero", "if (rem > half || (rem == half && (sticky || (q & 1)))) ++q;",
     "if (rem >= half) ++q;"),
    ("f32ops contracts", "    float v = p + q;\n    z[i] = out_bf16",
     "    float v = (float)((double)a * x[i] + (double)b * y[i]);\n    z[i] = out_bf16"),
    ("scan exclusive off by one", "    if (exclusive) out[i] = (int64_t)s;\n    s += (uint64_t)(int64_t)x[i];",
     "    s += (uint64_t)(int64_t)x[i];\n    if (exclusive) out[i] = (int64_t)s;"),
    ("scan records before adding", "    neumaier_add(&s, &c, (double)x[i]);\n    neumaier_add(&as, &ac, fabs((double)x[i]));\n    incl[i] = s + c;",
     "    incl[i] = s + c;\n    neumaier_add(&s, &c, (double)x[i]);\n    neumaier_add(&as, &ac, fabs((double)x[i]));"),
    ("affine composed in the wrong order", "    B = a[i] * B + b[i];", "    B = B + A * b[i];"),
    ("scan drops compensation", "    incl[i] = s + c;\n    if (abs_prefix)", "    incl[i] = s;\n    if (abs_prefix)"),
    ("running max keeps the first", "    if (x[i] > m) m = x[i];\n    out[i] = m;",
     "    if (m == -INFINITY) m = x[i];\n    out[i] = m;"),
]


def _build(src_text, path):
    c_path = path + ".c"
    open(c_path, "w").write(src_text)
    cmd = oracle.build_cmd()
    cmd[cmd.index(oracle.LIB_PATH)] = path
    cmd[cmd.index(os.path.join(os.path.dirname(oracle.__file__), "oracle.c"))] = c_path
    subprocess.run(cmd, check=True, capture_output=True)


def _pins_pass(lib_path):
    env = dict(os.environ, ORACLE_LIB=lib_path)
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, capture_output=True, text=True, cwd=ROOT)
    return p.returncode == 0


@pytest.fixture(scope="module")
def original():
    return open(SRC).read()


def test_unmodified_copy_passes(tmp_path, original):
    lib = str(tmp_path / "orig.so")
    _build(original, lib)
    assert _pins_pass(lib)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, original, name, old, new):
    assert original.count(old) == 1, "mutation anchor not unique: " + name
    lib = str(tmp_path / "mutant.so")
    _build(original.replace(old, new), lib)
    assert not _pins_pass(lib), "the pins did not catch: " + name
