"""Error bounds used by the parity tests, each derived in its docstring from
the rounding of the operations it covers.

u = 2^-24 is the unit roundoff of binary32 (half an ulp at 1).
"""
import numpy as np

U = 2.0 ** -24
TINY = 2.0 ** -140  # absolute slack for subnormal results


def lin_comb_f32_bound(z64, t_abs):
    """z = RN(RN(a x) + RN(b y)) (or one FMA): |z - z64| <= u (|ax| + |by|)(1 + u) + u |z64|."""
    return U * t_abs * (1 + U) + U * np.abs(z64) + TINY


def lin_comb_bf16_bound(z64, t_abs):
    """binary32 evaluation then one rounding to bfloat16 (unit roundoff 2^-8)."""
    s = np.abs(z64) + 2 * U * t_abs
    return 2.0 ** -8 * s * (1 + 2.0 ** -7) + 2 * U * t_abs + TINY


def gauss_sin_bound(z64, t1, t2, y):
    """z = RN(RN(x expf(RN(-y y))) + RN(sinf(u) w)) with expf / sinf within 2 ulp
    (4u relative): |z - z64| <= (y^2 + 5) u |t1| + 5 u |t2| + u |z64|."""
    y = np.asarray(y, np.float64)
    return (y * y + 5) * U * np.abs(t1) * (1 + 8 * U) + 5 * U * np.abs(t2) * (1 + 8 * U) \
        + U * np.abs(z64) + TINY


def ulp32(v):
    v = np.abs(np.asarray(v, np.float32))
    return np.spacing(v).astype(np.float64)


def plain_sum_bound(abs_sum):
    """Stated tolerance of a plain binary32 reduction: 8 * 2^-24 * sum |terms|."""
    return 8 * U * abs_sum


def compensated_sum_bound(exact, abs_sum):
    """Stated tolerance of the compensated reduction: 4 u |S| + 2^-48 sum |terms|."""
    return 4 * U * abs(exact) + 2.0 ** -48 * abs_sum
