/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, single-threaded CPU statement of what the map and map-reduce
 * path computes, used to judge the CUDA path.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the library never does.
 * It shares no code, header or constant with the CUDA path.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math (no contraction, IEEE
 * binary64, round to nearest even).
 *
 * What is computed (Klockner et al., "GPU Scripting and Code Generation with
 * PyCUDA"):
 *   Map (Sec. 3.2.4, Listing 3a): a statement is run for every value of the
 *     formal index i over equal-length arrays, in a single pass.  The oracle
 *     evaluates each configured statement in binary64 from the exact input
 *     values and rounds once to the output storage type.
 *   Map-reduce (Sec. 3.2.5, Listing 3b): r = R(...R(R(neutral, M(0)), M(1))...,
 *     M(n-1)) for an associative reduce expression R with neutral element.  For
 *     integer sums, max/min and argmin/argmax this is exact and independent of
 *     association order; floating-point sums are accumulated in binary64 with
 *     Neumaier compensation and also returned with sum |terms| so the caller
 *     can apply error bounds.  An exact superaccumulator is provided to check
 *     the compensated binary64 sums themselves.
 *
 * Parity pins: see tests/test_oracle_pins.py (closed forms, brute force with
 * exact rational arithmetic, library routines, invariants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ rounding */

/* Round a binary64 value to the nearest bfloat16 (8 significant bits, 8
 * exponent bits), ties to even, and return it as a double.  One rounding from
 * the exact binary64 value (no intermediate binary32 step). */
double orc_round_bf16(double d) {
  if (d != d || d == 0.0 || isinf(d)) return d;
  const double max_bf16 = 0x1.FEp127;     /* largest finite bfloat16 */
  const double min_normal = 0x1p-126;
  double a = fabs(d), q;
  if (a < min_normal) {
    q = nearbyint(a * 0x1p133) * 0x1p-133; /* subnormal spacing 2^-133 */
  } else {
    int e;
    double m = frexp(a, &e);               /* a = m * 2^e, m in [0.5, 1) */
    q = ldexp(nearbyint(ldexp(m, 8)), e - 8);
    /* the rounding boundary of the largest finite value: max + half ulp */
    if (q > max_bf16) q = INFINITY;
  }
  return d < 0 ? -q : q;
}

/* Round a binary64 value to binary32, nearest even (C conversion). */
float orc_round_f32(double d) { return (float)d; }

/* ------------------------------------------------------------ maps */

/* Listing 1 / Listing 2: z[i] = s * x[i]. */
void orc_map_scale(int64_t n, double s, const float* x, float* z, double* z64) {
  for (int64_t i = 0; i < n; ++i) {
    double v = s * (double)x[i];
    if (z64) z64[i] = v;
    z[i] = (float)v;
  }
}

/* Listing 4: tgt[i] = op1[i] + op2[i]. */
void orc_map_add(int64_t n, const float* x, const float* y, float* z, double* z64) {
  for (int64_t i = 0; i < n; ++i) {
    double v = (double)x[i] + (double)y[i];
    if (z64) z64[i] = v;
    z[i] = (float)v;
  }
}

/* Listing 3a: z[i] = a*x[i] + b*y[i].  Inputs are given as binary32 values
 * (bfloat16 inputs are exactly representable there).  out_bf16 selects the
 * output storage: 0 = binary32, 1 = bfloat16 (returned as binary32 values).
 * z64 receives the binary64 value, t_abs the sum |a*x[i]| + |b*y[i]|. */
void orc_map_lin_comb(int64_t n, double a, const float* x, double b, const float* y,
                      int out_bf16, float* z, double* z64, double* t_abs) {
  for (int64_t i = 0; i < n; ++i) {
    double p = a * (double)x[i];
    double q = b * (double)y[i];
    double v = p + q;
    if (z64) z64[i] = v;
    if (t_abs) t_abs[i] = fabs(p) + fabs(q);
    z[i] = out_bf16 ? (float)orc_round_bf16(v) : (float)v;
  }
}

/* Listing 3a as C source on binary32 operands: with the declared types every
 * operation rounds to binary32 in source order (no contraction):
 * z = RN32(RN32(a*x) + RN32(b*y)); out_bf16 = 1 rounds that binary32 value to
 * bfloat16 on the store.  Inputs given as binary32 values. */
void orc_map_lin_comb_f32ops(int64_t n, float a, const float* x, float b, const float* y,
                             int out_bf16, float* z) {
  for (int64_t i = 0; i < n; ++i) {
    float p = a * x[i];
    float q = b * y[i];
    float v = p + q;
    z[i] = out_bf16 ? (float)orc_round_bf16((double)v) : v;
  }
}

/* The four-input map z[i] = x[i]*exp(-y[i]*y[i]) + sin(u[i])*w[i].
 * t1 and t2 receive the two top-level addends in binary64. */
void orc_map_gauss_sin(int64_t n, const float* x, const float* y, const float* u,
                       const float* w, float* z, double* z64, double* t1, double* t2) {
  for (int64_t i = 0; i < n; ++i) {
    double yy = (double)y[i];
    double a = (double)x[i] * exp(-(yy * yy));
    double b = sin((double)u[i]) * (double)w[i];
    double v = a + b;
    if (z64) z64[i] = v;
    if (t1) t1[i] = a;
    if (t2) t2[i] = b;
    z[i] = (float)v;
  }
}

/* The same four-input map at selected indices only (for sampled checks of
 * very large outputs). */
void orc_map_gauss_sin_at(int64_t k, const int64_t* idx, const float* x, const float* y,
                          const float* u, const float* w, double* z64, double* t1,
                          double* t2) {
  for (int64_t j = 0; j < k; ++j) {
    int64_t i = idx[j];
    double yy = (double)y[i];
    double a = (double)x[i] * exp(-(yy * yy));
    double b = sin((double)u[i]) * (double)w[i];
    z64[j] = a + b;
    t1[j] = a;
    t2[j] = b;
  }
}

/* ------------------------------------------------------------ reductions */

/* Neumaier's improved Kahan summation in binary64.  Adds t into (s, c). */
static inline void neumaier_add(double* s, double* c, double t) {
  double u = *s + t;
  if (fabs(*s) >= fabs(t))
    *c += (*s - u) + t;
  else
    *c += (t - u) + *s;
  *s = u;
}

/* Listing 3b with reduce "a+b", neutral 0 and map x[i]: sum of binary32
 * values, accumulated in binary64 (compensated).  *abs_sum = sum |x[i]|. */
double orc_sum_f32(int64_t n, const float* x, double* abs_sum) {
  double s = 0.0, c = 0.0, as = 0.0, ac = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    neumaier_add(&s, &c, (double)x[i]);
    neumaier_add(&as, &ac, fabs((double)x[i]));
  }
  if (abs_sum) *abs_sum = as + ac;
  return s + c;
}

/* Listing 3b: map x[i]*y[i], reduce a+b, neutral 0.  The product of two
 * binary32 values is exact in binary64 (24 + 24 <= 53 significant bits). */
double orc_dot_f32(int64_t n, const float* x, const float* y, double* abs_sum) {
  double s = 0.0, c = 0.0, as = 0.0, ac = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = (double)x[i] * (double)y[i];
    neumaier_add(&s, &c, t);
    neumaier_add(&as, &ac, fabs(t));
  }
  if (abs_sum) *abs_sum = as + ac;
  return s + c;
}

/* Dot products over consecutive segments [off[s], off[s+1]) of x and y. */
void orc_dot_segments_f32(int64_t nseg, const int64_t* off, const float* x, const float* y,
                          double* out, double* abs_out) {
  for (int64_t s = 0; s < nseg; ++s) {
    int64_t a = off[s], len = off[s + 1] - off[s];
    out[s] = orc_dot_f32(len, x + a, y + a, abs_out ? &abs_out[s] : NULL);
  }
}

/* Integer sum of int32 values into a 64-bit accumulator with two's-complement
 * wrap-around (unsigned arithmetic). */
int64_t orc_sum_i32_i64(int64_t n, const int32_t* x) {
  uint64_t s = 0;
  for (int64_t i = 0; i < n; ++i) s += (uint64_t)(int64_t)x[i];
  return (int64_t)s;
}

/* Integer dot product of int32 vectors into int64 (wrap-around). */
int64_t orc_dot_i32_i64(int64_t n, const int32_t* x, const int32_t* y) {
  uint64_t s = 0;
  for (int64_t i = 0; i < n; ++i) s += (uint64_t)((int64_t)x[i] * (int64_t)y[i]);
  return (int64_t)s;
}

/* Max and min with neutral -inf / +inf (reduce expression "a > b ? a : b"). */
float orc_max_f32(int64_t n, const float* x) {
  float m = -INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (x[i] > m) m = x[i];
  return m;
}

float orc_min_f32(int64_t n, const float* x) {
  float m = INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (x[i] < m) m = x[i];
  return m;
}

/* argmin / argmax (Sec. 3.2.5): the fold r = R(r, (x[i], i)) from the neutral
 * element, where R keeps the smaller (larger) value and, on equal values, the
 * smaller index.  The neutral element that makes R an identity is
 * (+inf / -inf, INT64_MAX); it is the result for n == 0.  Scanning upward,
 * the first occurrence of the extremum wins. */
void orc_argmin_f32(int64_t n, const float* x, float* v, int64_t* idx) {
  float bv = INFINITY;
  int64_t bi = INT64_MAX;
  for (int64_t i = 0; i < n; ++i)
    if (x[i] < bv || (x[i] == bv && i < bi)) { bv = x[i]; bi = i; }
  *v = bv;
  *idx = bi;
}

void orc_argmax_f32(int64_t n, const float* x, float* v, int64_t* idx) {
  float bv = -INFINITY;
  int64_t bi = INT64_MAX;
  for (int64_t i = 0; i < n; ++i)
    if (x[i] > bv || (x[i] == bv && i < bi)) { bv = x[i]; bi = i; }
  *v = bv;
  *idx = bi;
}

/* ------------------------------------------------------------ scans */

/* Parallel prefix sums (Sec. 3.2.6) with scan expression a+b over binary32
 * values: incl[i] = x[0] + ... + x[i] accumulated in binary64 (compensated,
 * as orc_sum_f32), abs_prefix[i] = |x[0]| + ... + |x[i]| for error bounds. */
void orc_scan_sum_f32(int64_t n, const float* x, double* incl, double* abs_prefix) {
  double s = 0.0, c = 0.0, as = 0.0, ac = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    neumaier_add(&s, &c, (double)x[i]);
    neumaier_add(&as, &ac, fabs((double)x[i]));
    incl[i] = s + c;
    if (abs_prefix) abs_prefix[i] = as + ac;
  }
}

/* Prefix sums of int32 values into int64 with two's-complement wrap-around:
 * inclusive (out[i] = x[0] + ... + x[i]) or exclusive (out[i] = x[0] + ... +
 * x[i-1], out[0] = 0, the neutral element). */
void orc_scan_sum_i32_i64(int64_t n, const int32_t* x, int exclusive, int64_t* out) {
  uint64_t s = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (exclusive) out[i] = (int64_t)s;
    s += (uint64_t)(int64_t)x[i];
    if (!exclusive) out[i] = (int64_t)s;
  }
}

/* Running maximum from the neutral element -inf (scan expression a > b ? a : b). */
void orc_scan_max_f32(int64_t n, const float* x, float* out) {
  float m = -INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] > m) m = x[i];
    out[i] = m;
  }
}

/* A scan whose operator does not commute: composition of the affine maps
 * f_k(v) = a[k] v + b[k] (mod 2^32), applied in index order.  The prefix up to
 * i is the map v -> A_i v + B_i with A_i = A_{i-1} a[i], B_i = a[i] B_{i-1} +
 * b[i] (A_{-1} = 1, B_{-1} = 0: the identity map), stored as A_i << 32 | B_i. */
void orc_scan_affine_u32(int64_t n, const uint32_t* a, const uint32_t* b, uint64_t* out) {
  uint32_t A = 1u, B = 0u;
  for (int64_t i = 0; i < n; ++i) {
    A = A * a[i];
    B = a[i] * B + b[i];
    out[i] = ((uint64_t)A << 32) | B;
  }
}

/* ------------------------------------------------------- superaccumulator */

/* Exact sum of binary64 values.  The accumulator is a signed fixed-point
 * integer with 32-bit limbs: limb j weighs 2^(32*j - 1074), which covers every
 * finite binary64 (smallest subnormal 2^-1074, largest < 2^1024) plus carry
 * headroom.  Each finite term m * 2^e (|m| < 2^53 integer, e >= -1074) is added
 * exactly into three limbs; carries are normalised periodically; the final
 * value is rounded once to binary64, ties to even.  Returns the correctly
 * rounded sum (NaN if any term is not finite). */
#define SA_LIMBS 72
typedef struct {
  int64_t limb[SA_LIMBS];
  int64_t pending;
  int bad;
} superacc;

static void sa_normalise(superacc* a) {
  int64_t carry = 0;
  for (int j = 0; j < SA_LIMBS; ++j) {
    int64_t v = a->limb[j] + carry;
    int64_t lo = v & 0xFFFFFFFFLL;     /* in [0, 2^32) */
    carry = (v - lo) / 4294967296LL;   /* exact: v - lo is a multiple of 2^32 */
    a->limb[j] = lo;
  }
  a->limb[SA_LIMBS - 1] += carry * 4294967296LL; /* sign lives in the top limb */
  a->pending = 0;
}

static void sa_add(superacc* a, double t) {
  if (!isfinite(t)) { a->bad = 1; return; }
  if (t == 0.0) return;
  int e;
  double m = frexp(fabs(t), &e);          /* |t| = m * 2^e, m in [0.5, 1) */
  /* integer significand M (53 bits) and its bit position p >= 0 */
  int64_t M = (int64_t)ldexp(m, 53);
  int p = e - 53 + 1074;
  if (p < 0) { M >>= -p; p = 0; }        /* subnormals: exact, low bits are zero */
  int j = p / 32, r = p % 32;
  unsigned __int128 v = (unsigned __int128)(uint64_t)M << r; /* < 2^85 */
  int64_t l0 = (int64_t)(uint64_t)(v & 0xFFFFFFFFu);
  int64_t l1 = (int64_t)(uint64_t)((v >> 32) & 0xFFFFFFFFu);
  int64_t l2 = (int64_t)(uint64_t)(v >> 64);
  if (t < 0) { l0 = -l0; l1 = -l1; l2 = -l2; }
  a->limb[j] += l0;
  if (j + 1 < SA_LIMBS) a->limb[j + 1] += l1;
  if (j + 2 < SA_LIMBS) a->limb[j + 2] += l2;
  if (++a->pending >= (1 << 28)) sa_normalise(a);
}

static double sa_round(superacc* a) {
  if (a->bad) return NAN;
  sa_normalise(a);
  int neg = a->limb[SA_LIMBS - 1] < 0;
  if (neg) { /* magnitude: negate and renormalise */
    for (int j = 0; j < SA_LIMBS; ++j) a->limb[j] = -a->limb[j];
    sa_normalise(a);
  }
  int top = -1;
  for (int j = SA_LIMBS - 1; j >= 0; --j)
    if (a->limb[j] != 0) { top = j; break; }
  if (top < 0) return 0.0;
  /* top three limbs as a 96-bit integer V, weight 2^(32*(top-2) - 1074) */
  unsigned __int128 V = 0;
  int sticky = 0;
  for (int j = top; j >= top - 2; --j) {
    V <<= 32;
    if (j >= 0) V |= (uint64_t)a->limb[j];
  }
  for (int j = top - 3; j >= 0; --j)
    if (a->limb[j] != 0) { sticky = 1; break; }
  int bitlen = 0;
  for (unsigned __int128 t = V; t; t >>= 1) ++bitlen;
  int base = 32 * (top - 2) - 1074;
  int s = bitlen - 53;
  uint64_t q;
  if (s > 0) {
    unsigned __int128 rem = V & (((unsigned __int128)1 << s) - 1);
    unsigned __int128 half = (unsigned __int128)1 << (s - 1);
    q = (uint64_t)(V >> s);
    if (rem > half || (rem == half && (sticky || (q & 1)))) ++q;
    if (q == ((uint64_t)1 << 53)) { q >>= 1; ++s; }
  } else {
    q = (uint64_t)V; /* exact (sticky is 0 since lower limbs lie below V) */
    s = 0;
  }
  double r = ldexp((double)q, s + base);
  return neg ? -r : r;
}

double orc_exact_sum_f64(int64_t n, const double* t) {
  superacc* a = (superacc*)calloc(1, sizeof(superacc));
  for (int64_t i = 0; i < n; ++i) sa_add(a, t[i]);
  double r = sa_round(a);
  free(a);
  return r;
}

/* Exact dot product of binary32 vectors (each product exact in binary64),
 * correctly rounded to binary64. */
double orc_exact_dot_f32(int64_t n, const float* x, const float* y) {
  superacc* a = (superacc*)calloc(1, sizeof(superacc));
  for (int64_t i = 0; i < n; ++i) sa_add(a, (double)x[i] * (double)y[i]);
  double r = sa_round(a);
  free(a);
  return r;
}

/* Exact sum of binary32 values, correctly rounded to binary64. */
double orc_exact_sum_f32(int64_t n, const float* x) {
  superacc* a = (superacc*)calloc(1, sizeof(superacc));
  for (int64_t i = 0; i < n; ++i) sa_add(a, (double)x[i]);
  double r = sa_round(a);
  free(a);
  return r;
}
