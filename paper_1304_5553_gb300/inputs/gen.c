/*
 * Seeded synthetic input generator shared by the tests, the oracle checks and
 * the benchmark.  It holds none of the map / map-reduce arithmetic: it only
 * turns (seed, stream, index) into input values.
 *
 * Every value is a pure function of (seed, stream, element index), so any
 * slice of an array can be regenerated independently and filling in parallel
 * gives the same bits as filling serially.
 *
 * Bit source: the SplitMix64 output function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014; public
 * domain reference by S. Vigna), used counter-style:
 *     key(seed, stream) = mix(mix(seed) ^ (stream * 0xD1B54A32D192ED03))
 *     bits(seed, stream, i) = mix(key + (i + 1) * 0x9E3779B97F4A7C15)
 * where mix() is the SplitMix64 finaliser applied to the advanced state.
 *
 * Distributions (all documented with the workload recipe):
 *   uniform24      u = (bits >> 40) * 2^-24 in [0,1); lo + (hi-lo)*u, exact in
 *                  binary32 for [-1,1) and [-2,2)
 *   lognormal      Box-Muller in binary64 from two 53-bit draws, value
 *                  exp(sigma*z), sign from one more random bit, rounded to
 *                  binary32
 *   int uniform    lo + (bits >> 11) mod (hi - lo + 1), inclusive range
 *   log-uniform    floor(2^(lg_lo + lg_span * U)) clamped to [min, max]
 *   exponential    -ln(1 - U) / rate  (Poisson-process inter-arrival gaps)
 *   index sample   bits mod n  (sampling with replacement)
 *
 * Built as a plain C shared library (no CUDA); multithreaded fills use
 * pthreads and split the index range only.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL
#define STREAM_MUL 0xD1B54A32D192ED03ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* One step of the classic sequential SplitMix64 generator (state += gamma;
 * return mix(state)); exported so that the published reference sequence can
 * pin mix64. */
uint64_t pycgen_splitmix64_next(uint64_t* state) {
  *state += GAMMA;
  return mix64(*state);
}

static inline uint64_t key_of(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed) ^ (stream * STREAM_MUL));
}

static inline uint64_t bits_at(uint64_t key, uint64_t i) {
  return mix64(key + (i + 1) * GAMMA);
}

uint64_t pycgen_bits(uint64_t seed, uint64_t stream, uint64_t i) {
  return bits_at(key_of(seed, stream), i);
}

/* ---------------------------------------------------------------- threads */

typedef void (*fill_fn)(void* ctx, int64_t lo, int64_t hi);

typedef struct {
  fill_fn fn;
  void* ctx;
  int64_t lo, hi;
} slice_t;

static void* run_slice(void* p) {
  slice_t* s = (slice_t*)p;
  s->fn(s->ctx, s->lo, s->hi);
  return NULL;
}

static void parallel_fill(fill_fn fn, void* ctx, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < (int64_t)1 << 16 || nthreads == 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t tid[256];
  slice_t sl[256];
  int started[256];
  int64_t per = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = (int64_t)t * per, hi = lo + per;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
    sl[t].fn = fn; sl[t].ctx = ctx; sl[t].lo = lo; sl[t].hi = hi;
    started[t] = pthread_create(&tid[t], NULL, run_slice, &sl[t]) == 0;
    if (!started[t]) run_slice(&sl[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(tid[t], NULL);
}

/* ---------------------------------------------------------------- uniform */

typedef struct {
  uint64_t key, offset;
  double lo, span;
  float* out;
} unif_ctx;

static void unif_body(void* p, int64_t a, int64_t b) {
  unif_ctx* c = (unif_ctx*)p;
  for (int64_t j = a; j < b; ++j) {
    uint64_t k = bits_at(c->key, c->offset + (uint64_t)j) >> 40; /* 24 bits */
    double u = (double)k * 0x1p-24;
    c->out[j] = (float)(c->lo + c->span * u);
  }
}

/* out[j] = lo + (hi - lo) * u24(seed, stream, offset + j) */
void pycgen_uniform_f32(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n,
                        double lo, double hi, float* out, int nthreads) {
  unif_ctx c = {key_of(seed, stream), offset, lo, hi - lo, out};
  parallel_fill(unif_body, &c, n, nthreads);
}

/* -------------------------------------------------------------- lognormal */

typedef struct {
  uint64_t key, offset;
  double sigma;
  float* out;
} logn_ctx;

static void logn_body(void* p, int64_t a, int64_t b) {
  logn_ctx* c = (logn_ctx*)p;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t j = a; j < b; ++j) {
    uint64_t e = 2 * (c->offset + (uint64_t)j);
    uint64_t r1 = bits_at(c->key, e), r2 = bits_at(c->key, e + 1);
    double u1 = (double)((r1 >> 11) + 1) * 0x1p-53; /* (0, 1] */
    double u2 = (double)(r2 >> 11) * 0x1p-53;       /* [0, 1) */
    double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    double v = exp(c->sigma * z);
    if (r2 & 1) v = -v;
    c->out[j] = (float)v;
  }
}

/* out[j] = +-exp(sigma * N(0,1)), sign uniformly random. */
void pycgen_lognormal_signed_f32(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n,
                                 double sigma, float* out, int nthreads) {
  logn_ctx c = {key_of(seed, stream), offset, sigma, out};
  parallel_fill(logn_body, &c, n, nthreads);
}

/* ------------------------------------------------------------ integer draws */

typedef struct {
  uint64_t key, offset;
  int64_t lo;
  uint64_t range;
  int32_t* out32;
  int64_t* out64;
} int_ctx;

static void int_body(void* p, int64_t a, int64_t b) {
  int_ctx* c = (int_ctx*)p;
  for (int64_t j = a; j < b; ++j) {
    uint64_t r = bits_at(c->key, c->offset + (uint64_t)j) >> 11;
    int64_t v = c->lo + (int64_t)(r % c->range);
    if (c->out32) c->out32[j] = (int32_t)v;
    else c->out64[j] = v;
  }
}

/* out[j] uniform on the inclusive range [lo, hi]. */
void pycgen_int_uniform_i32(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n,
                            int64_t lo, int64_t hi, int32_t* out, int nthreads) {
  int_ctx c = {key_of(seed, stream), offset, lo, (uint64_t)(hi - lo + 1), out, NULL};
  parallel_fill(int_body, &c, n, nthreads);
}

/* out[j] = bits mod n_range: positions sampled with replacement. */
void pycgen_index_sample(uint64_t seed, uint64_t stream, uint64_t offset, int64_t k,
                         int64_t n_range, int64_t* out) {
  int_ctx c = {key_of(seed, stream), offset, 0, (uint64_t)n_range, NULL, out};
  int_body(&c, 0, k);
}

/* out[j] = clamp(floor(2^(lg_lo + lg_span * U)), vmin, vmax), U in [0,1). */
void pycgen_loguniform_i64(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n,
                           double lg_lo, double lg_span, int64_t vmin, int64_t vmax,
                           int64_t* out) {
  uint64_t key = key_of(seed, stream);
  for (int64_t j = 0; j < n; ++j) {
    double u = (double)(bits_at(key, offset + (uint64_t)j) >> 11) * 0x1p-53;
    double v = floor(exp2(lg_lo + lg_span * u));
    int64_t l = (int64_t)v;
    if (l < vmin) l = vmin;
    if (l > vmax) l = vmax;
    out[j] = l;
  }
}

/* out[j] = -ln(1 - U) / rate: exponential gaps of a Poisson process. */
void pycgen_exponential_f64(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n,
                            double rate, double* out) {
  uint64_t key = key_of(seed, stream);
  for (int64_t j = 0; j < n; ++j) {
    double u = (double)(bits_at(key, offset + (uint64_t)j) >> 11) * 0x1p-53;
    out[j] = -log1p(-u) / rate;
  }
}

/* out[j] = U in [0,1) with 53 bits (used for categorical choices). */
void pycgen_unit_f64(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n, double* out) {
  uint64_t key = key_of(seed, stream);
  for (int64_t j = 0; j < n; ++j)
    out[j] = (double)(bits_at(key, offset + (uint64_t)j) >> 11) * 0x1p-53;
}
