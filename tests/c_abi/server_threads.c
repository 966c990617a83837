/* Many client threads on one serving loop, with the loop's batches executed on
 * the host (pyc_server_create_host), so that the scheduler's shared state --
 * queue, admission budget, batch slots, result hand-off, release -- is driven
 * concurrently without a GPU.  Built against a ThreadSanitizer-instrumented
 * build of the library by tests/test_race_cpu.py, which requires a clean run.
 *
 * Every client first creates a handle of one new spec at the same moment
 * (the kernel cache compiles it once and the others wait for that result).
 * Eight clients each submit 300 requests (dot products and z = a*x + b*y maps
 * at random offsets and lengths, outputs allocated by the server), poll them
 * in a scrambled order, check every result against the same computation done
 * here, and release them; a ninth thread reads the statistics throughout.
 * Prints "ok <completed> <batches>" and exits 0, or names the first mismatch
 * and exits 1. */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pyc.h"

#define POOL (1 << 16)
#define CLIENTS 8
#define PER_CLIENT 300
#define WINDOW 24

static float g_x[POOL], g_y[POOL];
static pyc_server_t g_srv;
static pyc_map_t g_map;
static pyc_reduce_t g_dot;
static volatile int g_clients_done;
static const float A = 2.5f, B = -0.75f;

/* per-thread pseudo-random numbers (xorshift32) */
static unsigned next_u32(unsigned* s) {
  unsigned v = *s;
  v ^= v << 13;
  v ^= v >> 17;
  v ^= v << 5;
  return *s = v;
}

/* The executor: one call per request, on the loop's executor thread. */
static int exec_fn(void* user, const pyc_request* req, void* value) {
  const float* x = (const float*)req->ptrs[0];
  const float* y = (const float*)req->ptrs[1];
  int64_t i;
  (void)user;
  if (req->kind == PYC_REQ_REDUCE) {
    double s = 0.0;
    for (i = 0; i < req->n; ++i) s += (double)x[i] * (double)y[i];
    *(float*)value = (float)s;
  } else {
    float a, b;
    float* z = (float*)req->ptrs[2];
    memcpy(&a, req->scalars, 4);
    memcpy(&b, (const char*)req->scalars + 4, 4);
    for (i = 0; i < req->n; ++i) z[i] = a * x[i] + b * y[i];
  }
  return PYC_OK;
}

typedef struct {
  uint64_t id;
  int kind;
  int64_t n, off;
  void* ptrs[3];
  float scal[2];
} Pending;

static int check(const Pending* p, const pyc_result* r) {
  int64_t i;
  if (r->status != PYC_OK) {
    fprintf(stderr, "request %llu failed: %d\n", (unsigned long long)p->id, r->status);
    return 1;
  }
  if (p->kind == PYC_REQ_REDUCE) {
    double s = 0.0;
    float got;
    for (i = 0; i < p->n; ++i) s += (double)g_x[p->off + i] * (double)g_y[p->off + i];
    memcpy(&got, r->value, 4);
    if (got != (float)s) {
      fprintf(stderr, "dot of request %llu: %g, want %g\n", (unsigned long long)p->id, got, s);
      return 1;
    }
  } else {
    const float* z = (const float*)r->d_out;
    if ((uintptr_t)z % 256 != (uintptr_t)(g_x + p->off) % 256) {
      fprintf(stderr, "output of request %llu is not at its input's alignment\n",
              (unsigned long long)p->id);
      return 1;
    }
    for (i = 0; i < p->n; ++i)
      if (z[i] != A * g_x[p->off + i] + B * g_y[p->off + i]) {
        fprintf(stderr, "map of request %llu differs at %lld\n", (unsigned long long)p->id,
                (long long)i);
        return 1;
      }
  }
  return 0;
}

static pthread_barrier_t g_start;

static void* client(void* arg) {
  unsigned seed = (unsigned)(uintptr_t)arg * 7919u + 17u;
  Pending pend[WINDOW];
  int npend = 0, k, sent = 0;
  pyc_map_t own;
  /* all clients at once: one compilation of this spec, shared */
  pthread_barrier_wait(&g_start);
  if (pyc_map_create("float *x, float *y", "y[i] = x[i] * 0.5f + 7.0f", NULL, NULL, &own) !=
      PYC_OK) {
    fprintf(stderr, "create in a thread: %s\n", pyc_last_error());
    exit(1);
  }
  pyc_map_destroy(own);
  while (sent < PER_CLIENT || npend > 0) {
    if (sent < PER_CLIENT && npend < WINDOW) {
      Pending* p = &pend[npend];
      pyc_request q;
      memset(&q, 0, sizeof q);
      p->kind = (next_u32(&seed) % 5 < 2) ? PYC_REQ_MAP : PYC_REQ_REDUCE;
      p->n = 1 + next_u32(&seed) % 3000;
      p->off = next_u32(&seed) % (POOL - p->n);
      p->ptrs[0] = g_x + p->off;
      p->ptrs[1] = g_y + p->off;
      p->ptrs[2] = NULL; /* map output: allocated by the server */
      p->scal[0] = A;
      p->scal[1] = B;
      q.kind = p->kind;
      q.handle = p->kind == PYC_REQ_MAP ? (void*)g_map : (void*)g_dot;
      q.n = p->n;
      q.ptrs = p->ptrs;
      q.scalars = p->kind == PYC_REQ_MAP ? (const void*)p->scal : NULL;
      if (pyc_server_submit(g_srv, &q, &p->id) != PYC_OK) {
        fprintf(stderr, "submit: %s\n", pyc_last_error());
        exit(1);
      }
      ++npend;
      ++sent;
      continue;
    }
    /* poll one pending request, picked pseudo-randomly, to the end */
    k = next_u32(&seed) % npend;
    {
      pyc_result r;
      pyc_status st = pyc_server_poll(g_srv, pend[k].id, &r, 10000000);
      if (st != PYC_OK) {
        fprintf(stderr, "poll: %d %s\n", st, pyc_last_error());
        exit(1);
      }
      if (check(&pend[k], &r)) exit(1);
      if (pyc_server_release(g_srv, pend[k].id) != PYC_OK) {
        fprintf(stderr, "release: %s\n", pyc_last_error());
        exit(1);
      }
      pend[k] = pend[--npend];
    }
  }
  return NULL;
}

static void* watcher(void* arg) {
  pyc_server_stats st;
  (void)arg;
  while (!__atomic_load_n(&g_clients_done, __ATOMIC_ACQUIRE)) {
    if (pyc_server_get_stats(g_srv, &st) != PYC_OK ||
        st.peak_admitted_bytes > ((int64_t)1 << 22)) {
      fprintf(stderr, "stats: admitted beyond the budget\n");
      exit(1);
    }
  }
  return NULL;
}

int main(void) {
  pthread_t th[CLIENTS + 1];
  pyc_server_cfg cfg;
  pyc_server_stats st;
  int k;
  for (k = 0; k < POOL; ++k) {
    g_x[k] = (float)((k * 37) % 101) * 0.125f - 6.0f;
    g_y[k] = (float)((k * 53) % 89) * 0.25f - 11.0f;
  }
  if (pyc_map_create("float a, float *x, float b, float *y, float *z", "z[i] = a*x[i] + b*y[i]",
                     "lin_comb", NULL, &g_map) != PYC_OK ||
      pyc_reduce_create(PYC_F32, "0", "a+b", "x[i]*y[i]", "float *x, float *y", NULL,
                        &g_dot) != PYC_OK) {
    fprintf(stderr, "create: %s\n", pyc_last_error());
    return 1;
  }
  memset(&cfg, 0, sizeof cfg);
  cfg.mem_budget_bytes = (int64_t)1 << 22; /* about 100 requests at a time */
  cfg.arena_bytes = (int64_t)1 << 22;
  cfg.max_batch = 16;
  cfg.max_inflight = 4;
  cfg.num_streams = 2;
  if (pyc_server_create_host(&cfg, exec_fn, NULL, &g_srv) != PYC_OK) {
    fprintf(stderr, "server: %s\n", pyc_last_error());
    return 1;
  }
  pthread_barrier_init(&g_start, NULL, CLIENTS);
  for (k = 0; k < CLIENTS; ++k) pthread_create(&th[k], NULL, client, (void*)(uintptr_t)k);
  pthread_create(&th[CLIENTS], NULL, watcher, NULL);
  for (k = 0; k < CLIENTS; ++k) pthread_join(th[k], NULL);
  __atomic_store_n(&g_clients_done, 1, __ATOMIC_RELEASE);
  pthread_join(th[CLIENTS], NULL);
  if (pyc_server_get_stats(g_srv, &st) != PYC_OK || st.completed != CLIENTS * PER_CLIENT ||
      st.failed != 0 || st.admitted_bytes != 0 || st.arena_in_use != 0) {
    fprintf(stderr, "final stats differ\n");
    return 1;
  }
  printf("ok %lld %lld\n", (long long)st.completed, (long long)st.batches);
  pthread_barrier_destroy(&g_start);
  pyc_server_destroy(g_srv);
  pyc_map_destroy(g_map);
  pyc_reduce_destroy(g_dot);
  return 0;
}
