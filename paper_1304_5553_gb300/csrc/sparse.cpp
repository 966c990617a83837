// Sparse matrices and the conjugate-gradient solver (Sec. 3.2.6: GPU sparse
// matrices after Bell and Garland, and a CG-based Krylov solver for large sparse
// systems).
//
// CSR matrix-vector product: T lanes share a row (T in {1, 2, ..., 32}, from the
// mean row length or timed), lanes stride over the row's nonzeros, products are
// folded per lane and then across the T lanes by a shuffle tree.  Warps step
// over rows in lockstep (32 / T rows at a time), so the shuffles never diverge.
//
// CG (Hestenes and Stiefel) runs entirely on the device.  Set-up (r = b - Ax,
// p = r, r.r, b.b) uses the library's map and map-reduce kernels; each step is
// three kernels of this module -- q = Ap with p.q folded in; the x and r
// updates with r.r folded in (its last CTA also forms beta and counts the
// step); p = r + beta p -- and the step lengths stay in device memory, so the
// host reads the scalars back every 8 steps (a CUDA graph of 8 steps, two in
// flight, so the GPU does not wait for the host).  After convergence the updates
// freeze (zero step lengths).
#include <algorithm>
#include <iterator>
#include <cmath>
#include <map>
#include <mutex>
#include <string>

#include "cudrv.h"
#include "handles.h"
#include "kcache.h"

namespace pyc {

namespace {

const char* kSpmvSource = R"PYC(
// CSR y = A x with T lanes per row (generated for one value type V)
typedef long long pyc_i64;
// L2 eviction policies (createpolicy).  A CG step keeps the work vectors that fit
// in L2 together (evict_last) across its three kernels; the matrix, read once per
// step, and the vectors that do not fit go first (evict_first).
__device__ __forceinline__ unsigned long long pyc_pol(bool keep) {
  unsigned long long p;
  if (keep) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Loads with a policy: read-only data through the non-coherent path (not volatile,
// so that the compiler may batch them); stores are ordered.
__device__ __forceinline__ int pyc_ldnc(const int* a, unsigned long long pol) {
  int v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ pyc_i64 pyc_ldnc(const pyc_i64* a, unsigned long long pol) {
  pyc_i64 v;
  asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float pyc_ldnc(const float* a, unsigned long long pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ double pyc_ldnc(const double* a, unsigned long long pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void pyc_sth(float* a, float v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" :: "l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void pyc_sth(double* a, double v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" :: "l"(a), "d"(v), "l"(pol) : "memory");
}
// 16 bytes of V
struct __align__(16) pyc_vw {
  V v[16 / sizeof(V)];
};
// a thread loads and stores only its own 16-byte groups, so a load may move
// freely except past the store of the same group, which depends on it
__device__ __forceinline__ void pyc_ld16(const float* a, float* v, unsigned long long pol) {
  asm("ld.global.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(a), "l"(pol));
}
__device__ __forceinline__ void pyc_ld16(const double* a, double* v, unsigned long long pol) {
  asm("ld.global.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
      : "=d"(v[0]), "=d"(v[1]) : "l"(a), "l"(pol));
}
__device__ __forceinline__ void pyc_st16(float* a, const float* v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;"
               :: "l"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol) : "memory");
}
__device__ __forceinline__ void pyc_st16(double* a, const double* v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;"
               :: "l"(a), "d"(v[0]), "d"(v[1]), "l"(pol) : "memory");
}
__device__ __forceinline__ pyc_vw pyc_ldv(const pyc_vw* a, unsigned long long pol) {
  pyc_vw r;
  pyc_ld16(a->v, r.v, pol);
  return r;
}
__device__ __forceinline__ void pyc_stv(pyc_vw* a, const pyc_vw& r, unsigned long long pol) {
  pyc_st16(a->v, r.v, pol);
}
// Returns the L2 lines of [a, a + bytes) to normal eviction priority (after a
// solve, so that kept lines do not crowd later work).  Every 128-byte line
// visited holds at least one byte of the range.
extern "C" __global__ void __launch_bounds__(256) pyc_l2_release(const char* a,
    const pyc_i64 bytes) {
  const unsigned long long lo = (unsigned long long)a & ~127ull;
  const unsigned long long hi = (unsigned long long)a + (unsigned long long)bytes;
  const unsigned long long step = 128ull * gridDim.x * blockDim.x;
  for (unsigned long long l = lo + 128ull * (blockIdx.x * blockDim.x + threadIdx.x); l < hi;
       l += step)
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" :: "l"(l) : "memory");
}
template <int T>
__device__ __forceinline__ void pyc_spmv(const pyc_i64* __restrict__ rowptr,
    const int* __restrict__ col, const V* __restrict__ val, const V* __restrict__ x,
    V* __restrict__ y, const pyc_i64 nrows) {
  constexpr int R = 32 / T;  // rows per warp step
  const int lane = threadIdx.x & 31;
  const int sub = lane % T;
  const pyc_i64 warp = ((pyc_i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const pyc_i64 nwarps = ((pyc_i64)gridDim.x * blockDim.x) >> 5;
  for (pyc_i64 base = warp * R; base < nrows; base += nwarps * R) {
    const pyc_i64 r = base + lane / T;
    V s = 0;
    if (r < nrows) {
      const pyc_i64 b = rowptr[r], e = rowptr[r + 1];
      for (pyc_i64 k = b + sub; k < e; k += T) s += val[k] * __ldg(x + col[k]);
    }
#pragma unroll
    for (int d = T / 2; d >= 1; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d, T);
    if (sub == 0 && r < nrows) y[r] = s;
  }
}
#define PYC_SPMV(T) \
  extern "C" __global__ void __launch_bounds__(256) pyc_spmv_t##T(const pyc_i64* rowptr, \
      const int* col, const V* val, const V* x, V* y, const pyc_i64 nrows) { \
    pyc_spmv<T>(rowptr, col, val, x, y, nrows); \
  }
PYC_SPMV(1)
PYC_SPMV(2)
PYC_SPMV(4)
PYC_SPMV(8)
PYC_SPMV(16)
PYC_SPMV(32)

// Width 0: a sliced-ELL copy of the matrix.  Rows are taken in slices of 32;
// slice c holds m_c = (off[c+1] - off[c]) / 32 entries per row (its longest
// row), stored entry-major: entry j of row 32c + l at off[c] + 32 j + l, so a
// warp's 32 lanes read 128 consecutive bytes per entry and no row pointers.
// len[r] is row r's own length (LT: 1, 2 or 4 bytes); slots past it hold
// zeros and are loaded but never used.  Row r is added in entry order, as one
// lane per row adds it.
template <class LT>
__device__ __forceinline__ V pyc_sell_row(const pyc_i64* __restrict__ off,
    const int* __restrict__ scol, const V* __restrict__ sval, const LT* __restrict__ len,
    const V* __restrict__ x, const pyc_i64 c, const int l, const pyc_i64 nrows,
    const unsigned long long pm, const unsigned long long px) {
  const pyc_i64 o = pyc_ldnc(off + c, pm), m = (pyc_ldnc(off + c + 1, pm) - o) >> 5;
  const pyc_i64 r = c * 32 + l;
  const int lr = r < nrows ? (int)len[r] : 0;
  V y = 0;
  pyc_i64 j = 0;
  for (; j + 4 <= m; j += 4) {  // four entries' loads in flight, then added in order
    int ck[4];
    V vk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ck[u] = pyc_ldnc(scol + o + (j + u) * 32 + l, pm);
      vk[u] = pyc_ldnc(sval + o + (j + u) * 32 + l, pm);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (j + u < lr) y += vk[u] * pyc_ldnc(x + ck[u], px);
  }
  for (; j < m; ++j)
    if (j < lr) y += pyc_ldnc(sval + o + j * 32 + l, pm) * pyc_ldnc(x + pyc_ldnc(scol + o + j * 32 + l, pm), px);
  return y;
}
#define PYC_SELL(LT, TAG) \
  extern "C" __global__ void __launch_bounds__(256) pyc_spmv_sell_##TAG(const pyc_i64* off, \
      const int* scol, const V* sval, const LT* len, const V* x, V* y, const pyc_i64 nrows) { \
    const pyc_i64 warp = ((pyc_i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; \
    const pyc_i64 nwarps = ((pyc_i64)gridDim.x * blockDim.x) >> 5; \
    const int l = threadIdx.x & 31; \
    const unsigned long long pm = pyc_pol(false), px = pyc_pol(true); \
    for (pyc_i64 c = warp; c * 32 < nrows; c += nwarps) { \
      const V v = pyc_sell_row<LT>(off, scol, sval, len, x, c, l, nrows, pm, px); \
      if (c * 32 + l < nrows) y[c * 32 + l] = v; \
    } \
  }
PYC_SELL(unsigned char, u8)
PYC_SELL(unsigned short, u16)
PYC_SELL(unsigned, u32)
// Building the copy.  pyc_sell_len: len[r] and each slice's longest row
// (one warp per slice).  pyc_sell_fill: the entries, zeros past each row.
extern "C" __global__ void __launch_bounds__(256) pyc_sell_len(const pyc_i64* rowptr,
    const pyc_i64 nrows, int* cmax) {
  const pyc_i64 warp = ((pyc_i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const pyc_i64 nwarps = ((pyc_i64)gridDim.x * blockDim.x) >> 5;
  const int l = threadIdx.x & 31;
  for (pyc_i64 c = warp; c * 32 < nrows; c += nwarps) {
    const pyc_i64 r = c * 32 + l;
    int len = r < nrows ? (int)(rowptr[r + 1] - rowptr[r]) : 0;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, d));
    if (l == 0) cmax[c] = len;
  }
}
template <class LT>
__device__ __forceinline__ void pyc_sell_fill(const pyc_i64* rowptr, const int* col,
    const V* val, const pyc_i64 nrows, const pyc_i64* off, int* scol, V* sval, LT* len) {
  const pyc_i64 warp = ((pyc_i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const pyc_i64 nwarps = ((pyc_i64)gridDim.x * blockDim.x) >> 5;
  const int l = threadIdx.x & 31;
  for (pyc_i64 c = warp; c * 32 < nrows; c += nwarps) {
    const pyc_i64 o = off[c], m = (off[c + 1] - o) >> 5, r = c * 32 + l;
    const pyc_i64 b = r < nrows ? rowptr[r] : 0, lr = r < nrows ? rowptr[r + 1] - b : 0;
    if (r < nrows) len[r] = (LT)lr;
    for (pyc_i64 j = 0; j < m; ++j) {
      scol[o + j * 32 + l] = j < lr ? col[b + j] : 0;
      sval[o + j * 32 + l] = j < lr ? val[b + j] : (V)0;
    }
  }
}
#define PYC_SELL_FILL(LT, TAG) \
  extern "C" __global__ void __launch_bounds__(256) pyc_sell_fill_##TAG(const pyc_i64* rowptr, \
      const int* col, const V* val, const pyc_i64 nrows, const pyc_i64* off, int* scol, V* sval, \
      LT* len) { \
    pyc_sell_fill<LT>(rowptr, col, val, nrows, off, scol, sval, len); \
  }
PYC_SELL_FILL(unsigned char, u8)
PYC_SELL_FILL(unsigned short, u16)
PYC_SELL_FILL(unsigned, u32)

// ---- fused conjugate-gradient step: 3 kernels.  s[0] = r.r, s[1] = p.Ap,
// s[2] = tol^2, s[3] = new r.r, s[4] = b.b, s[5] = beta; it = steps taken.
// Dot products are finished deterministically: per-CTA partials, then the last
// CTA to arrive folds them in index order (fixed grid, fixed assignment).
__device__ __forceinline__ V pyc_block_sum(V v) {
  __shared__ V sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = 0;
  if (w == 0) {
    v = lane < nw ? sh[lane] : (V)0;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  }
  return v;  // thread 0: the block's sum
}
// Thread 0 of every CTA passes its sum; returns true (in every thread) in the
// last CTA to arrive, where *total = the partials folded in index order.
__device__ __forceinline__ bool pyc_grid_sum(V mine, V* part, unsigned* ticket, V* total) {
  __shared__ unsigned last;
  __shared__ V res;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = mine;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  V v = 0;
  for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) v += __ldcg(part + j);
  v = pyc_block_sum(v);
  if (threadIdx.x == 0) {
    res = v;
    *ticket = 0u;
  }
  __syncthreads();
  *total = res;
  return true;
}
// q = A p and s[1] = p.q.  keep: bit 0 p, bit 1 r, bit 2 q, bit 3 x stay in L2.
template <int T>
__device__ __forceinline__ void pyc_cg_a(const pyc_i64* __restrict__ rowptr,
    const int* __restrict__ col, const V* __restrict__ val, const V* __restrict__ p,
    V* __restrict__ q, const pyc_i64 nrows, V* part, unsigned* ticket, V* s,
    const unsigned keep) {
  const unsigned long long pm = pyc_pol(false), pp = pyc_pol(keep & 1u), pq = pyc_pol(keep & 4u);
  constexpr int R = 32 / T;
  const int lane = threadIdx.x & 31;
  const int sub = lane % T;
  const pyc_i64 warp = ((pyc_i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const pyc_i64 nwarps = ((pyc_i64)gridDim.x * blockDim.x) >> 5;
  V dot = 0;
  for (pyc_i64 base = warp * R; base < nrows; base += nwarps * R) {
    const pyc_i64 r = base + lane / T;
    V y = 0;
    if (r < nrows) {
      const pyc_i64 b = pyc_ldnc(rowptr + r, pm), e = pyc_ldnc(rowptr + r + 1, pm);
      for (pyc_i64 k = b + sub; k < e; k += T)
        y += pyc_ldnc(val + k, pm) * pyc_ldnc(p + pyc_ldnc(col + k, pm), pp);
    }
#pragma unroll
    for (int d = T / 2; d >= 1; d >>= 1) y += __shfl_down_sync(0xffffffffu, y, d, T);
    if (sub == 0 && r < nrows) {
      pyc_sth(q + r, y, pq);
      dot += pyc_ldnc(p + r, pp) * y;
    }
  }
  V tot;
  if (pyc_grid_sum(pyc_block_sum(dot), part, ticket, &tot) && threadIdx.x == 0) s[1] = tot;
}
#define PYC_CGA(T) \
  extern "C" __global__ void __launch_bounds__(256) pyc_cg_a_t##T(const pyc_i64* rowptr, \
      const int* col, const V* val, const V* p, V* q, const pyc_i64 nrows, V* part, \
      unsigned* ticket, V* s, const unsigned keep) { \
    pyc_cg_a<T>(rowptr, col, val, p, q, nrows, part, ticket, s, keep); \
  }
PYC_CGA(1)
PYC_CGA(2)
PYC_CGA(4)
PYC_CGA(8)
PYC_CGA(16)
PYC_CGA(32)
// width 0 (the sliced-ELL copy): q = A p and s[1] = p.q
#define PYC_CGA_SELL(LT, TAG) \
  extern "C" __global__ void __launch_bounds__(256) pyc_cg_a_sell_##TAG(const pyc_i64* off, \
      const int* scol, const V* sval, const LT* len, const V* p, V* q, const pyc_i64 nrows, \
      V* part, unsigned* ticket, V* s, const unsigned keep) { \
    const pyc_i64 warp = ((pyc_i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; \
    const pyc_i64 nwarps = ((pyc_i64)gridDim.x * blockDim.x) >> 5; \
    const int l = threadIdx.x & 31; \
    const unsigned long long pm = pyc_pol(false), pp = pyc_pol(keep & 1u), \
                             pq = pyc_pol(keep & 4u); \
    V dot = 0; \
    for (pyc_i64 c = warp; c * 32 < nrows; c += nwarps) { \
      const V y = pyc_sell_row<LT>(off, scol, sval, len, p, c, l, nrows, pm, pp); \
      const pyc_i64 r = c * 32 + l; \
      if (r < nrows) { \
        pyc_sth(q + r, y, pq); \
        dot += pyc_ldnc(p + r, pp) * y; \
      } \
    } \
    V tot; \
    if (pyc_grid_sum(pyc_block_sum(dot), part, ticket, &tot) && threadIdx.x == 0) s[1] = tot; \
  }
PYC_CGA_SELL(unsigned char, u8)
PYC_CGA_SELL(unsigned short, u16)
PYC_CGA_SELL(unsigned, u32)
// x += al p, r -= al q, s[3] = r.r; the last CTA sets beta and advances the step.
// VEC: 16-byte accesses with L2 policies (x 16-byte aligned; the work vectors
// always are).
template <bool VEC>
__device__ __forceinline__ void pyc_cg_b_body(V* __restrict__ x, V* __restrict__ r,
    const V* __restrict__ p, const V* __restrict__ q, const pyc_i64 n, V* part,
    unsigned* ticket, V* s, pyc_i64* it, const unsigned keep) {
  constexpr int W = 16 / sizeof(V);
  const V s0 = s[0], s1 = s[1], s2 = s[2];
  const bool go = s0 > s2;
  const V al = (go && s1 != 0) ? s0 / s1 : (V)0;
  V acc = 0;
  const pyc_i64 stride = (pyc_i64)gridDim.x * blockDim.x;
  const pyc_i64 t0 = (pyc_i64)blockIdx.x * blockDim.x + threadIdx.x;
  pyc_i64 done = 0;
  if (VEC) {
    const pyc_i64 nv = n / W;
    pyc_vw* xv = reinterpret_cast<pyc_vw*>(x);
    pyc_vw* rv = reinterpret_cast<pyc_vw*>(r);
    const pyc_vw* pv = reinterpret_cast<const pyc_vw*>(p);
    const pyc_vw* qv = reinterpret_cast<const pyc_vw*>(q);
    const unsigned long long pp = pyc_pol(keep & 1u), pr = pyc_pol(keep & 2u),
                             pq = pyc_pol(keep & 4u), px = pyc_pol(keep & 8u);
    for (pyc_i64 j = t0; j < nv; j += stride) {
      pyc_vw xa = pyc_ldv(xv + j, px), ra = pyc_ldv(rv + j, pr);
      const pyc_vw pa = pyc_ldv(pv + j, pp), qa = pyc_ldv(qv + j, pq);
#pragma unroll
      for (int l = 0; l < W; ++l) {
        xa.v[l] += al * pa.v[l];
        ra.v[l] -= al * qa.v[l];
        acc += ra.v[l] * ra.v[l];
      }
      pyc_stv(xv + j, xa, px);
      pyc_stv(rv + j, ra, pr);
    }
    done = nv * W;
  }
  for (pyc_i64 i = done + t0; i < n; i += stride) {
    x[i] += al * p[i];
    const V ri = r[i] - al * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  V tot;
  if (pyc_grid_sum(pyc_block_sum(acc), part, ticket, &tot) && threadIdx.x == 0) {
    s[3] = tot;
    s[5] = go ? tot / s0 : (V)0;
    if (go) {
      s[0] = tot;
      it[0] += 1;
    }
  }
}
extern "C" __global__ void __launch_bounds__(256) pyc_cg_b(V* x, V* r, const V* p,
    const V* q, const pyc_i64 n, V* part, unsigned* ticket, V* s, pyc_i64* it,
    const unsigned keep) {
  pyc_cg_b_body<true>(x, r, p, q, n, part, ticket, s, it, keep);
}
extern "C" __global__ void __launch_bounds__(256) pyc_cg_b_s(V* x, V* r, const V* p,
    const V* q, const pyc_i64 n, V* part, unsigned* ticket, V* s, pyc_i64* it,
    const unsigned keep) {
  pyc_cg_b_body<false>(x, r, p, q, n, part, ticket, s, it, keep);
}
// p = r + beta p (16-byte accesses; p and r are work vectors)
extern "C" __global__ void __launch_bounds__(256) pyc_cg_c(V* __restrict__ p,
    const V* __restrict__ r, const pyc_i64 n, const V* __restrict__ s, const unsigned keep) {
  constexpr int W = 16 / sizeof(V);
  const V be = s[5];
  const pyc_i64 stride = (pyc_i64)gridDim.x * blockDim.x;
  const pyc_i64 t0 = (pyc_i64)blockIdx.x * blockDim.x + threadIdx.x;
  const pyc_i64 nv = n / W;
  pyc_vw* pv = reinterpret_cast<pyc_vw*>(p);
  const pyc_vw* rv = reinterpret_cast<const pyc_vw*>(r);
  const unsigned long long pp = pyc_pol(keep & 1u), pr = pyc_pol(keep & 2u);
  for (pyc_i64 j = t0; j < nv; j += stride) {
    pyc_vw pa = pyc_ldv(pv + j, pp);
    const pyc_vw ra = pyc_ldv(rv + j, pr);
#pragma unroll
    for (int l = 0; l < W; ++l) pa.v[l] = ra.v[l] + be * pa.v[l];
    pyc_stv(pv + j, pa, pp);
  }
  for (pyc_i64 i = nv * W + t0; i < n; i += stride) p[i] = r[i] + be * p[i];
}
)PYC";

// Widths: lanes per row, or 0 for the sliced-ELL copy.
const int kWidths[] = {0, 1, 2, 4, 8, 16, 32};
constexpr int kMaxPartials = 4096;  // CTAs of one CG-step launch (per-CTA partial sums)

int default_width(int64_t nrows, int64_t nnz) {
  const double mean = nrows ? (double)nnz / (double)nrows : 1.0;
  int t = 1;
  while (t < 32 && 2 * t <= mean) t *= 2;
  return t;
}

}  // namespace

}  // namespace pyc

struct pyc_csr {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  CUdeviceptr rowptr = 0, col = 0, val = 0;
  pyc_dtype vt = PYC_F32;
  int width = 1;
  // width 0: the sliced-ELL copy (slice offsets, entries, values, row lengths of
  // s_lb bytes; s_lb = 0: no copy), built from the CSR arrays when selected
  CUdeviceptr s_off = 0, s_col = 0, s_val = 0, s_len = 0;
  int s_lb = 0;
  std::shared_ptr<pyc::Module> mod;
  // CG: step kernels (the library's map / map-reduce) and per-stream work space
  std::mutex mu;
  pyc_reduce_t dot = nullptr;
  pyc_map_t init_r = nullptr, copy = nullptr, set_tol = nullptr;
  struct Work {
    CUdeviceptr base = 0;
    int64_t n = 0;
    // a graph of 8 steps for one x pointer, captured on a private stream
    CUstream cap = nullptr;
    CUgraphExec graph = nullptr;
    CUdeviceptr graph_x = 0, graph_base = 0, graph_sell = 0;
    int graph_width = 0;
    // page-locked read-back slots of the device scalars, one event each
    unsigned char* host = nullptr;
    CUevent ev[2] = {nullptr, nullptr};
  };
  std::map<std::pair<CUcontext, CUstream>, Work> work;
};

namespace pyc {

namespace {

int vbytes(pyc_dtype t) { return t == PYC_F64 ? 8 : 4; }

const char* sell_tag(int lb) { return lb == 1 ? "u8" : lb == 2 ? "u16" : "u32"; }

void free_sell(pyc_csr* a) {
  for (CUdeviceptr* d : {&a->s_off, &a->s_col, &a->s_val, &a->s_len})
    if (*d) {
      drv().cuMemFree(*d);
      *d = 0;
    }
  a->s_lb = 0;
}

// Builds the sliced-ELL copy from the CSR arrays as they are now (on `s`,
// synchronously): slice lengths on the device, slice offsets on the host, then
// the entries.  With max_entries >= 0, a copy that would hold more padded
// entries than that is not built (returns false).
bool build_sell(pyc_csr* a, CUstream s, int64_t max_entries = -1) {
  free_sell(a);
  const int64_t n = a->nrows, nch = (n + 31) / 32;
  if (n == 0) {
    a->s_lb = 1;
    return true;
  }
  const Driver& d = drv();
  CUdeviceptr cmax = 0;
  PYC_CU(d.cuMemAlloc(&cmax, (size_t)(nch * 4)));
  try {
    CUfunction fl = a->mod->function("pyc_sell_len");
    const unsigned gl =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident_ctas(fl, 256), (nch + 7) / 8));
    int64_t nn = n;
    void* pl[] = {&a->rowptr, &nn, &cmax};
    PYC_CU(d.cuLaunchKernel(fl, gl, 1, 1, 256, 1, 1, 0, s, pl, nullptr));
    PYC_CU(d.cuStreamSynchronize(s));
    std::vector<int> hmax((size_t)nch);
    PYC_CU(d.cuMemcpyDtoH(hmax.data(), cmax, (size_t)(nch * 4)));
    std::vector<int64_t> off((size_t)nch + 1, 0);
    int mx = 0;
    for (int64_t c = 0; c < nch; ++c) {
      if (hmax[c] < 0) fail(PYC_E_ARG, "rowptr is not nondecreasing");
      off[c + 1] = off[c] + 32 * (int64_t)hmax[c];
      mx = std::max(mx, hmax[c]);
    }
    const int lb = mx <= 255 ? 1 : mx <= 65535 ? 2 : 4;
    const int64_t total = off[nch], vb = vbytes(a->vt);
    if (max_entries >= 0 && total > max_entries) {
      d.cuMemFree(cmax);
      return false;
    }
    PYC_CU(d.cuMemAlloc(&a->s_off, (size_t)((nch + 1) * 8)));
    PYC_CU(d.cuMemAlloc(&a->s_col, (size_t)std::max<int64_t>(total * 4, 4)));
    PYC_CU(d.cuMemAlloc(&a->s_val, (size_t)std::max<int64_t>(total * vb, vb)));
    PYC_CU(d.cuMemAlloc(&a->s_len, (size_t)(n * lb)));
    PYC_CU(d.cuMemcpyHtoD(a->s_off, off.data(), (size_t)((nch + 1) * 8)));
    CUfunction ff = a->mod->function(std::string("pyc_sell_fill_") + sell_tag(lb));
    void* pf[] = {&a->rowptr, &a->col, &a->val, &nn, &a->s_off, &a->s_col, &a->s_val, &a->s_len};
    PYC_CU(d.cuLaunchKernel(ff, gl, 1, 1, 256, 1, 1, 0, s, pf, nullptr));
    PYC_CU(d.cuStreamSynchronize(s));
    a->s_lb = lb;
  } catch (...) {
    d.cuMemFree(cmax);
    free_sell(a);
    throw;
  }
  d.cuMemFree(cmax);
  return true;
}

void launch_spmv(pyc_csr* a, int width, CUdeviceptr x, CUdeviceptr y, CUstream s) {
  if (a->nrows == 0) return;
  if (width == 0) {
    if (!a->s_lb) fail(PYC_E_INTERNAL, "width 0 without its sliced copy");
    CUfunction f = a->mod->function(std::string("pyc_spmv_sell_") + sell_tag(a->s_lb));
    const int64_t nch = (a->nrows + 31) / 32;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident_ctas(f, 256), (nch + 7) / 8));
    void* params[] = {&a->s_off, &a->s_col, &a->s_val, &a->s_len, &x, &y, &a->nrows};
    PYC_CU(drv().cuLaunchKernel(f, grid, 1, 1, 256, 1, 1, 0, s, params, nullptr));
    return;
  }
  CUfunction f = a->mod->function("pyc_spmv_t" + std::to_string(width));
  const int block = 256;
  const int64_t rows_per_block = (int64_t)(block / 32) * (32 / width);
  const int resident = resident_ctas(f, block);
  const int64_t need = (a->nrows + rows_per_block - 1) / rows_per_block;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, need));
  void* params[] = {&a->rowptr, &a->col, &a->val, &x, &y, &a->nrows};
  PYC_CU(drv().cuLaunchKernel(f, grid, 1, 1, block, 1, 1, 0, s, params, nullptr));
}

// Grid of a CG vector kernel: resident CTAs, at most one per 256 elements and
// at most kMaxPartials.
// Work vectors a CG step keeps in L2 (bit 0 p, bit 1 r, bit 2 q, bit 3 x, in
// order of use): as many as fit together in 9/16 of L2; the matrix streams
// through the rest.
unsigned cg_keep(int64_t vec_bytes) {
  const int64_t budget = (int64_t)current_device_props().l2_bytes * 9 / 16;
  unsigned keep = 0;
  int64_t used = 0;
  for (unsigned bit : {1u, 2u, 4u, 8u}) {
    if (used + vec_bytes > budget) break;
    used += vec_bytes;
    keep |= bit;
  }
  return keep;
}

unsigned cg_grid(CUfunction f, int64_t units) {
  const int resident = resident_ctas(f, 256);
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)resident, (units + 255) / 256, (int64_t)kMaxPartials}));
}

void make_cg_kernels(pyc_csr* a) {
  std::lock_guard<std::mutex> lk(a->mu);
  if (a->dot) return;
  const std::string T = a->vt == PYC_F64 ? "double" : "float";
  auto mk = [&](const std::string& spec, const std::string& stmt, const char* name) {
    pyc_map_t h = nullptr;
    pyc_status st = pyc_map_create(spec.c_str(), stmt.c_str(), name, nullptr, &h);
    if (st != PYC_OK) throw Error(st, pyc_last_error());
    return h;
  };
  // s[0] = rs (r.r), s[1] = p.Ap, s[2] = tol^2, s[3] = r.r after the update, s[4] = b.b
  pyc_status st = pyc_reduce_create(a->vt, "0", "a+b", "x[i]*y[i]",
                                    (T + " *x, " + T + " *y").c_str(), nullptr, &a->dot);
  if (st != PYC_OK) throw Error(st, pyc_last_error());
  a->init_r = mk(T + " *r, " + T + " *b, " + T + " *q", "r[i] = b[i] - q[i]", "cg_init");
  a->copy = mk(T + " *d, " + T + " *s", "d[i] = s[i]", "cg_copy");
  a->set_tol = mk(T + " *s, double rtol2", "if (i == 0) s[2] = (" + T + ")(rtol2 * (double)s[4])",
                  "cg_tol");
}

pyc_csr::Work& cg_work(pyc_csr* a, CUstream s, int64_t n) {
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(a->mu);
  auto& w = a->work[std::make_pair(ctx, s)];
  if (w.n < n) {
    if (w.base) {
      PYC_CU(drv().cuStreamSynchronize(s));
      drv().cuMemFree(w.base);
      w.base = 0;
      w.n = 0;  // until the new block exists (an allocation below may fail)
    }
    const int64_t vb = (int64_t)vbytes(a->vt);
    const int64_t vec = (n * vb + 255) / 256 * 256;
    PYC_CU(drv().cuMemAlloc(&w.base, (size_t)(3 * vec + 256 + kMaxPartials * vb)));
    w.n = n;
  }
  return w;
}

void map_launch(pyc_map_t h, int64_t n, std::initializer_list<CUdeviceptr> ptrs,
                const void* scalars, CUstream s) {
  std::vector<void*> p;
  for (CUdeviceptr d : ptrs) p.push_back(reinterpret_cast<void*>(d));
  pyc_status st = pyc_map_launch(h, n, p.data(), scalars, s);
  if (st != PYC_OK) throw Error(st, pyc_last_error());
}

void dot_launch(pyc_reduce_t h, int64_t n, CUdeviceptr x, CUdeviceptr y, CUdeviceptr out,
                CUstream s) {
  void* p[] = {reinterpret_cast<void*>(x), reinterpret_cast<void*>(y)};
  pyc_status st = pyc_reduce_launch(h, n, p, nullptr, reinterpret_cast<void*>(out), s);
  if (st != PYC_OK) throw Error(st, pyc_last_error());
}

}  // namespace

}  // namespace pyc

using namespace pyc;

namespace {
// Device arrays must be aligned to their element size: a kernel given a
// misaligned one would fault, so it is an argument error here.
void check_aligned(const void* p, int64_t bytes, const char* what) {
  if (reinterpret_cast<uintptr_t>(p) % (uintptr_t)bytes)
    fail(PYC_E_ARG, std::string(what) + " is not aligned to its element size");
}
}  // namespace

PYC_API pyc_status pyc_csr_create(int64_t nrows, int64_t ncols, int64_t nnz, const void* rowptr,
                                  const void* colidx, const void* vals, pyc_dtype vt,
                                  pyc_csr_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (nrows < 0 || ncols < 0 || nnz < 0) fail(PYC_E_ARG, "negative size");
    if (ncols > 0x7fffffffLL) fail(PYC_E_ARG, "column indices are int32: ncols < 2^31");
    if (vt != PYC_F32 && vt != PYC_F64) fail(PYC_E_ARG, "values are F32 or F64");
    if (nrows > 0 && !rowptr) fail(PYC_E_ARG, "rowptr is NULL");
    if (nnz > 0 && (!colidx || !vals)) fail(PYC_E_ARG, "colidx / vals are NULL");
    check_aligned(rowptr, 8, "rowptr");
    check_aligned(colidx, 4, "colidx");
    check_aligned(vals, vt == PYC_F64 ? 8 : 4, "vals");
    auto a = std::make_unique<pyc_csr>();
    a->nrows = nrows;
    a->ncols = ncols;
    a->nnz = nnz;
    a->rowptr = reinterpret_cast<CUdeviceptr>(rowptr);
    a->col = reinterpret_cast<CUdeviceptr>(colidx);
    a->val = reinterpret_cast<CUdeviceptr>(vals);
    a->vt = vt;
    a->width = default_width(nrows, nnz);
    std::string src = std::string("#define V ") + (vt == PYC_F64 ? "double" : "float") + "\n" +
                      kSpmvSource;
    a->mod = get_module(src, true);
    *out = a.release();
  });
}

PYC_API pyc_status pyc_csr_width(pyc_csr_t a, int* width) {
  return guarded([&] {
    if (!a || !width) fail(PYC_E_ARG, "NULL argument");
    *width = a->width;
  });
}

PYC_API pyc_status pyc_csr_set_width(pyc_csr_t a, int width) {
  return guarded([&] {
    if (!a) fail(PYC_E_ARG, "matrix is NULL");
    if (std::find(std::begin(kWidths), std::end(kWidths), width) == std::end(kWidths))
      fail(PYC_E_ARG, "width is 0, 1, 2, 4, 8, 16 or 32");
    if (width == 0) {
      build_sell(a, nullptr);
    } else {
      free_sell(a);
    }
    a->width = width;
  });
}

PYC_API pyc_status pyc_spmv(pyc_csr_t a, const void* x, void* y, pyc_stream_t stream) {
  return guarded([&] {
    if (!a) fail(PYC_E_ARG, "matrix is NULL");
    if (a->nrows > 0 && (!x || !y)) fail(PYC_E_ARG, "x / y is NULL");
    check_aligned(x, vbytes(a->vt), "x");
    check_aligned(y, vbytes(a->vt), "y");
    launch_spmv(a, a->width, reinterpret_cast<CUdeviceptr>(x), reinterpret_cast<CUdeviceptr>(y),
                reinterpret_cast<CUstream>(stream));
  });
}

PYC_API pyc_status pyc_spmv_autotune(pyc_csr_t a, const void* x, void* y, pyc_stream_t stream) {
  return guarded([&] {
    if (!a) fail(PYC_E_ARG, "matrix is NULL");
    if (a->nrows == 0) return;
    if (!x || !y) fail(PYC_E_ARG, "x / y is NULL");
    check_aligned(x, vbytes(a->vt), "x");
    check_aligned(y, vbytes(a->vt), "y");
    CUstream s = reinterpret_cast<CUstream>(stream);
    CUevent e0, e1;
    PYC_CU(drv().cuEventCreate(&e0, CU_EVENT_DEFAULT));
    PYC_CU(drv().cuEventCreate(&e1, CU_EVENT_DEFAULT));
    float best = 1e30f;
    int best_w = a->width;
    for (int w : kWidths) {
      // the sliced copy is tried only while padding at most doubles the entries
      if (w == 0 && !build_sell(a, s, 2 * a->nnz + 32 * ((a->nrows + 31) / 32))) continue;
      for (int k = 0; k < 2; ++k)
        launch_spmv(a, w, reinterpret_cast<CUdeviceptr>(x), reinterpret_cast<CUdeviceptr>(y), s);
      PYC_CU(drv().cuEventRecord(e0, s));
      for (int k = 0; k < 5; ++k)
        launch_spmv(a, w, reinterpret_cast<CUdeviceptr>(x), reinterpret_cast<CUdeviceptr>(y), s);
      PYC_CU(drv().cuEventRecord(e1, s));
      PYC_CU(drv().cuEventSynchronize(e1));
      float ms = 0;
      PYC_CU(drv().cuEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms, best_w = w;
    }
    drv().cuEventDestroy(e0);
    drv().cuEventDestroy(e1);
    if (best_w != 0) free_sell(a);
    a->width = best_w;
  });
}

PYC_API pyc_status pyc_cg_solve(pyc_csr_t a, const void* b, void* x, double rtol, int64_t maxit,
                                pyc_stream_t stream, pyc_cg_info* info) {
  return guarded([&] {
    if (!a || !b || !x) fail(PYC_E_ARG, "NULL argument");
    if (a->nrows != a->ncols) fail(PYC_E_ARG, "CG needs a square matrix");
    check_aligned(b, vbytes(a->vt), "b");
    check_aligned(x, vbytes(a->vt), "x");
    if (!(rtol >= 0) || maxit < 0) fail(PYC_E_ARG, "rtol >= 0 and maxit >= 0");
    const int64_t n = a->nrows;
    CUstream s = reinterpret_cast<CUstream>(stream);
    make_cg_kernels(a);
    pyc_csr::Work& w = cg_work(a, s, n);
    const int64_t vb = vbytes(a->vt);
    const int64_t vec = (n * vb + 255) / 256 * 256;
    const CUdeviceptr r = w.base, p = w.base + vec, q = w.base + 2 * vec;
    const CUdeviceptr sc = w.base + 3 * vec;   // s[0..5]
    const CUdeviceptr it = sc + 8 * vb;       // iteration counter (int64)
    CUdeviceptr ticket = sc + 128;            // last-CTA ticket of the step kernels
    CUdeviceptr part = sc + 256;              // per-CTA partial sums
    int64_t nn = n;
    const CUdeviceptr bx = reinterpret_cast<CUdeviceptr>(b), xx = reinterpret_cast<CUdeviceptr>(x);
    CUdeviceptr xx_v = xx, sc_v = sc, it_v = it;
    PYC_CU(drv().cuMemsetD8Async(sc, 0, 256, s));
    int64_t iters = 0;
    double rs = 0, bb = 0, tol2 = 0;
    if (n > 0) {
      // r = b - A x, p = r, s[0] = r.r, s[4] = b.b, s[2] = rtol^2 b.b
      launch_spmv(a, a->width, xx, q, s);
      map_launch(a->init_r, n, {r, bx, q}, nullptr, s);
      map_launch(a->copy, n, {p, r}, nullptr, s);
      dot_launch(a->dot, n, r, r, sc, s);
      dot_launch(a->dot, n, bx, bx, sc + 4 * vb, s);
      const double rt2 = rtol * rtol;
      map_launch(a->set_tol, 1, {sc}, &rt2, s);
      const int64_t chunk = 8;
      CUfunction fa = a->width == 0
                          ? a->mod->function(std::string("pyc_cg_a_sell_") + sell_tag(a->s_lb))
                          : a->mod->function("pyc_cg_a_t" + std::to_string(a->width));
      // 16-byte accesses to x need a 16-byte aligned x (the work vectors are)
      CUfunction fb = a->mod->function(xx % 16 == 0 ? "pyc_cg_b" : "pyc_cg_b_s");
      CUfunction fc = a->mod->function("pyc_cg_c");
      const int64_t rows_per_cta = (int64_t)(256 / 32) * (a->width == 0 ? 32 : 32 / a->width);
      const unsigned ga = a->width == 0 ? cg_grid(fa, (n + 31) / 32 * 32)
                                        : cg_grid(fa, (n + rows_per_cta - 1) / rows_per_cta * 256);
      const int64_t wv = 16 / vb;  // elements per 16-byte access
      const unsigned gb = cg_grid(fb, (n + wv - 1) / wv), gc = cg_grid(fc, (n + wv - 1) / wv);
      CUdeviceptr pp = p, qq = q, rr = r;
      unsigned keep = cg_keep(n * vb);
      void* pa_csr[] = {&a->rowptr, &a->col, &a->val, &pp, &qq, &nn, &part, &ticket, &sc_v, &keep};
      void* pa_sell[] = {&a->s_off, &a->s_col, &a->s_val, &a->s_len, &pp, &qq, &nn,
                         &part, &ticket, &sc_v, &keep};
      void** pa = a->width == 0 ? pa_sell : pa_csr;
      void* pb[] = {&xx_v, &rr, &pp, &qq, &nn, &part, &ticket, &sc_v, &it_v, &keep};
      void* pc[] = {&pp, &rr, &nn, &sc_v, &keep};
      auto steps = [&](CUstream st, int64_t k) {
        for (int64_t j = 0; j < k; ++j) {
          // q = A p, s[1] = p.q
          PYC_CU(drv().cuLaunchKernel(fa, ga, 1, 1, 256, 1, 1, 0, st, pa, nullptr));
          // x += al p, r -= al q, s[3] = r.r, beta, step count
          PYC_CU(drv().cuLaunchKernel(fb, gb, 1, 1, 256, 1, 1, 0, st, pb, nullptr));
          // p = r + beta p
          PYC_CU(drv().cuLaunchKernel(fc, gc, 1, 1, 256, 1, 1, 0, st, pc, nullptr));
        }
      };
      {
        std::lock_guard<std::mutex> lk(a->mu);
        if (!w.host) {
          void* h = nullptr;
          PYC_CU(drv().cuMemAllocHost(&h, 256));
          w.host = static_cast<unsigned char*>(h);
          for (CUevent& e : w.ev) PYC_CU(drv().cuEventCreate(&e, CU_EVENT_DISABLE_TIMING));
        }
        if (w.graph && (w.graph_x != xx || w.graph_base != w.base || w.graph_width != a->width ||
                        w.graph_sell != a->s_col)) {
          drv().cuGraphExecDestroy(w.graph);
          w.graph = nullptr;
        }
        if (!w.graph && maxit >= chunk) {
          if (!w.cap) PYC_CU(drv().cuStreamCreate(&w.cap, CU_STREAM_NON_BLOCKING));
          PYC_CU(drv().cuStreamBeginCapture(w.cap, CU_STREAM_CAPTURE_MODE_RELAXED));
          CUgraph g = nullptr;
          try {
            steps(w.cap, chunk);
          } catch (...) {
            drv().cuStreamEndCapture(w.cap, &g);
            if (g) drv().cuGraphDestroy(g);
            throw;
          }
          PYC_CU(drv().cuStreamEndCapture(w.cap, &g));
          CUresult ir = drv().cuGraphInstantiateWithFlags(&w.graph, g, 0);
          drv().cuGraphDestroy(g);
          check(ir, "cuGraphInstantiateWithFlags");
          w.graph_x = xx;
          w.graph_base = w.base;
          w.graph_width = a->width;
          w.graph_sell = a->s_col;
        }
      }
      // read back s[0..5] and the step count of the chunk just queued
      auto readback = [&](int slot) {
        PYC_CU(drv().cuMemcpyDtoHAsync(w.host + 128 * slot, sc, 6 * vb, s));
        PYC_CU(drv().cuMemcpyDtoHAsync(w.host + 128 * slot + 64, it, 8, s));
        PYC_CU(drv().cuEventRecord(w.ev[slot], s));
      };
      auto consume = [&](int slot) {
        PYC_CU(drv().cuEventSynchronize(w.ev[slot]));
        const unsigned char* hb = w.host + 128 * slot;
        auto get = [&](int k) {
          return a->vt == PYC_F64 ? reinterpret_cast<const double*>(hb)[k]
                                  : (double)reinterpret_cast<const float*>(hb)[k];
        };
        rs = get(0);
        tol2 = get(2);
        bb = get(4);
        iters = *reinterpret_cast<const int64_t*>(hb + 64);
      };
      readback(0);
      consume(0);
      // two chunks in flight: the GPU runs chunk c + 1 while the host checks c;
      // steps after convergence are frozen, so running ahead changes nothing
      int64_t launched = 0;
      int slot = 0, inflight = 0;
      int order[2];
      while (rs > tol2 && (launched < maxit || inflight > 0)) {
        while (inflight < 2 && launched < maxit) {
          const int64_t k = std::min<int64_t>(chunk, maxit - launched);
          if (k == chunk && w.graph) PYC_CU(drv().cuGraphLaunch(w.graph, s));
          else steps(s, k);
          readback(slot);
          order[inflight++] = slot;
          slot ^= 1;
          launched += k;
        }
        consume(order[0]);
        order[0] = order[1];
        --inflight;
      }
      while (inflight > 0) {  // let the queued chunks finish; keep the latest numbers
        consume(order[0]);
        order[0] = order[1];
        --inflight;
      }
      // kept vectors back to normal eviction priority
      CUfunction fr = a->mod->function("pyc_l2_release");
      const unsigned gr = cg_grid(fr, (n * vb + 127) / 128);
      const CUdeviceptr vecs[] = {p, r, q, xx};
      for (int k = 0; k < 4; ++k) {
        if (!(keep & (1u << k))) continue;
        CUdeviceptr v = vecs[k];
        int64_t bytes = n * vb;
        void* pr[] = {&v, &bytes};
        PYC_CU(drv().cuLaunchKernel(fr, gr, 1, 1, 256, 1, 1, 0, s, pr, nullptr));
      }
    }
    if (info) {
      info->iterations = iters;
      info->residual = bb > 0 ? std::sqrt(std::max(rs, 0.0) / bb) : std::sqrt(std::max(rs, 0.0));
      info->converged = n == 0 || !(rs > tol2) ? 1 : 0;
    }
  });
}

PYC_API void pyc_csr_destroy(pyc_csr_t a) {
  if (!a) return;
  try {
    for (auto& kv : a->work) {
      auto& w = kv.second;
      if (w.graph) drv().cuGraphExecDestroy(w.graph);
      if (w.cap) drv().cuStreamDestroy(w.cap);
      if (w.host) drv().cuMemFreeHost(w.host);
      for (CUevent e : w.ev)
        if (e) drv().cuEventDestroy(e);
      if (w.base) drv().cuMemFree(w.base);
    }
    pyc_reduce_destroy(a->dot);
    for (pyc_map_t h : {a->init_r, a->copy, a->set_tol})
      pyc_map_destroy(h);
    free_sell(a);
  } catch (...) {
  }
  delete a;
}
