// Source generation for map and map-reduce kernels (see codegen.h).
//
// Kernel design (GB300, sm_103a; the path is HBM-bound, so no tensor cores):
//  * map: persistent grid-stride CTAs over tiles of blockDim * E * U elements.
//    Thread t of a tile owns U groups of E consecutive elements, group u at
//    tile_base + (u * blockDim + t) * E, so each vector instruction of a warp
//    covers one contiguous, fully coalesced span.  Lifted arrays move through
//    registers with 16- or 32-byte loads/stores (L1 no-allocate); the user
//    statement runs once per element on the register copies; a scalar loop
//    covers the unaligned head and the ragged tail.
//  * map-reduce: the index range is cut into chunks (a multiple of the tile).
//    A CTA folds a chunk with up to E*U independent accumulators per thread
//    (short serial chains; at most 128 bytes of them), combines them pairwise, then a warp-shuffle tree and a
//    shared-memory tree give the chunk's partial.  The last CTA to finish
//    (atomic ticket after a fence) combines the partials in index order and
//    writes the result: one launch, no host round trip.  Every order is a
//    fixed function of (n, tuning), so results are reproducible.
//  * batched map-reduce: one persistent launch over a work list of CTA items
//    (chunks of large segments) and warp bundles (one small segment per warp);
//    a per-segment ticket lets the last chunk of each segment finish it.
#include "codegen.h"
#include "kcache.h"

#include <sstream>

namespace pyc {

namespace {

const char* kPrelude = R"PYC(
// ---------------------------------------------------------------- pyc prelude
typedef long long pyc_i64;
typedef unsigned long long pyc_u64;
#ifndef INFINITY
#define INFINITY __int_as_float(0x7f800000)
#endif
#ifndef NAN
#define NAN __int_as_float(0x7fffffff)
#endif
#ifndef HUGE_VALF
#define HUGE_VALF INFINITY
#endif
#ifndef FLT_MAX
#define FLT_MAX 3.402823466e+38F
#endif
#ifndef FLT_MIN
#define FLT_MIN 1.175494351e-38F
#endif
#ifndef DBL_MAX
#define DBL_MAX 1.7976931348623158e+308
#endif
#ifndef INT_MAX
#define INT_MAX 2147483647
#endif
#ifndef INT_MIN
#define INT_MIN (-2147483647 - 1)
#endif
#ifndef UINT_MAX
#define UINT_MAX 4294967295U
#endif
#ifndef LLONG_MAX
#define LLONG_MAX 9223372036854775807LL
#endif
#ifndef LLONG_MIN
#define LLONG_MIN (-9223372036854775807LL - 1LL)
#endif
#ifndef ULLONG_MAX
#define ULLONG_MAX 18446744073709551615ULL
#endif

// bfloat16 / binary16 storage: read as binary32, rounded to nearest even on
// assignment (hardware cvt.rn).
__device__ __forceinline__ unsigned short pyc_f32_to_bf16_bits(float f) {
  unsigned short h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
  return h;
}
__device__ __forceinline__ unsigned short pyc_f32_to_f16_bits(float f) {
  unsigned short h;
  asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
  return h;
}
__device__ __forceinline__ float pyc_f16_bits_to_f32(unsigned short h) {
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
  return f;
}

struct pyc_bf16 {
  unsigned short bits;
  pyc_bf16() = default;
  __device__ __forceinline__ pyc_bf16(float f) : bits(pyc_f32_to_bf16_bits(f)) {}
  __device__ __forceinline__ operator float() const { return __uint_as_float(((unsigned)bits) << 16); }
  __device__ __forceinline__ pyc_bf16& operator=(float f) { bits = pyc_f32_to_bf16_bits(f); return *this; }
  __device__ __forceinline__ pyc_bf16& operator+=(float f) { return *this = float(*this) + f; }
  __device__ __forceinline__ pyc_bf16& operator-=(float f) { return *this = float(*this) - f; }
  __device__ __forceinline__ pyc_bf16& operator*=(float f) { return *this = float(*this) * f; }
  __device__ __forceinline__ pyc_bf16& operator/=(float f) { return *this = float(*this) / f; }
};

struct pyc_f16 {
  unsigned short bits;
  pyc_f16() = default;
  __device__ __forceinline__ pyc_f16(float f) : bits(pyc_f32_to_f16_bits(f)) {}
  __device__ __forceinline__ operator float() const { return pyc_f16_bits_to_f32(bits); }
  __device__ __forceinline__ pyc_f16& operator=(float f) { bits = pyc_f32_to_f16_bits(f); return *this; }
  __device__ __forceinline__ pyc_f16& operator+=(float f) { return *this = float(*this) + f; }
  __device__ __forceinline__ pyc_f16& operator-=(float f) { return *this = float(*this) - f; }
  __device__ __forceinline__ pyc_f16& operator*=(float f) { return *this = float(*this) * f; }
  __device__ __forceinline__ pyc_f16& operator/=(float f) { return *this = float(*this) / f; }
};

// (value, index) pair of argmin / argmax reductions (16 bytes).
struct pyc_argf32 {
  float v;
  int pad;
  long long i;
};

// compensated binary32 accumulator: value s plus running error c.
struct pyc_cf32 {
  float s;
  float c;
};

// Wide global accesses.  Loads skip L1 allocation (streamed once).
template <int B> struct pyc_vio;
template <> struct pyc_vio<16> {
  static __device__ __forceinline__ void ld(void* d, const void* s) {
    unsigned* r = reinterpret_cast<unsigned*>(d);
    asm volatile("ld.global.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(s));
  }
  static __device__ __forceinline__ void st(void* d, const void* s) {
    const unsigned* r = reinterpret_cast<const unsigned*>(s);
    asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};"
                 :: "l"(d), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]) : "memory");
  }
};
template <> struct pyc_vio<32> {
  static __device__ __forceinline__ void ld(void* d, const void* s) {
    unsigned* r = reinterpret_cast<unsigned*>(d);
    asm volatile("ld.global.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]),
                   "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "l"(s));
  }
  static __device__ __forceinline__ void st(void* d, const void* s) {
    const unsigned* r = reinterpret_cast<const unsigned*>(s);
    asm volatile("st.global.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "l"(d), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]),
                    "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]) : "memory");
  }
};
// G bytes in pieces of P bytes (G a multiple of P).
template <int G, int P>
__device__ __forceinline__ void pyc_ldg(void* d, const void* s) {
#pragma unroll
  for (int j = 0; j < G / P; ++j)
    pyc_vio<P>::ld(reinterpret_cast<char*>(d) + j * P, reinterpret_cast<const char*>(s) + j * P);
}
template <int G, int P>
__device__ __forceinline__ void pyc_stg(void* d, const void* s) {
#pragma unroll
  for (int j = 0; j < G / P; ++j)
    pyc_vio<P>::st(reinterpret_cast<char*>(d) + j * P, reinterpret_cast<const char*>(s) + j * P);
}

// Accesses with an L2 cache policy (createpolicy): 16- and 32-byte pieces.
template <int B> struct pyc_vioh;
template <> struct pyc_vioh<16> {
  static __device__ __forceinline__ void ld(void* d, const void* s, unsigned long long pol) {
    unsigned* r = reinterpret_cast<unsigned*>(d);
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(s), "l"(pol));
  }
  static __device__ __forceinline__ void st(void* d, const void* s, unsigned long long pol) {
    const unsigned* r = reinterpret_cast<const unsigned*>(s);
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;"
                 :: "l"(d), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "l"(pol) : "memory");
  }
};
template <> struct pyc_vioh<32> {
  static __device__ __forceinline__ void ld(void* d, const void* s, unsigned long long pol) {
    unsigned* r = reinterpret_cast<unsigned*>(d);
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]),
                   "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "l"(s), "l"(pol));
  }
  static __device__ __forceinline__ void st(void* d, const void* s, unsigned long long pol) {
    const unsigned* r = reinterpret_cast<const unsigned*>(s);
    asm volatile("st.global.L2::cache_hint.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8}, %9;"
                 :: "l"(d), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]),
                    "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "l"(pol) : "memory");
  }
};
template <int G, int P>
__device__ __forceinline__ void pyc_ldgh(void* d, const void* s, unsigned long long pol) {
#pragma unroll
  for (int j = 0; j < G / P; ++j)
    pyc_vioh<P>::ld(reinterpret_cast<char*>(d) + j * P, reinterpret_cast<const char*>(s) + j * P, pol);
}
template <int G, int P>
__device__ __forceinline__ void pyc_stgh(void* d, const void* s, unsigned long long pol) {
#pragma unroll
  for (int j = 0; j < G / P; ++j)
    pyc_vioh<P>::st(reinterpret_cast<char*>(d) + j * P, reinterpret_cast<const char*>(s) + j * P, pol);
}
__device__ __forceinline__ unsigned long long pyc_policy_keep() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long pyc_policy_drop() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Word-wise shuffle / L2 load of any trivially copyable 4-byte-multiple type.
template <typename T>
union pyc_words {
  T t;
  unsigned w[sizeof(T) / 4];
};
template <typename T>
__device__ __forceinline__ T pyc_shfl_down(const T v, int d) {
  static_assert(sizeof(T) % 4 == 0, "accumulator size must be a multiple of 4 bytes");
  pyc_words<T> u;
  u.t = v;
#pragma unroll
  for (int j = 0; j < (int)(sizeof(T) / 4); ++j) u.w[j] = __shfl_down_sync(0xffffffffu, u.w[j], d);
  return u.t;
}
template <typename T>
__device__ __forceinline__ T pyc_ld_cg(const T* p) {
  pyc_words<T> u;
  const unsigned* q = reinterpret_cast<const unsigned*>(p);
#pragma unroll
  for (int j = 0; j < (int)(sizeof(T) / 4); ++j)
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(u.w[j]) : "l"(q + j));
  return u.t;
}

// Fixed-shape trees: lane j combines with lane j+d (left operand = lower
// index), so the result does not depend on timing.
template <typename T, typename Op>
__device__ __forceinline__ T pyc_warp_reduce(T v, Op op) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    T o = pyc_shfl_down(v, d);
    v = op(v, o);
  }
  return v;  // valid in lane 0
}
template <typename T, typename Op>
__device__ __forceinline__ T pyc_block_reduce(T v, Op op, const T neutral) {
  __shared__ T pyc_sm[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = pyc_warp_reduce(v, op);
  __syncthreads();  // pyc_sm may still be read from a previous call
  if (lane == 0) pyc_sm[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? pyc_sm[lane] : neutral;
    v = pyc_warp_reduce(v, op);
  }
  return v;  // valid in thread 0
}

// Error-free transformation of a sum (Knuth's two-sum): s + e == a + b exactly.
__device__ __forceinline__ void pyc_two_sum(const float a, const float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
__device__ __forceinline__ void pyc_two_sum_d(const double a, const double b, double& s, double& e) {
  s = a + b;
  const double bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
// Bounds-checked build (PYC_BOUNDS defined by opts.debug_bounds): every access
// the generated code makes to an array -- a vector group [idx, idx + cnt) or one
// element -- is checked against the array's index range [lo, hi), and a vector
// group's address against its access width; the first violation in the module
// is recorded in pyc_bounds_rec (code, index, bound, block << 16 | thread) and
// the access is skipped.  PYC_BOUNDS_SHRINK (a test hook) narrows every range
// by that many elements at its top.  Without PYC_BOUNDS the checks are absent.
#ifdef PYC_BOUNDS
#ifndef PYC_BOUNDS_SHRINK
#define PYC_BOUNDS_SHRINK 0
#endif
__device__ unsigned long long pyc_bounds_rec[4];
__device__ __noinline__ bool pyc_bounds_fail(const long long idx, const long long bound,
                                             const int code) {
  if (atomicCAS(&pyc_bounds_rec[0], 0ull, (unsigned long long)code) == 0ull) {
    pyc_bounds_rec[1] = (unsigned long long)idx;
    pyc_bounds_rec[2] = (unsigned long long)bound;
    pyc_bounds_rec[3] = ((unsigned long long)blockIdx.x << 16) | threadIdx.x;
  }
  return false;
}
#define PYC_IN(idx, cnt, lo, hi, code)                                                \
  (((long long)(idx) >= (long long)(lo) &&                                              \
    (long long)(idx) + (long long)(cnt) <= (long long)(hi) - PYC_BOUNDS_SHRINK) ||       \
   pyc_bounds_fail((long long)(idx), (long long)(hi), (code)))
#define PYC_ALIGNED(ptr, width, code)                                                  \
  ((unsigned long long)(ptr) % (unsigned long long)(width) == 0ull ||                   \
   pyc_bounds_fail((long long)(unsigned long long)(ptr), (long long)(width), (code)))
#else
#define PYC_IN(idx, cnt, lo, hi, code) true
#define PYC_ALIGNED(ptr, width, code) true
#endif

// Programmatic dependent launch.  The single map and map-reduce kernels are
// launched with programmatic stream serialization, so they may be scheduled
// before the previous kernel on their stream has finished: each waits here for
// that kernel to complete (and its memory to be visible) before its first
// memory access, which keeps stream order, and lets the next launch be
// scheduled once every CTA has signalled.  Launched without the attribute,
// both are no-ops.
__device__ __forceinline__ void pyc_grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pyc_grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Arrival at a ticket shared by the CTAs of one launch (or one segment): an add
// with release-acquire semantics at GPU scope.  The partials the arriving thread
// stored before it are visible to whichever thread sees the last arrival, and
// that thread sees every earlier arrival's partials; a CTA barrier then hands
// the outcome (and that visibility) to the rest of its CTA.
__device__ __forceinline__ unsigned pyc_ticket_arrive(unsigned* t) {
  unsigned prev;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(t) : "memory");
  return prev;
}
// ------------------------------------------------------------ end of prelude
)PYC";

}  // namespace

std::string device_type(pyc_dtype t) { return type_info(t).device_name; }

const std::vector<Variant>& all_variants() {
  static const std::vector<Variant> v = {{16, 1}, {16, 2}, {16, 4}, {32, 1}, {32, 2}, {32, 4}};
  return v;
}

std::string variant_suffix(const Variant& v) {
  return "v" + std::to_string(v.vec_bytes) + "_u" + std::to_string(v.unroll);
}

int lifted_min_bytes(const ArgSpec& spec) {
  int m = 0;
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted) {
      int b = type_info(p.dtype).bytes;
      if (m == 0 || b < m) m = b;
    }
  return m == 0 ? 4 : m;
}

namespace {

std::string args_struct(const ArgSpec& spec) {
  std::ostringstream o;
  o << "struct pyc_args {\n";
  for (auto& p : spec.params) {
    o << "  " << (p.is_const && p.is_ptr ? "const " : "") << device_type(p.dtype)
      << (p.is_ptr ? "* " : " ") << p.name << ";\n";
  }
  if (spec.params.empty()) o << "  int pyc_unused;\n";
  o << "};\n";
  o << "static_assert(sizeof(pyc_args) == " << (spec.params.empty() ? 4 : spec.args_bytes)
    << ", \"argument struct layout\");\n";
  return o.str();
}

// Local names for the declared parameters (the statement refers to them).
std::string aliases(const ArgSpec& spec, const char* src) {
  std::ostringstream o;
  for (auto& p : spec.params) {
    std::string t = device_type(p.dtype);
    if (p.is_ptr)
      o << "  " << (p.is_const ? "const " : "") << t << "* const " << p.name << " = " << src
        << "." << p.name << ";\n";
    else
      o << "  const " << t << " " << p.name << " = " << src << "." << p.name << ";\n";
  }
  // keep unused-variable diagnostics quiet
  for (auto& p : spec.params) o << "  (void)" << p.name << ";\n";
  return o.str();
}

// Register copies of the lifted arrays, `count` elements each.
std::string reg_decls(const ArgSpec& spec, const std::string& count) {
  std::ostringstream o;
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted)
      o << "      __align__(32) " << device_type(p.dtype) << " pyc_r_" << p.name << "[" << count
        << "];\n";
  return o.str();
}

// Vector loads (reads) of group u for every lifted array that is read.
std::string group_io(const ArgSpec& spec, bool load) {
  std::ostringstream o;
  for (auto& p : spec.params) {
    if (!(p.is_ptr && p.lifted)) continue;
    if (load ? !p.read : !p.written) continue;
    int b = type_info(p.dtype).bytes;
    o << "        if (PYC_IN(pyc_e0, E, pyc_lo, pyc_hi, " << (load ? 1 : 2) << ") && PYC_ALIGNED("
      << p.name << " + pyc_e0, VB, 5)) ";
    if (load)
      o << "pyc_ldg<E * " << b << ", VB>(&pyc_r_" << p.name << "[pyc_u * E], " << p.name
        << " + pyc_e0);\n";
    else
      o << "pyc_stg<E * " << b << ", VB>(" << p.name << " + pyc_e0, &pyc_r_" << p.name
        << "[pyc_u * E]);\n";
  }
  return o.str();
}

// Double-buffer declarations / loads / name bindings / fold of one tile for
// the reduction span (lifted arrays only; a map expression never writes them).
std::string buf_decls(const ArgSpec& spec, const char* prefix, const std::string& count) {
  std::ostringstream o;
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted)
      o << "  __align__(32) " << device_type(p.dtype) << " " << prefix << p.name << "[" << count
        << "];\n";
  return o.str();
}

std::string buf_load(const ArgSpec& spec, const char* prefix, const std::string& base) {
  std::ostringstream o;
  o << "#pragma unroll\n    for (int pyc_u = 0; pyc_u < U; ++pyc_u) {\n"
    << "      const pyc_i64 pyc_e0 = (" << base << ") + (pyc_i64)pyc_u * pyc_step;\n";
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted && p.read)
      o << "      if (PYC_IN(pyc_e0, E, pyc_lo, pyc_hi, 1) && PYC_ALIGNED(" << p.name
        << " + pyc_e0, VB, 5)) pyc_ldg<E * " << type_info(p.dtype).bytes << ", VB>(&" << prefix
        << p.name << "[pyc_u * E], " << p.name << " + pyc_e0);\n";
  o << "    }\n";
  return o.str();
}

// buf_load for the lifted arrays `code` reads (rewritten form).
std::string buf_load_used(const ArgSpec& spec, const char* prefix, const std::string& base,
                          const std::string& code) {
  std::ostringstream o;
  o << "#pragma unroll\n    for (int pyc_u = 0; pyc_u < U; ++pyc_u) {\n"
    << "      const pyc_i64 pyc_e0 = (" << base << ") + (pyc_i64)pyc_u * pyc_step;\n";
  for (auto& p : spec.params) {
    if (!(p.is_ptr && p.lifted && p.read)) continue;
    if (code.find("pyc_r_" + p.name + " ") == std::string::npos &&
        code.find("pyc_r_" + p.name + "[") == std::string::npos)
      continue;
    o << "      if (PYC_IN(pyc_e0, E, pyc_lo, pyc_hi, 1) && PYC_ALIGNED(" << p.name
      << " + pyc_e0, VB, 5)) pyc_ldg<E * " << type_info(p.dtype).bytes << ", VB>(&" << prefix
      << p.name << "[pyc_u * E], " << p.name << " + pyc_e0);\n";
  }
  o << "    }\n";
  return o.str();
}

// Scan sweep 1: fold the rows of one step (RU rows from `base`) into pyc_wagg
// in element order; `rag` guards every element with i < te.
std::string fold_rows(const std::string& input_expr, const std::string& base, bool rag) {
  std::ostringstream o;
  o << "#pragma unroll\n      for (int pyc_u = 0; pyc_u < RU; ++pyc_u) {\n"
    << "        pyc_acc_t pyc_v = pyc_neutral();\n"
    << "#pragma unroll\n        for (int pyc_e = 0; pyc_e < E; ++pyc_e) {\n"
    << "          const int pyc_k = pyc_u * E + pyc_e;\n"
    << "          const pyc_i64 i = (" << base << ") + (pyc_i64)pyc_u * (32 * E) + pyc_e;\n"
    << "          (void)i;\n"
    << "          pyc_acc_t pyc_x = pyc_neutral();\n"
    << "          " << (rag ? "if (i < te) " : "") << "pyc_x = (pyc_acc_t)(" << input_expr
    << ");\n"
    << "          pyc_v = pyc_e == 0 ? pyc_x : pyc_combine(pyc_v, pyc_x);\n"
    << "        }\n"
    << "        // ordered fold across the row: lane 0 ends with lanes 0..31 in order\n"
    << "#pragma unroll\n        for (int d = 1; d < 32; d <<= 1) {\n"
    << "          const pyc_acc_t o = pyc_shfl_down(pyc_v, d);\n"
    << "          if (lane + d < 32) pyc_v = pyc_combine(pyc_v, o);\n"
    << "        }\n"
    << "        pyc_wagg = pyc_combine(pyc_wagg, pyc_v);\n"
    << "      }\n";
  return o.str();
}

std::string buf_refs(const ArgSpec& spec, const char* prefix) {
  std::ostringstream o;
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted)
      o << "      " << device_type(p.dtype) << " (&pyc_r_" << p.name << ")[T] = " << prefix
        << p.name << ";\n";
  return o.str();
}

std::string fold_tile(const std::string& map_expr, const std::string& base) {
  std::ostringstream o;
  o << "#pragma unroll\n      for (int pyc_k = 0; pyc_k < T; ++pyc_k) {\n"
    << "        const pyc_i64 i = (" << base << ") + (pyc_i64)(pyc_k / E) * pyc_step + (pyc_k % E);\n"
    << "        pyc_fold_ordered(pyc_acc[pyc_k % A], (" << map_expr << "), i);\n      }\n";
  return o.str();
}

// Bytes of the lifted arrays read per element (what one pass over a tile loads).
int stage_elem_bytes(const ArgSpec& spec) {
  int b = 0;
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted && p.read) b += type_info(p.dtype).bytes;
  return b;
}

// Vector loads of group u for the lifted arrays that `code` (already
// rewritten to register slots) reads.
std::string group_loads_used(const ArgSpec& spec, const std::string& code) {
  std::ostringstream o;
  for (auto& p : spec.params) {
    if (!(p.is_ptr && p.lifted && p.read)) continue;
    if (code.find("pyc_r_" + p.name + " ") == std::string::npos &&
        code.find("pyc_r_" + p.name + "[") == std::string::npos)
      continue;
    o << "        if (PYC_IN(pyc_e0, E, pyc_lo, pyc_hi, 1) && PYC_ALIGNED(" << p.name
      << " + pyc_e0, VB, 5)) pyc_ldg<E * " << type_info(p.dtype).bytes << ", VB>(&pyc_r_"
      << p.name << "[pyc_u * E], " << p.name << " + pyc_e0);\n";
  }
  return o.str();
}

// L2 prefetch hints (evict-last) over [ts, te) of every lifted array `code`
// reads: thread tid of nt takes every nt-th 128-byte line, from the line that
// holds element ts; every line touched holds at least one element of the range.
std::string prefetch_used(const ArgSpec& spec, const std::string& code) {
  std::ostringstream o;
  for (auto& p : spec.params) {
    if (!(p.is_ptr && p.lifted && p.read)) continue;
    if (code.find("pyc_r_" + p.name + " ") == std::string::npos &&
        code.find("pyc_r_" + p.name + "[") == std::string::npos)
      continue;
    o << "  {\n"
      << "    const unsigned long long pyc_pb = (unsigned long long)(" << p.name << " + ts);\n"
      << "    const unsigned long long pyc_pe = (unsigned long long)(" << p.name << " + te);\n"
      << "    for (unsigned long long q = (pyc_pb & ~127ull) + 128ull * tid; q < pyc_pe;\n"
      << "         q += 128ull * nt)\n"
      << "      asm volatile(\"prefetch.global.L2::evict_last [%0];\" ::\"l\"(q));\n"
      << "  }\n";
  }
  return o.str();
}

// Element-wise loads into register slot pyc_k at index i of the lifted arrays
// read (by `code` only, if it is not empty), and stores of those written.
std::string scalar_loads_k(const ArgSpec& spec, const std::string& code) {
  std::ostringstream o;
  for (auto& p : spec.params) {
    if (!(p.is_ptr && p.lifted && p.read)) continue;
    if (!code.empty() && code.find("pyc_r_" + p.name + " ") == std::string::npos &&
        code.find("pyc_r_" + p.name + "[") == std::string::npos)
      continue;
    o << "          pyc_r_" << p.name << "[pyc_k] = " << p.name << "[i];\n";
  }
  return o.str();
}

std::string scalar_stores_k(const ArgSpec& spec) {
  std::ostringstream o;
  for (auto& p : spec.params)
    if (p.is_ptr && p.lifted && p.written)
      o << "            " << p.name << "[i] = pyc_r_" << p.name << "[pyc_k];\n";
  return o.str();
}

// The same loads / stores with an L2 cache policy `pol` (pyc_ldgh / pyc_stgh).
std::string with_policy(const std::string& code, const std::string& pol) {
  std::string out, line;
  std::istringstream in(code);
  while (std::getline(in, line)) {
    for (const char* f : {"pyc_ldg<", "pyc_stg<"}) {
      size_t k = line.find(f);
      if (k == std::string::npos) continue;
      line.insert(k + 7, "h");
      size_t e = line.rfind(");");
      if (e != std::string::npos) line.insert(e, ", " + pol);
    }
    out += line + "\n";
  }
  return out;
}

std::string scalar_io(const ArgSpec& spec, bool load) {
  std::ostringstream o;
  for (auto& p : spec.params) {
    if (!(p.is_ptr && p.lifted)) continue;
    if (load && p.read)
      o << "      if (PYC_IN(i, 1, pyc_lo, pyc_hi, 3)) pyc_r_" << p.name << "[0] = " << p.name
        << "[i];\n";
    if (!load && p.written)
      o << "      if (PYC_IN(i, 1, pyc_lo, pyc_hi, 4)) " << p.name << "[i] = pyc_r_" << p.name
        << "[0];\n";
  }
  return o.str();
}

}  // namespace

MapGen generate_map(const ArgSpec& spec, const std::string& stmt, const std::string& preamble,
                    const std::string& tag) {
  const int mins = lifted_min_bytes(spec);
  std::ostringstream o;
  o << "// pyc map kernel: " << spec.canonical << "\n";
  o << kPrelude;
  if (!preamble.empty()) o << "// ---- user preamble\n" << preamble << "\n";
  o << args_struct(spec);
  o << "#define PYC_MIN_BYTES " << mins << "\n";
  o << R"PYC(
template <int VB, int U>
__device__ __forceinline__ void pyc_map_body(const pyc_args& pyc_p, const pyc_i64 n,
                                             const pyc_i64 pyc_head) {
  constexpr int E = VB / PYC_MIN_BYTES;  // elements per vector group
  constexpr int T = E * U;               // elements per thread per tile
)PYC";
  o << aliases(spec, "pyc_p");
  o << R"PYC(  const pyc_i64 pyc_lo = 0, pyc_hi = n;  // every array holds n elements
  (void)pyc_lo;
  (void)pyc_hi;
  pyc_grid_dependency_wait();
  pyc_grid_launch_dependents();  // the next launch may be scheduled at once
  const pyc_i64 pyc_step = (pyc_i64)blockDim.x * E;
  const pyc_i64 pyc_tile = pyc_step * U;
  // aligned body [h, h + nfull * tile) in whole tiles; head [0, h) and tail scalar
  const pyc_i64 pyc_h = pyc_head < 0 ? 0 : (pyc_head < n ? pyc_head : n);
  const pyc_i64 pyc_nfull = pyc_head < 0 ? 0 : (n - pyc_h) / pyc_tile;
  for (pyc_i64 pyc_t = blockIdx.x; pyc_t < pyc_nfull; pyc_t += gridDim.x) {
    const pyc_i64 pyc_b0 = pyc_h + pyc_t * pyc_tile + (pyc_i64)threadIdx.x * E;
    {
)PYC";
  o << reg_decls(spec, "T");
  o << R"PYC(#pragma unroll
      for (int pyc_u = 0; pyc_u < U; ++pyc_u) {
        const pyc_i64 pyc_e0 = pyc_b0 + (pyc_i64)pyc_u * pyc_step;
)PYC";
  o << group_io(spec, true);
  o << R"PYC(      }
#pragma unroll
      for (int pyc_k = 0; pyc_k < T; ++pyc_k) {
        const pyc_i64 i = pyc_b0 + (pyc_i64)(pyc_k / E) * pyc_step + (pyc_k % E);
        (void)i;
        { )PYC" << stmt << R"PYC( ; }
      }
#pragma unroll
      for (int pyc_u = 0; pyc_u < U; ++pyc_u) {
        const pyc_i64 pyc_e0 = pyc_b0 + (pyc_i64)pyc_u * pyc_step;
)PYC";
  o << group_io(spec, false);
  o << R"PYC(      }
    }
  }
  const pyc_i64 pyc_tail0 = pyc_h + pyc_nfull * pyc_tile;
  const pyc_i64 pyc_nrem = pyc_h + (n - pyc_tail0);
  for (pyc_i64 pyc_j = (pyc_i64)blockIdx.x * blockDim.x + threadIdx.x; pyc_j < pyc_nrem;
       pyc_j += (pyc_i64)gridDim.x * blockDim.x) {
    const pyc_i64 i = pyc_j < pyc_h ? pyc_j : pyc_tail0 + (pyc_j - pyc_h);
)PYC";
  o << reg_decls(spec, "1");
  o << scalar_io(spec, true);
  o << "      { const int pyc_k = 0; (void)pyc_k; " << stmt << " ; }\n";
  o << scalar_io(spec, false);
  o << "  }\n}\n\n";
  // Span form for batched launches: [vs, ve) aligned vector body plus the
  // scalar range [ss, se), processed by a group of nthr threads (a CTA).
  o << R"PYC(template <int VB, int U>
__device__ __forceinline__ void pyc_map_span(const pyc_args& pyc_p, const pyc_i64 n,
    const pyc_i64 pyc_vs, const pyc_i64 pyc_ve, const pyc_i64 pyc_ss, const pyc_i64 pyc_se,
    const int pyc_tid, const int pyc_nthr) {
  constexpr int E = VB / PYC_MIN_BYTES;
  constexpr int T = E * U;
)PYC";
  o << aliases(spec, "pyc_p");
  o << R"PYC(  (void)n;
  const pyc_i64 pyc_lo = 0, pyc_hi = n;  // every array of the task holds n elements
  (void)pyc_lo;
  (void)pyc_hi;
  const pyc_i64 pyc_step = (pyc_i64)pyc_nthr * E;
  const pyc_i64 pyc_tile = pyc_step * U;
  const pyc_i64 pyc_nt = pyc_ve > pyc_vs ? (pyc_ve - pyc_vs) / pyc_tile : 0;
  for (pyc_i64 pyc_t = 0; pyc_t < pyc_nt; ++pyc_t) {
    const pyc_i64 pyc_b0 = pyc_vs + pyc_t * pyc_tile + (pyc_i64)pyc_tid * E;
    {
)PYC";
  o << reg_decls(spec, "T");
  o << R"PYC(#pragma unroll
      for (int pyc_u = 0; pyc_u < U; ++pyc_u) {
        const pyc_i64 pyc_e0 = pyc_b0 + (pyc_i64)pyc_u * pyc_step;
)PYC";
  o << group_io(spec, true);
  o << R"PYC(      }
#pragma unroll
      for (int pyc_k = 0; pyc_k < T; ++pyc_k) {
        const pyc_i64 i = pyc_b0 + (pyc_i64)(pyc_k / E) * pyc_step + (pyc_k % E);
        (void)i;
        { )PYC" << stmt << R"PYC( ; }
      }
#pragma unroll
      for (int pyc_u = 0; pyc_u < U; ++pyc_u) {
        const pyc_i64 pyc_e0 = pyc_b0 + (pyc_i64)pyc_u * pyc_step;
)PYC";
  o << group_io(spec, false);
  o << R"PYC(      }
    }
  }
  const pyc_i64 pyc_r0 = pyc_vs + pyc_nt * pyc_tile;
  const pyc_i64 pyc_ns = pyc_se - pyc_ss;
  const pyc_i64 pyc_nr = (pyc_ve > pyc_r0 ? pyc_ve - pyc_r0 : 0) + pyc_ns;
  for (pyc_i64 pyc_j = pyc_tid; pyc_j < pyc_nr; pyc_j += pyc_nthr) {
    const pyc_i64 i = pyc_j < pyc_ns ? pyc_ss + pyc_j : pyc_r0 + (pyc_j - pyc_ns);
)PYC";
  o << reg_decls(spec, "1");
  o << scalar_io(spec, true);
  o << "      { const int pyc_k = 0; (void)pyc_k; " << stmt << " ; }\n";
  o << scalar_io(spec, false);
  o << R"PYC(  }
}

// Batched map: one record per request, one work item per chunk.
struct pyc_mtask {
  pyc_args args;
  pyc_i64 n;
  pyc_i64 head;   // vector body start (-1: scalar only)
  pyc_i64 chunk;  // chunk length (a multiple of the tile)
};
struct pyc_mitem {
  int task;
  int chunk;
};

template <int VB, int U>
__device__ __forceinline__ void pyc_map_batched_body(const pyc_mtask* __restrict__ tasks,
    const pyc_mitem* __restrict__ items, const int nitems, unsigned* __restrict__ ctl) {
  // Item order: CTA b takes item b first (no counter round trip before its
  // first load); later items come from the counter (offset by the grid), the
  // next index fetched by thread 0 while the current item runs and handed to
  // the CTA through one of two shared slots (the other may still be read).
  __shared__ int pyc_it[2];
  int it = (int)blockIdx.x;
  for (int k = 0; it < nitems; ++k) {
    int next = 0;
    if (threadIdx.x == 0) next = (int)gridDim.x + (int)atomicAdd(&ctl[0], 1u);
    const pyc_mitem I = items[it];
    const pyc_mtask& T = tasks[I.task];
    const pyc_i64 n = T.n, head = T.head, chunk = T.chunk, c = I.chunk;
    if (head >= 0) {
      const pyc_i64 vs = head + c * chunk;
      const pyc_i64 ve = vs + chunk < n ? vs + chunk : n;
      pyc_map_span<VB, U>(T.args, n, vs, ve, 0, c == 0 ? head : 0, threadIdx.x, blockDim.x);
    } else {
      const pyc_i64 ss = c * chunk;
      const pyc_i64 se = ss + chunk < n ? ss + chunk : n;
      pyc_map_span<VB, U>(T.args, n, 0, 0, ss, se, threadIdx.x, blockDim.x);
    }
    if (threadIdx.x == 0) pyc_it[k & 1] = next;
    __syncthreads();
    it = pyc_it[k & 1];
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl[1], 1u) == gridDim.x - 1) {
      ctl[0] = 0u;
      ctl[1] = 0u;
      __threadfence();
    }
  }
}

)PYC";
  MapGen g;
  int off = (spec.params.empty() ? 4 : spec.args_bytes);
  off = (off + 7) / 8 * 8;
  g.task_off_n = off;
  g.task_off_head = off + 8;
  g.task_off_chunk = off + 16;
  g.task_bytes = off + 24;
  o << "static_assert(sizeof(pyc_mtask) == " << g.task_bytes << ", \"task layout\");\n";
  // one compilation unit per kernel (kUnitMark): NVRTC compiles them in parallel
  for (auto& v : all_variants()) {
    o << kUnitMark;
    o << "extern \"C\" __global__ void __launch_bounds__(512) pyc_map_" << tag << "_"
      << variant_suffix(v) << "(const pyc_args pyc_p, const pyc_i64 n, const pyc_i64 pyc_head) {\n"
      << "  pyc_map_body<" << v.vec_bytes << ", " << v.unroll << ">(pyc_p, n, pyc_head);\n}\n";
    o << kUnitMark;
    o << "extern \"C\" __global__ void __launch_bounds__(512) pyc_mbatch_" << tag << "_"
      << variant_suffix(v)
      << "(const pyc_mtask* tasks, const pyc_mitem* items, const int nitems, unsigned* ctl) {\n"
      << "  pyc_map_batched_body<" << v.vec_bytes << ", " << v.unroll
      << ">(tasks, items, nitems, ctl);\n}\n";
  }
  g.source = o.str();
  return g;
}

ReduceGen generate_reduce(const ArgSpec& spec, pyc_dtype out_dtype, ReduceKind kind,
                          const std::string& neutral, const std::string& reduce_expr,
                          const std::string& map_expr, const std::string& preamble,
                          const std::string& tag, int ordered_arg, bool emit_kernels) {
  ReduceGen g;
  const int mins = lifted_min_bytes(spec);
  std::string acc_t, out_t;
  switch (kind) {
    case ReduceKind::Arg:
      acc_t = out_t = "pyc_argf32";
      g.acc_bytes = g.out_bytes = 16;
      break;
    case ReduceKind::Compensated:
      acc_t = "pyc_cf32";
      out_t = "float";
      g.acc_bytes = 8;
      g.out_bytes = 4;
      break;
    case ReduceKind::Plain:
      if (out_dtype == PYC_BF16 || out_dtype == PYC_F16) {
        acc_t = "float";
        g.acc_bytes = 4;
      } else {
        acc_t = device_type(out_dtype);
        g.acc_bytes = type_info(out_dtype).bytes;
      }
      out_t = device_type(out_dtype);
      g.out_bytes = type_info(out_dtype).bytes;
      break;
  }
  // batched task record: args, then n, head, chunk, out, nchunks, slot0
  int off = (spec.params.empty() ? 4 : spec.args_bytes);
  off = (off + 7) / 8 * 8;
  g.task_off_n = off;
  g.task_off_head = off + 8;
  g.task_off_chunk = off + 16;
  g.task_off_out = off + 24;
  g.task_off_nchunks = off + 32;
  g.task_off_slot0 = off + 36;
  g.task_bytes = off + 40;

  std::ostringstream o;
  o << "// pyc map-reduce kernel: " << spec.canonical << "\n";
  o << kPrelude;
  if (!preamble.empty()) o << "// ---- user preamble\n" << preamble << "\n";
  o << args_struct(spec);
  o << "#define PYC_MIN_BYTES " << mins << "\n";
  o << "typedef " << acc_t << " pyc_acc_t;\n";
  o << "typedef " << out_t << " pyc_out_t;\n";
  o << "static_assert(sizeof(pyc_acc_t) == " << g.acc_bytes << ", \"accumulator size\");\n";
  o << "static_assert(sizeof(pyc_out_t) == " << g.out_bytes << ", \"result size\");\n";
  // neutral, combine, fold, finalize
  switch (kind) {
    case ReduceKind::Plain:
      o << "__device__ __forceinline__ pyc_acc_t pyc_neutral() { return (pyc_acc_t)(" << neutral
        << "); }\n";
      o << "__device__ __forceinline__ pyc_acc_t pyc_combine(const pyc_acc_t a, const pyc_acc_t b) "
           "{ return (pyc_acc_t)(" << reduce_expr << "); }\n";
      o << "template <typename V> __device__ __forceinline__ void pyc_fold(pyc_acc_t& pyc_a, const V pyc_v, "
           "const pyc_i64) { pyc_a = pyc_combine(pyc_a, (pyc_acc_t)(pyc_v)); }\n";
      if (out_dtype == PYC_BF16 || out_dtype == PYC_F16)
        o << "__device__ __forceinline__ pyc_out_t pyc_finalize(const pyc_acc_t a) { return pyc_out_t(a); }\n";
      else
        o << "__device__ __forceinline__ pyc_out_t pyc_finalize(const pyc_acc_t a) { return a; }\n";
      break;
    case ReduceKind::Arg:
      o << "__device__ __forceinline__ pyc_acc_t pyc_neutral() { return " << neutral << "; }\n";
      o << "__device__ __forceinline__ pyc_acc_t pyc_combine(const pyc_acc_t a, const pyc_acc_t b) "
           "{ return (" << reduce_expr << "); }\n";
      o << "template <typename V> __device__ __forceinline__ void pyc_fold(pyc_acc_t& pyc_a, const V pyc_v, "
           "const pyc_i64 pyc_i) { pyc_argf32 pyc_e; pyc_e.v = (float)(pyc_v); pyc_e.pad = 0; "
           "pyc_e.i = pyc_i; pyc_a = pyc_combine(pyc_a, pyc_e); }\n";
      o << "__device__ __forceinline__ pyc_out_t pyc_finalize(const pyc_acc_t a) { return a; }\n";
      break;
    case ReduceKind::Compensated:
      o << R"PYC(__device__ __forceinline__ pyc_acc_t pyc_neutral() { pyc_cf32 z; z.s = 0.0f; z.c = 0.0f; return z; }
// (s1 + c1) + (s2 + c2): exact two-sum of the leading parts, errors summed.
__device__ __forceinline__ pyc_acc_t pyc_combine(const pyc_acc_t a, const pyc_acc_t b) {
  pyc_cf32 r; float e;
  pyc_two_sum(a.s, b.s, r.s, e);
  r.c = (a.c + b.c) + e;
  return r;
}
template <typename V> __device__ __forceinline__ void pyc_fold(pyc_acc_t& pyc_a, const V pyc_v, const pyc_i64) {
  float s, e;
  pyc_two_sum(pyc_a.s, (float)(pyc_v), s, e);
  pyc_a.s = s;
  pyc_a.c += e;
}
__device__ __forceinline__ pyc_out_t pyc_finalize(const pyc_acc_t a) {
  return __double2float_rn((double)a.s + (double)a.c);
}
)PYC";
      break;
  }
  // Fold used in the vector body.  Each accumulator slot k sees the indices
  // of its elements in increasing order there, so for the built-in argmin /
  // argmax rule a strict comparison already keeps the first index; the
  // neutral element (index LLONG_MAX) is replaced by the first value seen.
  // Everything else (and the scalar leftovers, which visit the head after the
  // body) uses the full fold.
  if (ordered_arg == 1 || ordered_arg == 2) {
    o << "template <typename V> __device__ __forceinline__ void pyc_fold_ordered(pyc_acc_t& pyc_a, "
         "const V pyc_v, const pyc_i64 pyc_i) {\n"
         "  const float pyc_f = (float)(pyc_v);\n"
         "  if (pyc_f " << (ordered_arg == 1 ? "<" : ">") << " pyc_a.v || pyc_a.i == LLONG_MAX) { "
         "pyc_a.v = pyc_f; pyc_a.i = pyc_i; }\n}\n";
  } else {
    o << "template <typename V> __device__ __forceinline__ void pyc_fold_ordered(pyc_acc_t& pyc_a, "
         "const V pyc_v, const pyc_i64 pyc_i) { pyc_fold(pyc_a, pyc_v, pyc_i); }\n";
  }
  o << R"PYC(
struct pyc_combine_op {
  __device__ __forceinline__ pyc_acc_t operator()(const pyc_acc_t a, const pyc_acc_t b) const { return pyc_combine(a, b); }
};

// Fold [vs, ve) (vs aligned to VB for every lifted array) with vector groups,
// plus the scalar range [ss, se), by a group of `nthr` threads (a CTA or a
// warp); returns this thread's accumulator.  [lo, hi) is the index range the
// arrays hold (for the bounds-checked build).
template <int VB, int U>
__device__ __forceinline__ pyc_acc_t pyc_reduce_span(const pyc_args& pyc_p, const pyc_i64 n,
    const pyc_i64 pyc_vs, const pyc_i64 pyc_ve, const pyc_i64 pyc_ss, const pyc_i64 pyc_se,
    const int pyc_tid, const int pyc_nthr, const pyc_i64 pyc_lo, const pyc_i64 pyc_hi) {
  constexpr int E = VB / PYC_MIN_BYTES;
  constexpr int T = E * U;
  // independent accumulators: element position k folds into acc[k % A]
  constexpr int AMAX = 128 / (int)sizeof(pyc_acc_t) > 0 ? 128 / (int)sizeof(pyc_acc_t) : 1;
  constexpr int A = T < AMAX ? T : AMAX;
)PYC";
  o << aliases(spec, "pyc_p");
  o << R"PYC(  (void)n;
  (void)pyc_lo;
  (void)pyc_hi;
  pyc_acc_t pyc_acc[A];
#pragma unroll
  for (int k = 0; k < A; ++k) pyc_acc[k] = pyc_neutral();
  // Tiles are register double-buffered: the loads of tile t+1 are issued
  // before tile t is folded, so memory traffic overlaps the arithmetic.
  const pyc_i64 pyc_step = (pyc_i64)pyc_nthr * E;
  const pyc_i64 pyc_tile = pyc_step * U;
  const pyc_i64 pyc_nt = pyc_ve > pyc_vs ? (pyc_ve - pyc_vs) / pyc_tile : 0;
  const pyc_i64 pyc_tb = pyc_vs + (pyc_i64)pyc_tid * E;
)PYC";
  // unroll 1-2: double-buffered; unroll 4 (registers already full): single buffer
  o << "  if constexpr (U <= 2) {\n";
  o << buf_decls(spec, "pyc_ba_", "T") << buf_decls(spec, "pyc_bb_", "T");
  o << "  if (pyc_nt > 0) {\n" << buf_load(spec, "pyc_ba_", "pyc_tb") << "  }\n";
  o << R"PYC(  for (pyc_i64 pyc_t = 0; pyc_t < pyc_nt; pyc_t += 2) {
    const pyc_i64 pyc_b0 = pyc_tb + pyc_t * pyc_tile;
    const pyc_i64 pyc_b1 = pyc_b0 + pyc_tile;
    const bool pyc_has1 = pyc_t + 1 < pyc_nt;
    if (pyc_has1) {
)PYC";
  o << buf_load(spec, "pyc_bb_", "pyc_b1");
  o << "    }\n    {\n" << buf_refs(spec, "pyc_ba_") << fold_tile(map_expr, "pyc_b0") << "    }\n";
  o << "    if (pyc_t + 2 < pyc_nt) {\n" << buf_load(spec, "pyc_ba_", "pyc_b1 + pyc_tile") << "    }\n";
  o << "    if (pyc_has1) {\n" << buf_refs(spec, "pyc_bb_") << fold_tile(map_expr, "pyc_b1")
    << "    }\n  }\n";
  o << "  } else {\n";
  o << "  for (pyc_i64 pyc_t = 0; pyc_t < pyc_nt; ++pyc_t) {\n"
       "    const pyc_i64 pyc_b0 = pyc_tb + pyc_t * pyc_tile;\n    {\n";
  o << buf_decls(spec, "pyc_ba_", "T") << buf_load(spec, "pyc_ba_", "pyc_b0");
  o << buf_refs(spec, "pyc_ba_") << fold_tile(map_expr, "pyc_b0") << "    }\n  }\n  }\n";
  o << R"PYC(
  const pyc_i64 pyc_r0 = pyc_vs + pyc_nt * pyc_tile;
  const pyc_i64 pyc_ns = pyc_se - pyc_ss;
  const pyc_i64 pyc_nr = (pyc_ve > pyc_r0 ? pyc_ve - pyc_r0 : 0) + pyc_ns;
  for (pyc_i64 pyc_j = pyc_tid; pyc_j < pyc_nr; pyc_j += pyc_nthr) {
    const pyc_i64 i = pyc_j < pyc_ns ? pyc_ss + pyc_j : pyc_r0 + (pyc_j - pyc_ns);
)PYC";
  o << reg_decls(spec, "1");
  o << scalar_io(spec, true);
  o << "      { const int pyc_k = 0; (void)pyc_k; pyc_fold(pyc_acc[0], (" << map_expr << "), i); }\n";
  o << R"PYC(  }
#pragma unroll
  for (int s = 1; s < A; s *= 2)
#pragma unroll
    for (int k = 0; k + s < A; k += 2 * s) pyc_acc[k] = pyc_combine(pyc_acc[k], pyc_acc[k + s]);
  return pyc_acc[0];
}

// Fold the chunk c of a range of length n whose vector body starts at head
// (head < 0: no vector body).  Chunk 0 also takes the scalar head [0, head).
template <int VB, int U>
__device__ __forceinline__ pyc_acc_t pyc_chunk(const pyc_args& pyc_p, const pyc_i64 n,
    const pyc_i64 head, const pyc_i64 chunk, const pyc_i64 c, const int tid, const int nthr) {
  if (head >= 0) {
    const pyc_i64 vs = head + c * chunk;
    const pyc_i64 ve = vs + chunk < n ? vs + chunk : n;
    return pyc_reduce_span<VB, U>(pyc_p, n, vs, ve, 0, c == 0 ? head : 0, tid, nthr, 0, n);
  }
  const pyc_i64 ss = c * chunk;
  const pyc_i64 se = ss + chunk < n ? ss + chunk : n;
  return pyc_reduce_span<VB, U>(pyc_p, n, 0, 0, ss, se, tid, nthr, 0, n);
}

)PYC";
  // partial combine (shared by the single reduction and the batched one)
  if (kind == ReduceKind::Compensated) {
    o << R"PYC(// Final combine of compensated partials in binary64: each thread sums its
// partials' (s, c) with a binary64 two-sum, then a fixed tree; thread 0 rounds.
struct pyc_dd { double hi; double lo; };
struct pyc_dd_op {
  __device__ __forceinline__ pyc_dd operator()(const pyc_dd a, const pyc_dd b) const {
    pyc_dd r; double e;
    pyc_two_sum_d(a.hi, b.hi, r.hi, e);
    r.lo = (a.lo + b.lo) + e;
    return r;
  }
};
__device__ __forceinline__ pyc_out_t pyc_combine_partials(const pyc_acc_t* part, const int count) {
  pyc_dd acc; acc.hi = 0.0; acc.lo = 0.0;
  pyc_dd_op op;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const pyc_acc_t p = pyc_ld_cg(part + j);
    pyc_dd t; t.hi = (double)p.s; t.lo = (double)p.c;
    acc = op(acc, t);
  }
  pyc_dd z; z.hi = 0.0; z.lo = 0.0;
  acc = pyc_block_reduce(acc, op, z);
  return __double2float_rn(acc.hi + acc.lo);
}
// The same for count <= 1 partials held by thread 0 in v (the same arithmetic).
__device__ __forceinline__ pyc_out_t pyc_combine_partials_reg(const pyc_acc_t v, const int count) {
  pyc_dd acc; acc.hi = 0.0; acc.lo = 0.0;
  pyc_dd_op op;
  if ((int)threadIdx.x < count) {
    pyc_dd t; t.hi = (double)v.s; t.lo = (double)v.c;
    acc = op(acc, t);
  }
  pyc_dd z; z.hi = 0.0; z.lo = 0.0;
  acc = pyc_block_reduce(acc, op, z);
  return __double2float_rn(acc.hi + acc.lo);
}
)PYC";
  } else {
    o << R"PYC(__device__ __forceinline__ pyc_out_t pyc_combine_partials(const pyc_acc_t* part, const int count) {
  pyc_acc_t acc = pyc_neutral();
  for (int j = threadIdx.x; j < count; j += blockDim.x) acc = pyc_combine(acc, pyc_ld_cg(part + j));
  acc = pyc_block_reduce(acc, pyc_combine_op(), pyc_neutral());
  return pyc_finalize(acc);
}
// The same for count <= 1 partials held by thread 0 in v (the same arithmetic).
__device__ __forceinline__ pyc_out_t pyc_combine_partials_reg(const pyc_acc_t v, const int count) {
  pyc_acc_t acc = pyc_neutral();
  if ((int)threadIdx.x < count) acc = pyc_combine(acc, v);
  acc = pyc_block_reduce(acc, pyc_combine_op(), pyc_neutral());
  return pyc_finalize(acc);
}
)PYC";
  }
  // accumulator record of a shard (sharded reductions): 16 bytes
  if (kind == ReduceKind::Compensated) {
    o << R"PYC(// Record of a shard: the binary64 pair (hi, lo) whose sum is the shard's sum.
struct pyc_record { double hi; double lo; };
__device__ __forceinline__ pyc_record pyc_record_partials(const pyc_acc_t* part, const int count) {
  pyc_dd acc; acc.hi = 0.0; acc.lo = 0.0;
  pyc_dd_op op;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const pyc_acc_t p = pyc_ld_cg(part + j);
    pyc_dd t; t.hi = (double)p.s; t.lo = (double)p.c;
    acc = op(acc, t);
  }
  pyc_dd z; z.hi = 0.0; z.lo = 0.0;
  acc = pyc_block_reduce(acc, op, z);
  pyc_record r; r.hi = acc.hi; r.lo = acc.lo;
  return r;
}
// Combine of k records in record order (then a fixed tree); one rounding.
__device__ __forceinline__ pyc_out_t pyc_combine_records(const pyc_record* rec, const pyc_i64 k) {
  pyc_dd acc; acc.hi = 0.0; acc.lo = 0.0;
  pyc_dd_op op;
  for (pyc_i64 j = threadIdx.x; j < k; j += blockDim.x) {
    pyc_dd t; t.hi = rec[j].hi; t.lo = rec[j].lo;
    acc = op(acc, t);
  }
  pyc_dd z; z.hi = 0.0; z.lo = 0.0;
  acc = pyc_block_reduce(acc, op, z);
  return __double2float_rn(acc.hi + acc.lo);
}
)PYC";
  } else {
    if (g.acc_bytes == 16)
      o << "// Record of a shard: its accumulator, before conversion to the result type.\n"
           "struct pyc_record { pyc_acc_t acc; };\n";
    else
      o << "// Record of a shard: its accumulator, before conversion to the result type.\n"
           "struct pyc_record { pyc_acc_t acc; unsigned char pad[16 - sizeof(pyc_acc_t)]; };\n";
    o << R"PYC(__device__ __forceinline__ pyc_record pyc_record_partials(const pyc_acc_t* part, const int count) {
  pyc_acc_t acc = pyc_neutral();
  for (int j = threadIdx.x; j < count; j += blockDim.x) acc = pyc_combine(acc, pyc_ld_cg(part + j));
  acc = pyc_block_reduce(acc, pyc_combine_op(), pyc_neutral());
  pyc_record r;
  unsigned char* b = reinterpret_cast<unsigned char*>(&r);
#pragma unroll
  for (int j = 0; j < 16; ++j) b[j] = 0;
  r.acc = acc;
  return r;
}
// Combine of k records with the reduce expression in record order (then a
// fixed tree), converted to the result type once.
__device__ __forceinline__ pyc_out_t pyc_combine_records(const pyc_record* rec, const pyc_i64 k) {
  pyc_acc_t acc = pyc_neutral();
  for (pyc_i64 j = threadIdx.x; j < k; j += blockDim.x) acc = pyc_combine(acc, rec[j].acc);
  acc = pyc_block_reduce(acc, pyc_combine_op(), pyc_neutral());
  return pyc_finalize(acc);
}
)PYC";
  }
  o << "static_assert(sizeof(pyc_record) == 16, \"record size\");\n";
  o << R"PYC(
// Single reduction: CTAs take chunks c = blockIdx.x, blockIdx.x + gridDim.x, ...;
// the last CTA to arrive combines the partials and resets the ticket.  A launch
// of one CTA with at most one chunk (n up to one tile) skips both.
template <int VB, int U>
__device__ __forceinline__ void pyc_reduce_body(const pyc_args& pyc_p, const pyc_i64 n,
    const pyc_i64 head, const pyc_i64 chunk, const pyc_i64 nchunks,
    pyc_acc_t* __restrict__ part, unsigned* __restrict__ ticket, pyc_out_t* __restrict__ out) {
  __shared__ unsigned pyc_last;
  // one CTA and at most one chunk: its partial is the only one, so it is
  // combined where it is, with no partial slot, ticket or second read
  const bool pyc_solo = gridDim.x == 1 && nchunks <= 1;
  pyc_grid_dependency_wait();
  pyc_acc_t pyc_v1 = pyc_neutral();
  for (pyc_i64 c = blockIdx.x; c < nchunks; c += gridDim.x) {
    pyc_acc_t v = pyc_chunk<VB, U>(pyc_p, n, head, chunk, c, threadIdx.x, blockDim.x);
    v = pyc_block_reduce(v, pyc_combine_op(), pyc_neutral());
    if (pyc_solo) pyc_v1 = v;
    else if (threadIdx.x == 0) part[c] = v;
  }
  // the next launch on the stream may be scheduled while the partials are combined
  pyc_grid_launch_dependents();
  if (pyc_solo) {
    const pyc_out_t r = pyc_combine_partials_reg(pyc_v1, (int)nchunks);
    if (threadIdx.x == 0) *out = r;
    return;
  }
  // thread 0 stored every partial of this CTA; its arrival publishes them
  if (threadIdx.x == 0) pyc_last = pyc_ticket_arrive(ticket) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!pyc_last) return;
  const pyc_out_t r = pyc_combine_partials(part, (int)nchunks);
  if (threadIdx.x == 0) {
    *out = r;
    *ticket = 0u;
  }
}

// Sharded reduction: one shard [base, base + len) of a range of length n that
// is partitioned across devices.  The argument struct's array pointers are
// offset by -base elements, so element i of the shard's arrays is addressed as
// name[i] with the global index i, which the map expression (and an argmin's
// index) sees; chunk c starts at base + head + c * chunk.  The last CTA
// combines the partials into the shard's record instead of the result.
template <int VB, int U>
__device__ __forceinline__ pyc_acc_t pyc_chunk_at(const pyc_args& pyc_p, const pyc_i64 n,
    const pyc_i64 base, const pyc_i64 len, const pyc_i64 head, const pyc_i64 chunk,
    const pyc_i64 c, const int tid, const int nthr) {
  const pyc_i64 end = base + len;
  if (head >= 0) {
    const pyc_i64 vs = base + head + c * chunk;
    const pyc_i64 ve = vs + chunk < end ? vs + chunk : end;
    return pyc_reduce_span<VB, U>(pyc_p, n, vs, ve, base, c == 0 ? base + head : base, tid, nthr,
                                  base, end);
  }
  const pyc_i64 ss = base + c * chunk;
  const pyc_i64 se = ss + chunk < end ? ss + chunk : end;
  return pyc_reduce_span<VB, U>(pyc_p, n, 0, 0, ss, se, tid, nthr, base, end);
}
template <int VB, int U>
__device__ __forceinline__ void pyc_shard_body(const pyc_args& pyc_p, const pyc_i64 n,
    const pyc_i64 base, const pyc_i64 len, const pyc_i64 head, const pyc_i64 chunk,
    const pyc_i64 nchunks, pyc_acc_t* __restrict__ part, unsigned* __restrict__ ticket,
    pyc_record* __restrict__ rec) {
  __shared__ unsigned pyc_last;
  for (pyc_i64 c = blockIdx.x; c < nchunks; c += gridDim.x) {
    pyc_acc_t v = pyc_chunk_at<VB, U>(pyc_p, n, base, len, head, chunk, c, threadIdx.x, blockDim.x);
    v = pyc_block_reduce(v, pyc_combine_op(), pyc_neutral());
    if (threadIdx.x == 0) part[c] = v;
  }
  // thread 0 stored every partial of this CTA; its arrival publishes them
  if (threadIdx.x == 0) pyc_last = pyc_ticket_arrive(ticket) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!pyc_last) return;
  const pyc_record r = pyc_record_partials(part, (int)nchunks);
  if (threadIdx.x == 0) {
    *rec = r;
    *ticket = 0u;
  }
}

// Batched reduction: one task per segment.
struct pyc_task {
  pyc_args args;
  pyc_i64 n;
  pyc_i64 head;
  pyc_i64 chunk;
  pyc_out_t* out;
  int nchunks;   // 0: the task is reduced by one warp of a bundle item
  int slot0;     // first partial slot (tasks with nchunks > 1)
};
// chunk >= 0: a CTA reduces chunk `chunk` of task `task`;
// chunk <  0: warp w reduces task `task + w` for w < count.
struct pyc_item {
  int task;
  int chunk;
  int count;
  int pad;
};
)PYC";
  o << "static_assert(sizeof(pyc_task) == " << g.task_bytes << ", \"task layout\");\n";
  o << R"PYC(
// WU: unroll of the one-warp tasks (at most 2048 elements; the register-lean
// build uses 1 there).
template <int VB, int U, int WU>
__device__ __forceinline__ void pyc_batched_body(const pyc_task* __restrict__ tasks,
    const pyc_item* __restrict__ items, const int nitems, pyc_acc_t* __restrict__ part,
    unsigned* __restrict__ tickets, unsigned* __restrict__ ctl) {
  // Item order as in the batched map: CTA b takes item b first, then the
  // counter's (offset by the grid), the next index fetched while this item runs.
  __shared__ int pyc_it[2];
  __shared__ unsigned pyc_last;
  int it = (int)blockIdx.x;
  for (int k = 0; it < nitems; ++k) {
    int next = 0;
    if (threadIdx.x == 0) next = (int)gridDim.x + (int)atomicAdd(&ctl[0], 1u);
    const pyc_item I = items[it];
    if (I.chunk < 0) {
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (w < I.count) {
        const pyc_task& T = tasks[I.task + w];
        pyc_acc_t v = pyc_chunk<VB, WU>(T.args, T.n, T.head, T.chunk, 0, lane, 32);
        v = pyc_warp_reduce(v, pyc_combine_op());
        if (lane == 0) *T.out = pyc_finalize(v);
      }
    } else {
      const pyc_task& T = tasks[I.task];
      pyc_acc_t v = pyc_chunk<VB, U>(T.args, T.n, T.head, T.chunk, I.chunk, threadIdx.x, blockDim.x);
      v = pyc_block_reduce(v, pyc_combine_op(), pyc_neutral());
      if (T.nchunks == 1) {
        if (threadIdx.x == 0) *T.out = pyc_finalize(v);
      } else {
        if (threadIdx.x == 0) {
          part[T.slot0 + I.chunk] = v;
          __threadfence();
          pyc_last = atomicAdd(&tickets[I.task], 1u) == (unsigned)(T.nchunks - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (pyc_last) {
          __threadfence();
          const pyc_out_t r = pyc_combine_partials(part + T.slot0, T.nchunks);
          if (threadIdx.x == 0) {
            *T.out = r;
            tickets[I.task] = 0u;
          }
        }
      }
    }
    if (threadIdx.x == 0) pyc_it[k & 1] = next;
    __syncthreads();
    it = pyc_it[k & 1];
  }
  // the last CTA to leave resets the work counter for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl[1], 1u) == gridDim.x - 1) {
      ctl[0] = 0u;
      ctl[1] = 0u;
      __threadfence();
    }
  }
}

)PYC";
  // Entry points: the main module holds the single and batched reductions; the
  // extra module, compiled on first use, the sharded reduction, the combine of
  // shard records and the register-lean batched builds.  One compilation unit
  // per kernel (kUnitMark): NVRTC compiles them in parallel.
  std::ostringstream m, x;
  for (auto& v : all_variants()) {
    std::string sfx = variant_suffix(v);
    m << kUnitMark;
    m << "extern \"C\" __global__ void __launch_bounds__(512) pyc_reduce_" << tag << "_" << sfx
      << "(const pyc_args pyc_p, const pyc_i64 n, const pyc_i64 head, const pyc_i64 chunk, "
         "const pyc_i64 nchunks, pyc_acc_t* part, unsigned* ticket, pyc_out_t* out) {\n"
      << "  pyc_reduce_body<" << v.vec_bytes << ", " << v.unroll
      << ">(pyc_p, n, head, chunk, nchunks, part, ticket, out);\n}\n";
    m << kUnitMark;
    m << "extern \"C\" __global__ void __launch_bounds__(512) pyc_rbatch_" << tag << "_" << sfx
      << "(const pyc_task* tasks, const pyc_item* items, const int nitems, pyc_acc_t* part, "
         "unsigned* tickets, unsigned* ctl) {\n"
      << "  pyc_batched_body<" << v.vec_bytes << ", " << v.unroll << ", " << v.unroll
      << ">(tasks, items, nitems, part, tickets, ctl);\n}\n";
    x << kUnitMark;
    x << "extern \"C\" __global__ void __launch_bounds__(512) pyc_rshard_" << tag << "_" << sfx
      << "(const pyc_args pyc_p, const pyc_i64 n, const pyc_i64 base, const pyc_i64 len, "
         "const pyc_i64 head, const pyc_i64 chunk, const pyc_i64 nchunks, pyc_acc_t* part, "
         "unsigned* ticket, pyc_record* rec) {\n"
      << "  pyc_shard_body<" << v.vec_bytes << ", " << v.unroll
      << ">(pyc_p, n, base, len, head, chunk, nchunks, part, ticket, rec);\n}\n";
    // register-lean build of the 16-byte variants (a tuning candidate): at most
    // kLeanRegs registers, so more CTAs -- and more loads in flight -- per SM
    if (v.vec_bytes == 16)
      x << kUnitMark
        << "extern \"C\" __global__ void __maxnreg__(" << kLeanRegs << ") pyc_rbatch_" << tag << "_"
        << sfx << "_r" << kLeanRegs
        << "(const pyc_task* tasks, const pyc_item* items, const int nitems, pyc_acc_t* part, "
           "unsigned* tickets, unsigned* ctl) {\n"
        << "  pyc_batched_body<" << v.vec_bytes << ", " << v.unroll
        << ", 1>(tasks, items, nitems, part, tickets, ctl);\n}\n";
  }
  x << kUnitMark;
  x << "extern \"C\" __global__ void __launch_bounds__(" << kCombineBlock << ") pyc_rcomb_" << tag
    << "(const pyc_record* rec, const pyc_i64 k, pyc_out_t* out) {\n"
       "  const pyc_out_t r = pyc_combine_records(rec, k);\n"
       "  if (threadIdx.x == 0) *out = r;\n}\n";
  const std::string common = o.str();
  if (emit_kernels) {
    g.source = common + m.str();
    g.source_ext = common + x.str();
  } else {
    g.source = common;
  }
  return g;
}

ScanGen generate_scan(const ArgSpec& spec, pyc_dtype dtype, const std::string& neutral,
                      const std::string& scan_expr, const std::string& input_expr,
                      const std::string& output_stmt, const std::string& preamble,
                      const std::string& tag) {
  ReduceGen core = generate_reduce(spec, dtype, ReduceKind::Plain, neutral, scan_expr, input_expr,
                                   preamble, tag, 0, false);
  ScanGen g;
  g.acc_bytes = core.acc_bytes;
  g.stage_elem_bytes = stage_elem_bytes(spec);
  std::ostringstream o;
  o << core.source;
  // The scan of one step's rows with the output statement, then the vector
  // stores of the written arrays: shared by both forms of sweep 2.
  const std::string scan_rows = std::string(R"PYC(#pragma unroll
    for (int pyc_u = 0; pyc_u < RU; ++pyc_u) {
      pyc_acc_t pyc_l[E];
#pragma unroll
      for (int pyc_e = 0; pyc_e < E; ++pyc_e) {
        const int pyc_k = pyc_u * E + pyc_e;
        const pyc_i64 i = pyc_gb + (pyc_i64)pyc_u * (32 * E) + pyc_e;
        (void)i;
        pyc_acc_t pyc_x = pyc_neutral();
        if (!RAG || i < te) pyc_x = (pyc_acc_t)()PYC") + input_expr + R"PYC();
        pyc_l[pyc_e] = pyc_e == 0 ? pyc_x : pyc_combine(pyc_l[pyc_e - 1], pyc_x);
      }
      const pyc_acc_t pyc_in = pyc_warp_incl_scan(pyc_l[E - 1]);
      pyc_acc_t pyc_ex = pyc_shfl_up(pyc_in, 1);
      if (lane == 0) pyc_ex = pyc_neutral();
      const pyc_acc_t pyc_p0 = pyc_combine(pyc_run, pyc_ex);
#pragma unroll
      for (int pyc_e = 0; pyc_e < E; ++pyc_e) {
        const int pyc_k = pyc_u * E + pyc_e;
        const pyc_i64 i = pyc_gb + (pyc_i64)pyc_u * (32 * E) + pyc_e;
        (void)i;
        const pyc_acc_t item = pyc_combine(pyc_p0, pyc_l[pyc_e]);
        const pyc_acc_t prev_item = pyc_e == 0 ? pyc_p0 : pyc_combine(pyc_p0, pyc_l[pyc_e - 1]);
        (void)item;
        (void)prev_item;
        if (!RAG || i < te) {
          { )PYC" + output_stmt + R"PYC( ; }
          if constexpr (RAG) {
            if (PYC_OK(S, i, 1, S.n, 23, t)) {
)PYC" + scalar_stores_k(spec) + R"PYC(            }
          }
        }
      }
      pyc_run = pyc_combine(pyc_run, pyc_shfl_idx(pyc_in, 31));
    }
    if constexpr (!RAG) {
#pragma unroll
      for (int pyc_u = 0; pyc_u < RU; ++pyc_u) {
        const pyc_i64 pyc_e0 = pyc_gb + (pyc_i64)pyc_u * (32 * E);
        if (PYC_OK(S, pyc_e0, E, S.n, 24, t)) {
)PYC" + with_policy(group_io(spec, false), "pyc_pd") + "        }\n      }\n    }\n";

  o << R"PYC(
// ------------------------------------------------------------------ scan
template <typename T>
__device__ __forceinline__ T pyc_shfl_up(const T v, int d) {
  pyc_words<T> u;
  u.t = v;
#pragma unroll
  for (int j = 0; j < (int)(sizeof(T) / 4); ++j) u.w[j] = __shfl_up_sync(0xffffffffu, u.w[j], d);
  return u.t;
}
// Inclusive scan across a warp in lane order (the earlier operand on the left).
__device__ __forceinline__ pyc_acc_t pyc_warp_incl_scan(pyc_acc_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const pyc_acc_t o = pyc_shfl_up(v, d);
    if (lane >= d) v = pyc_combine(o, v);
  }
  return v;
}
template <typename T>
__device__ __forceinline__ T pyc_shfl_idx(const T v, int src) {
  pyc_words<T> u;
  u.t = v;
#pragma unroll
  for (int j = 0; j < (int)(sizeof(T) / 4); ++j) u.w[j] = __shfl_sync(0xffffffffu, u.w[j], src);
  return u.t;
}
__device__ __forceinline__ unsigned pyc_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void pyc_st_release(unsigned* p, const unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Launch parameters of the single-pass scan.  Tile t publishes a descriptor:
// flag[t] = epoch << 2 | state, state 1 = its aggregate is in agg[t], state 2 =
// its inclusive prefix is in inc[t].  ctl[0] hands out tile indices in order,
// ctl[1] counts CTAs that have finished (the last one resets both), ctl[2] is
// the error word (non-zero after a wait gave up; cleared by the host) and
// ctl[3] the epoch of the last launch in which a wait gave up.
struct pyc_scan_params {
  unsigned* flag;
  pyc_acc_t* agg;
  pyc_acc_t* inc;
  unsigned long long* ctl;
  pyc_i64 n;
  pyc_i64 head;         // < 0: every tile is ragged; else [0, head) is tile 0 if head > 0
  pyc_i64 nfull;        // vector tiles of `groups` row groups per warp after the head
  pyc_i64 ntiles;
  pyc_i64 spin_limit;   // polls of one descriptor window before giving up
  pyc_i64 stall_tile;   // test hook: this tile publishes nothing (-1: none)
  unsigned epoch;
  unsigned groups;      // row groups per warp in a vector tile
  unsigned tail_groups; // row groups of the vector tile after them (0: none)
  unsigned pad;
};
static_assert(sizeof(pyc_scan_params) == 96, "scan params layout");

// Bounds-checked build (PYC_CHECK defined): every access of the scan checks
// [idx, idx + cnt) against [0, bound); the first violation is recorded in
// ctl[4..7] (code, index, tile, block << 16 | thread) and the access skipped.
#ifdef PYC_CHECK
__device__ __noinline__ bool pyc_check_fail(const pyc_scan_params& S, const pyc_i64 idx,
                                            const int code, const pyc_i64 t) {
  if (atomicCAS(S.ctl + 4, 0ull, (unsigned long long)code) == 0ull) {
    S.ctl[5] = (unsigned long long)idx;
    S.ctl[6] = (unsigned long long)t;
    S.ctl[7] = ((unsigned long long)blockIdx.x << 16) | threadIdx.x;
  }
  return false;
}
// PYC_SCAN_SHRINK (a test hook) narrows the array ranges (codes below 30) by
// that many elements at their top; descriptor ranges are never narrowed.
#ifndef PYC_SCAN_SHRINK
#define PYC_SCAN_SHRINK 0
#endif
#define PYC_OK(S, idx, cnt, bound, code, t)                                        \
  (((pyc_i64)(idx) >= 0 &&                                                         \
    (pyc_i64)(idx) + (pyc_i64)(cnt) <=                                             \
        (pyc_i64)(bound) - ((code) < 30 ? (pyc_i64)PYC_SCAN_SHRINK : 0)) ||        \
   pyc_check_fail(S, (pyc_i64)(idx), code, t))
#else
#define PYC_OK(S, idx, cnt, bound, code, t) true
#endif

// Descriptors of 4-byte values are packed: one 64-bit word per tile holding
// (epoch << 2 | state) << 32 | value, written and read with single 64-bit
// accesses (atomic), so a reader that sees the state sees its value.  Wider
// values keep the state in flag[t] and the value in agg[t] / inc[t], ordered
// by release / acquire.
#define PYC_PACKED (sizeof(pyc_acc_t) == 4)
__device__ __forceinline__ void pyc_publish(const pyc_scan_params& S, const pyc_i64 t,
                                            const unsigned state, const pyc_acc_t v) {
  if (t == S.stall_tile) return;
  if (!PYC_OK(S, t, 1, S.ntiles, 31, t)) return;
  if constexpr (PYC_PACKED) {
    pyc_words<pyc_acc_t> u;
    u.t = v;
    const unsigned long long word =
        ((unsigned long long)((S.epoch << 2) | state) << 32) | (unsigned long long)u.w[0];
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;"
                 ::"l"(reinterpret_cast<unsigned long long*>(S.flag) + t), "l"(word) : "memory");
  } else {
    if (state == 1u) S.agg[t] = v;
    else S.inc[t] = v;
    pyc_st_release(S.flag + t, (S.epoch << 2) | state);
  }
}

// Exclusive prefix of tile t > 0, computed by one warp: look back over the
// descriptors of tiles t-1, t-2, ... in windows of 32 lanes x PYC_LB_K tiles
// (lane l reads the aligned group of PYC_LB_K descriptors l groups below the
// one holding t-1, flags with one relaxed vector load and an acquire fence)
// until a window holds an inclusive prefix with every tile after it
// published; the aggregates after it are combined in tile order.  Every tile
// below t was handed out before t, so its CTA is running and publishes
// without waiting on this one.  The wait is bounded: after spin_limit polls
// (or once another CTA of the same launch has given up) the error word is set
// and the neutral element is returned.
#define PYC_LB_K 4
__device__ __noinline__ pyc_acc_t pyc_lookback(const pyc_scan_params& S, const pyc_i64 t) {
  constexpr int K = PYC_LB_K;
  const int lane = threadIdx.x & 31;
  const unsigned want = S.epoch;
  pyc_acc_t run = pyc_neutral();
  pyc_i64 g0 = (t - 1) / K;
  pyc_i64 polls = 0;
  for (;;) {
    const pyc_i64 g = g0 - lane;
    unsigned st[K];  // 0: not published, 1: aggregate, 2: inclusive prefix, 3: not a predecessor
    unsigned val[K];  // packed descriptors: the value bits
    bool has_p, x_above;
    int jp;
    for (;;) {
      if (g >= 0 && PYC_OK(S, g * K, K, S.ntiles + K - 1, 32, t)) {
        unsigned f[K];
        if constexpr (PYC_PACKED) {
          unsigned long long d[K];
          asm volatile("ld.relaxed.gpu.global.v4.b64 {%0,%1,%2,%3}, [%4];"
                       : "=l"(d[0]), "=l"(d[1]), "=l"(d[2]), "=l"(d[3])
                       : "l"(reinterpret_cast<const unsigned long long*>(S.flag) + g * K)
                       : "memory");
#pragma unroll
          for (int j = 0; j < K; ++j) {
            f[j] = (unsigned)(d[j] >> 32);
            val[j] = (unsigned)d[j];
          }
        } else {
          asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                       : "=r"(f[0]), "=r"(f[1]), "=r"(f[2]), "=r"(f[3]) : "l"(S.flag + g * K)
                       : "memory");
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
          st[j] = g * K + j >= t ? 3u : ((f[j] >> 2) == want ? (f[j] & 3u) : 0u);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) st[j] = 2u;  // below tile 0: never selected
      }
      // from the top of the lane's group down: the first inclusive prefix, and
      // whether a tile above it has not published yet
      has_p = false;
      x_above = false;
      jp = 0;
#pragma unroll
      for (int j = K - 1; j >= 0; --j) {
        if (has_p || st[j] == 3u) continue;
        if (st[j] == 2u) {
          has_p = true;
          jp = j;
        } else if (st[j] == 0u) {
          x_above = true;
        }
      }
      const unsigned pm = __ballot_sync(0xffffffffu, has_p);
      const unsigned xm = __ballot_sync(0xffffffffu, x_above);
      if (pm ? (xm & ((2u << (__ffs(pm) - 1)) - 1u)) == 0u : xm == 0u) break;
      ++polls;
      bool give_up = polls > S.spin_limit;
      if ((polls & 63) == 0)
        give_up |= *(volatile const unsigned long long*)(S.ctl + 3) == (unsigned long long)want;
      if (__any_sync(0xffffffffu, give_up)) {
        if (lane == 0) {
          atomicOr(S.ctl + 2, polls > S.spin_limit ? 1ull : 2ull);
          atomicExch(S.ctl + 3, (unsigned long long)want);
        }
        return pyc_neutral();
      }
      __nanosleep(32);
    }
    if constexpr (!PYC_PACKED) asm volatile("fence.acq_rel.gpu;" ::: "memory");
    const unsigned pm = __ballot_sync(0xffffffffu, has_p);
    const int p = pm ? __ffs(pm) - 1 : 31;
    pyc_acc_t v = pyc_neutral();
    if (lane <= p && g >= 0) {
      // this lane's tiles from its first inclusive prefix (lane p) or its lowest
      // tile (lanes above p) up to its top, in tile order
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if (st[j] == 3u || (lane == p && j < jp)) continue;
        if (!PYC_OK(S, g * K + j, 1, S.ntiles, 33, t)) continue;
        pyc_acc_t d;
        if constexpr (PYC_PACKED) {
          pyc_words<pyc_acc_t> u;
          u.w[0] = val[j];
          d = u.t;
        } else {
          d = st[j] == 2u ? pyc_ld_cg(S.inc + g * K + j) : pyc_ld_cg(S.agg + g * K + j);
        }
        v = pyc_combine(v, d);
      }
    }
    // ordered fold: lane p (earliest tiles) first, lane 0 (tile t-1) last
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const pyc_acc_t o = pyc_shfl_down(v, d);
      if (lane + d < 32) v = pyc_combine(o, v);
    }
    run = pyc_combine(pyc_shfl_idx(v, 0), run);
    if (pm) return run;
    g0 -= 32;
  }
}

// Intra-CTA hand-offs: mbarriers, waited on with a bounded loop.
__device__ __forceinline__ unsigned pyc_saddr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void pyc_mbar_init(unsigned long long* bar, const unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(pyc_saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void pyc_mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(pyc_saddr(bar)) : "memory");
}
__device__ __forceinline__ bool pyc_mbar_try_wait(unsigned long long* bar, const unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(pyc_saddr(bar)), "r"(parity) : "memory");
  return ok != 0u;
}
// Waits for the phase of `bar` with the given parity to complete; false (and
// bit 8 set in the error word) if it has not after about 2^25 polls, a bound
// well above the look-back's own.
__device__ __forceinline__ bool pyc_mbar_wait(unsigned long long* bar, const unsigned parity,
                                              unsigned long long* err) {
  for (unsigned it = 0; !pyc_mbar_try_wait(bar, parity); ++it) {
    if (it > (1u << 25)) {
      atomicOr(err, 8ull);
      return false;
    }
    if (it > 64u) __nanosleep(128);
  }
  return true;
}

// Rows of a tile: warp w (of nw compute warps) owns rows [w*G*U, (w+1)*G*U),
// each of 32*E consecutive elements, lane l holding E consecutive elements of
// a row.  A vector tile is aligned and full: U rows at a time, one coalesced
// vector per array and row.  A ragged tile [ts, te) takes one row at a time
// with element-wise accesses where i < te.

// Sweep 1: the warp's aggregate in element order (valid in lane 0).
template <int VB, int U, bool RAG>
__device__ __forceinline__ pyc_acc_t pyc_sweep1(const pyc_args& pyc_p, const pyc_scan_params& S,
    const pyc_i64 t, const pyc_i64 ts, const pyc_i64 te, const int G, const int w,
    const int lane) {
  constexpr int E = VB / PYC_MIN_BYTES;
  constexpr int RU = RAG ? 1 : U;  // rows per step
  constexpr int T = E * RU;
)PYC";
  o << aliases(spec, "pyc_p");
  o << R"PYC(  (void)te;
  const pyc_i64 pyc_wb = ts + (pyc_i64)w * G * (U * 32 * E) + (pyc_i64)lane * E;
  // the tile is read again by sweep 2: keep it in L2
  const unsigned long long pyc_pk = pyc_policy_keep();
  pyc_acc_t pyc_wagg = pyc_neutral();
  const int pyc_steps = G * (U / RU);
  if constexpr (RAG) {
    for (int pyc_g = 0; pyc_g < pyc_steps; ++pyc_g) {
      const pyc_i64 pyc_gb = pyc_wb + (pyc_i64)pyc_g * (32 * E);
)PYC";
  o << reg_decls(spec, "T");
  o << R"PYC(#pragma unroll
      for (int pyc_k = 0; pyc_k < T; ++pyc_k) {
        const pyc_i64 i = pyc_gb + pyc_k;
        if (i < te) {
)PYC";
  o << "          if (PYC_OK(S, i, 1, S.n, 12, t)) {\n" << scalar_loads_k(spec, input_expr)
    << "          }\n";
  o << R"PYC(        }
      }
)PYC";
  o << fold_rows(input_expr, "pyc_gb", true);
  o << R"PYC(    }
  } else {
    // two register buffers: the rows of group g+1 load while group g folds
    const pyc_i64 pyc_step = 32 * E;
    constexpr int pyc_gs = U * 32 * E;  // elements between a warp's row groups
)PYC";
  o << buf_decls(spec, "pyc_a_", "T") << buf_decls(spec, "pyc_b_", "T");
  auto load = [&](const char* prefix, const std::string& base) {
    std::string l = buf_load_used(spec, prefix, base, input_expr);
    return "    if (PYC_OK(S, " + base + ", pyc_gs - 31 * E, S.n, 11, t)) {\n" +
           with_policy(l, "pyc_pk") + "    }\n";
  };
  o << load("pyc_a_", "pyc_wb");
  o << R"PYC(    for (int pyc_g = 0; pyc_g < pyc_steps; pyc_g += 2) {
      const pyc_i64 pyc_gb = pyc_wb + (pyc_i64)pyc_g * pyc_gs;
      if (pyc_g + 1 < pyc_steps) {
)PYC";
  o << load("pyc_b_", "pyc_gb + pyc_gs");
  o << "      }\n      {\n" << buf_refs(spec, "pyc_a_") << fold_rows(input_expr, "pyc_gb", false)
    << "      }\n";
  o << R"PYC(      if (pyc_g + 1 < pyc_steps) {
        if (pyc_g + 2 < pyc_steps) {
)PYC";
  o << load("pyc_a_", "pyc_gb + 2 * pyc_gs");
  o << "        }\n        {\n" << buf_refs(spec, "pyc_b_")
    << fold_rows(input_expr, "pyc_gb + pyc_gs", false) << "        }\n      }\n";
  o << R"PYC(    }
  }
  return pyc_wagg;
}

// Sweep 2: the warp's rows again (from L2), scanned from `run` (everything
// before the warp's first element), with the output statement.
template <int VB, int U, bool RAG>
__device__ __forceinline__ void pyc_sweep2(const pyc_args& pyc_p, const pyc_scan_params& S,
    const pyc_i64 t, const pyc_i64 ts, const pyc_i64 te, const int G, const int w,
    const int lane, pyc_acc_t pyc_run) {
  constexpr int E = VB / PYC_MIN_BYTES;
  constexpr int RU = RAG ? 1 : U;
  constexpr int T = E * RU;
)PYC";
  o << aliases(spec, "pyc_p");
  o << R"PYC(  (void)te;
  const pyc_i64 pyc_wb = ts + (pyc_i64)w * G * (U * 32 * E) + (pyc_i64)lane * E;
  // the last use of the input, and output that is not read here: evict first
  const unsigned long long pyc_pd = pyc_policy_drop();
  const int pyc_steps = G * (U / RU);
  for (int pyc_g = 0; pyc_g < pyc_steps; ++pyc_g) {
    const pyc_i64 pyc_gb = pyc_wb + (pyc_i64)pyc_g * (RU * 32 * E);
)PYC";
  o << reg_decls(spec, "T");
  o << R"PYC(    if constexpr (RAG) {
#pragma unroll
      for (int pyc_k = 0; pyc_k < T; ++pyc_k) {
        const pyc_i64 i = pyc_gb + pyc_k;
        if (i < te) {
)PYC";
  o << "          if (PYC_OK(S, i, 1, S.n, 21, t)) {\n" << scalar_loads_k(spec, "")
    << "          }\n";
  o << R"PYC(        }
      }
    } else {
#pragma unroll
      for (int pyc_u = 0; pyc_u < RU; ++pyc_u) {
        const pyc_i64 pyc_e0 = pyc_gb + (pyc_i64)pyc_u * (32 * E);
)PYC";
  o << "        if (PYC_OK(S, pyc_e0, E, S.n, 22, t)) {\n"
    << with_policy(group_io(spec, true), "pyc_pd") << "        }\n";
  o << "      }\n    }\n" << scan_rows << "  }\n}\n";
  o << R"PYC(

// Tile t: [ts, te), row groups per warp, and whether it is ragged.  Order: the
// scalar head (if head > 0), nfull vector tiles of `groups` row groups, one of
// `tail_groups` (if any), the ragged rest; with head < 0 every tile is ragged.
struct pyc_tinfo {
  pyc_i64 ts, te;
  int g;
  bool rag;
};
__device__ __forceinline__ pyc_tinfo pyc_tile_info(const pyc_scan_params& S, const pyc_i64 t,
                                                   const pyc_i64 base) {
  const pyc_i64 tile = base * S.groups;
  const pyc_i64 htile = S.head > 0 ? 1 : 0;
  pyc_tinfo r;
  if (S.head < 0) {
    r.ts = t * tile;
    r.te = r.ts + tile < S.n ? r.ts + tile : S.n;
    r.g = (int)S.groups;
    r.rag = true;
  } else if (t < htile) {
    r.ts = 0;
    r.te = S.head;
    r.g = 1;
    r.rag = true;
  } else if (t < htile + S.nfull) {
    r.ts = S.head + (t - htile) * tile;
    r.te = r.ts + tile;
    r.g = (int)S.groups;
    r.rag = false;
  } else if (t == htile + S.nfull && S.tail_groups > 0) {
    r.ts = S.head + S.nfull * tile;
    r.te = r.ts + base * S.tail_groups;
    r.g = (int)S.tail_groups;
    r.rag = false;
  } else {
    r.ts = S.head + S.nfull * tile + base * S.tail_groups;
    r.te = S.n;
    r.g = 1;
    r.rag = true;
  }
  return r;
}

// Start the whole input of tile [ts, te) moving from DRAM into L2 at once, so
// that sweep 1 is not held to the loads its registers can keep in flight.
)PYC";
  o << "__device__ __forceinline__ void pyc_prefetch_tile(const pyc_args& pyc_p, const pyc_i64 ts,\n"
       "    const pyc_i64 te, const int tid, const int nt) {\n";
  o << aliases(spec, "pyc_p");
  o << prefetch_used(spec, input_expr);
  o << "  (void)ts; (void)te; (void)tid; (void)nt;\n}\n";
  o << R"PYC(
// The look-back warp of a CTA (warp nw): for each tile the compute warps fold
// (slot k & 1), scan the warp aggregates, find the tile's exclusive prefix,
// publish its inclusive prefix and hand back the prefix of each compute warp's
// rows.  false if a wait ran out.
__device__ __forceinline__ bool pyc_lookback_warp(const pyc_scan_params& S, const int nw,
    const int lane, pyc_acc_t (*pyc_tot)[32], pyc_acc_t (*pyc_off)[32], pyc_i64* pyc_tq,
    unsigned long long* pyc_ma, unsigned long long* pyc_mp, unsigned long long* err) {
  for (int k = 0;; ++k) {
    const int sl = k & 1;
    const unsigned ph = (unsigned)(k >> 1) & 1u;
    if (!pyc_mbar_wait(&pyc_ma[sl], ph, err)) return false;
    const pyc_i64 t = pyc_tq[sl];
    if (t >= S.ntiles || !PYC_OK(S, t, 0, S.ntiles, 41, t)) return true;
    pyc_acc_t s = lane < nw ? pyc_tot[sl][lane] : pyc_neutral();
    s = pyc_warp_incl_scan(s);
    const pyc_acc_t agg = pyc_shfl_idx(s, nw - 1);  // (all lanes: a warp-wide shuffle)
    pyc_acc_t ex = pyc_neutral();
    if (t > 0) {
      ex = pyc_lookback(S, t);
      if (lane == 0) pyc_publish(S, t, 2u, pyc_combine(ex, agg));
    }
    pyc_acc_t o = pyc_shfl_up(s, 1);
    if (lane == 0) o = pyc_neutral();
    if (lane < nw) pyc_off[sl][lane] = pyc_combine(ex, o);
    __syncwarp();
    if (lane == 0) pyc_mbar_arrive(&pyc_mp[sl]);
  }
}

// A compute warp stores its aggregate `a` of tile t; the last of the nw warps to
// do so publishes the tile's aggregate at once (its inclusive prefix for tile
// 0), so that later tiles need not wait for this CTA's look-back warp.
__device__ __forceinline__ void pyc_store_aggregate(const pyc_scan_params& S, const pyc_i64 t,
    const int nw, const int w, const int lane, const pyc_acc_t a, pyc_acc_t* tot,
    unsigned* cnt) {
  unsigned last = 0u;
  if (lane == 0) {
    tot[w] = a;
    __threadfence_block();
    last = atomicAdd(cnt, 1u) == (unsigned)nw - 1u ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence_block();
    pyc_acc_t s = lane < nw ? tot[lane] : pyc_neutral();
    s = pyc_warp_incl_scan(s);
    const pyc_acc_t agg = pyc_shfl_idx(s, nw - 1);
    if (lane == 0) {
      pyc_publish(S, t, t == 0 ? 2u : 1u, agg);
      *cnt = 0u;
    }
  }
}

// Persistent single-pass scan with a look-back warp.  The CTA has nw compute
// warps and one look-back warp (the last).  Iteration k of the compute warps:
// take tile k, sweep 1 over it, publish its aggregate and hand the warp
// aggregates to the look-back warp, then (once its prefix is known) sweep 2
// over tile k-1.  The look-back warp finds tile k's exclusive prefix, publishes
// its inclusive prefix and hands back the prefix of every compute warp's rows,
// so the look-back of one tile runs while the compute warps scan the previous
// tile and fold the next.  Slots alternate with the parity of k:
//   m_tile[s]  compute warp 0 has posted the tile index (1 arrival),
//   m_agg[s]   every compute warp has stored its aggregate (nw arrivals),
//   m_pre[s]   the look-back warp has stored the warp prefixes (1 arrival);
// a slot is reused two iterations later, after both sides have passed the
// hand-off of the iteration between, so no wait can miss its phase.  The last
// compute warp to store its aggregate (a shared counter) publishes the tile's.
// A wait that runs out sets the error word and ends the CTA.
template <int VB, int U>
__device__ __forceinline__ void pyc_scan_body(const pyc_args& pyc_p, const pyc_scan_params& S) {
  constexpr int R = 32 * (VB / PYC_MIN_BYTES) * U;  // elements of one row group of a warp
  __shared__ pyc_acc_t pyc_tot[2][32];
  __shared__ pyc_acc_t pyc_off[2][32];
  __shared__ pyc_i64 pyc_tq[2];
  __shared__ unsigned pyc_cnt[2];
  __shared__ __align__(8) unsigned long long pyc_mt[2], pyc_ma[2], pyc_mp[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5) - 1;
  const pyc_i64 base = (pyc_i64)nw * R;
  unsigned long long* const err = S.ctl + 2;
  if (threadIdx.x == 0) {
    for (int j = 0; j < 2; ++j) {
      pyc_mbar_init(&pyc_mt[j], 1u);
      pyc_mbar_init(&pyc_ma[j], (unsigned)nw);
      pyc_mbar_init(&pyc_mp[j], 1u);
      pyc_cnt[j] = 0u;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (w == nw) {
    if (!pyc_lookback_warp(S, nw, lane, pyc_tot, pyc_off, pyc_tq, pyc_ma, pyc_mp, err)) return;
  } else {
    pyc_i64 tprev = -1;
    for (int k = 0;; ++k) {
      const int sl = k & 1;
      const unsigned ph = (unsigned)(k >> 1) & 1u;
      if (threadIdx.x == 0) {
        pyc_tq[sl] = (pyc_i64)atomicAdd(S.ctl, 1ull);
        pyc_mbar_arrive(&pyc_mt[sl]);
      }
      if (!pyc_mbar_wait(&pyc_mt[sl], ph, err)) return;
      const pyc_i64 t = pyc_tq[sl];
      if (t < S.ntiles && PYC_OK(S, t, 0, S.ntiles, 42, t)) {
        const pyc_tinfo I = pyc_tile_info(S, t, base);
        if (!PYC_OK(S, I.ts, I.te - I.ts, S.n, 43, t)) return;
        pyc_prefetch_tile(pyc_p, I.ts, I.te, (int)threadIdx.x, nw * 32);
        const pyc_acc_t a =
            I.rag ? pyc_sweep1<VB, U, true>(pyc_p, S, t, I.ts, I.te, I.g, w, lane)
                  : pyc_sweep1<VB, U, false>(pyc_p, S, t, I.ts, I.te, I.g, w, lane);
        pyc_store_aggregate(S, t, nw, w, lane, a, pyc_tot[sl], &pyc_cnt[sl]);
      }
      __syncwarp();
      if (lane == 0) pyc_mbar_arrive(&pyc_ma[sl]);
      if (tprev >= 0) {
        const int sp = (k - 1) & 1;
        if (!pyc_mbar_wait(&pyc_mp[sp], (unsigned)((k - 1) >> 1) & 1u, err)) return;
        const pyc_tinfo I = pyc_tile_info(S, tprev, base);
        const pyc_acc_t run = pyc_off[sp][w];
        if (I.rag) pyc_sweep2<VB, U, true>(pyc_p, S, tprev, I.ts, I.te, I.g, w, lane, run);
        else pyc_sweep2<VB, U, false>(pyc_p, S, tprev, I.ts, I.te, I.g, w, lane, run);
      }
      if (t >= S.ntiles) break;
      tprev = t;
    }
  }
  // the last CTA to leave resets the tile counter for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(S.ctl + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
      S.ctl[0] = 0ull;
      S.ctl[1] = 0ull;
      __threadfence();
    }
  }
}

)PYC";
  // one compilation unit per kernel (kUnitMark): NVRTC compiles them in parallel
  for (auto& v : all_variants()) {
    std::string sfx = variant_suffix(v);
    o << kUnitMark;
    o << "extern \"C\" __global__ void __launch_bounds__(544) pyc_scan_" << tag << "_" << sfx
      << "(const pyc_args pyc_p, const pyc_scan_params S) {\n"
      << "  pyc_scan_body<" << v.vec_bytes << ", " << v.unroll << ">(pyc_p, S);\n}\n";
  }
  g.source = o.str();
  return g;
}

}  // namespace pyc
