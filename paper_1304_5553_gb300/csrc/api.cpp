// C ABI: map and map-reduce creation and launches (see include/pyc.h).
#include <algorithm>
#include <cctype>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

int size_bucket(int64_t n) {
  int bl = 0;
  for (uint64_t v = (uint64_t)(n > 0 ? n : 1); v; v >>= 1) ++bl;
  return bl / 2;
}

std::string kernel_tag(const char* name, char prefix, const std::string& spec_text) {
  std::string t;
  if (name)
    for (const char* c = name; *c && t.size() < 40; ++c)
      t += (std::isalnum((unsigned char)*c) ? *c : '_');
  if (t.empty()) t = std::string(1, prefix) + digest(spec_text).substr(0, 8);
  return t;
}

LaunchCfg choose_cfg(HandleBase& h, int64_t n, bool reduce) {
  LaunchCfg c;
  c.v = reduce ? Variant{16, 4} : Variant{16, 4};
  c.block = 256;
  {
    std::lock_guard<std::mutex> lk(h.tune.mu);
    auto it = h.tune.by_bucket.find(size_bucket(n));
    if (it != h.tune.by_bucket.end()) c = it->second;
  }
  if (h.opts.block) c.block = h.opts.block;
  if (h.opts.vec_bytes) c.v.vec_bytes = h.opts.vec_bytes;
  if (h.opts.items_per_thread) c.v.unroll = h.opts.items_per_thread;
  return c;
}

std::vector<unsigned char> pack_args(const ArgSpec& spec, void* const* ptrs, const void* scalars) {
  std::vector<unsigned char> a(spec.params.empty() ? 4 : spec.args_bytes, 0);
  if (spec.num_ptrs > 0 && !ptrs) fail(PYC_E_ARG, "ptrs is NULL but the spec declares arrays");
  if (spec.scalar_bytes > 0 && !scalars)
    fail(PYC_E_ARG, "scalars is NULL but the spec declares scalar parameters");
  const unsigned char* s = static_cast<const unsigned char*>(scalars);
  for (auto& p : spec.params) {
    if (p.is_ptr) {
      void* v = ptrs[p.ptr_slot];
      std::memcpy(&a[p.args_offset], &v, 8);
    } else {
      std::memcpy(&a[p.args_offset], s + p.scalar_offset, type_info(p.dtype).bytes);
    }
  }
  return a;
}

void check_overlap(const ArgSpec& spec, void* const* ptrs, int64_t n) {
  if (n <= 0 || !ptrs) return;
  for (size_t a = 0; a < spec.params.size(); ++a) {
    const auto& p = spec.params[a];
    if (!(p.is_ptr && p.lifted && ptrs[p.ptr_slot])) continue;
    const uintptr_t pa = reinterpret_cast<uintptr_t>(ptrs[p.ptr_slot]);
    const int sa = type_info(p.dtype).bytes;
    for (size_t b = a + 1; b < spec.params.size(); ++b) {
      const auto& q = spec.params[b];
      if (!(q.is_ptr && q.lifted && ptrs[q.ptr_slot]) || !(p.written || q.written)) continue;
      const uintptr_t qa = reinterpret_cast<uintptr_t>(ptrs[q.ptr_slot]);
      const int sb = type_info(q.dtype).bytes;
      if (pa == qa && sa == sb) continue;  // exact aliasing: element i is element i
      const bool disjoint = pa + (uintptr_t)n * sa <= qa || qa + (uintptr_t)n * sb <= pa;
      if (!disjoint)
        fail(PYC_E_ARG, "arrays '" + p.name + "' and '" + q.name +
                            "' overlap in part (only the same pointer with the same element "
                            "type may alias a written array)");
    }
  }
}

int64_t vector_head(const ArgSpec& spec, void* const* ptrs, int vec_bytes, int min_bytes,
                    int64_t n) {
  bool any = false;
  // every array (also one the statement indexes other than as name[i]): a
  // NULL or misaligned one would fault in the kernel
  for (auto& p : spec.params) {
    if (!p.is_ptr) continue;
    uintptr_t a = reinterpret_cast<uintptr_t>(ptrs[p.ptr_slot]);
    int sz = type_info(p.dtype).bytes;
    if (n > 0 && a == 0) fail(PYC_E_ARG, "array '" + p.name + "' is NULL");
    if (a % (uintptr_t)sz)
      fail(PYC_E_ARG, "array '" + p.name + "' is not aligned to its element size");
    any = any || p.lifted;
  }
  if (!any) return 0;
  const int span = vec_bytes / min_bytes;
  for (int h = 0; h < span; ++h) {
    bool ok = true;
    for (auto& p : spec.params) {
      if (!(p.is_ptr && p.lifted)) continue;
      uintptr_t a = reinterpret_cast<uintptr_t>(ptrs[p.ptr_slot]);
      if ((a + (uintptr_t)h * type_info(p.dtype).bytes) % (uintptr_t)vec_bytes) {
        ok = false;
        break;
      }
    }
    if (ok) return h < n ? h : -1;
  }
  return -1;
}

int resident_ctas(CUfunction f, int block, int dyn_smem) {
  static std::mutex mu;
  static std::map<std::tuple<CUfunction, int, int>, int> cache;
  const auto key = std::make_tuple(f, block, dyn_smem);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int nb = 0;
  PYC_CU(drv().cuOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, (size_t)dyn_smem));
  if (nb < 1) fail(PYC_E_ARG, "block size " + std::to_string(block) + " cannot be resident");
  int r = nb * current_device_props().sm_count;
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = r;
  return r;
}

ChunkPlan plan_chunks(int64_t n, int64_t head, int64_t tile, int resident) {
  ChunkPlan p;
  p.head = head;
  int64_t body = n <= 0 ? 0 : (head >= 0 ? n - head : n);
  if (body <= 0) {
    p.chunk = tile;
    p.nchunks = 0;
    p.grid = 1;
    return p;
  }
  auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
  int64_t c = std::max<int64_t>(tile, cdiv(cdiv(body, resident), tile) * tile);
  if (cdiv(body, c) > kMaxChunks) c = cdiv(cdiv(body, kMaxChunks), tile) * tile;
  p.chunk = c;
  p.nchunks = cdiv(body, c);
  p.grid = (int)std::max<int64_t>(1, std::min<int64_t>(resident, p.nchunks));
  return p;
}

bool bounds_requested(const pyc_opts& o) {
  if (o.debug_bounds) return true;
  const char* e = std::getenv("PYC_DEBUG_BOUNDS");
  return e && e[0] == '1';
}

std::string bounds_defines() {
  std::string d = "#define PYC_BOUNDS 1\n";
  if (const char* k = std::getenv("PYC_DEBUG_BOUNDS_SHRINK")) {
    long long v = std::atoll(k);
    if (v > 0) d += "#define PYC_BOUNDS_SHRINK " + std::to_string(v) + "LL\n";
  }
  return d;
}

void check_bounds_record(HandleBase& h, pyc::Module* extra) {
  if (!h.bounds) fail(PYC_E_ARG, "the handle is not a bounds-checked build (opts.debug_bounds)");
  const Driver& d = drv();
  ensure_context();
  PYC_CU(d.cuCtxSynchronize());
  // every unit holds a record of its own: read them all, clear those that are set
  unsigned long long r[4] = {0, 0, 0, 0};
  for (pyc::Module* m : {h.mod.get(), extra}) {
    if (!m) continue;
    size_t bytes = 0;
    for (CUdeviceptr rec : m->globals("pyc_bounds_rec", &bytes)) {
      if (bytes != 32) fail(PYC_E_INTERNAL, "unexpected size of the bounds record");
      unsigned long long q[4] = {0, 0, 0, 0};
      PYC_CU(d.cuMemcpyDtoH(q, rec, sizeof(q)));
      if (q[0] == 0) continue;
      if (r[0] == 0) std::memcpy(r, q, sizeof(r));
      const unsigned long long z[4] = {0, 0, 0, 0};
      PYC_CU(d.cuMemcpyHtoD(rec, z, sizeof(z)));
    }
  }
  if (r[0] == 0) return;
  static const char* what[] = {"?", "vector load", "vector store", "element load",
                               "element store", "vector access"};
  const unsigned code = r[0] < 6 ? (unsigned)r[0] : 0u;
  std::string m = "bounds check: ";
  m += what[code];
  if (code == 5)
    m += " at address " + std::to_string(r[1]) + " not aligned to " + std::to_string(r[2]) +
         " bytes";
  else
    m += " at index " + std::to_string((long long)r[1]) + " outside the array's range (end " +
         std::to_string((long long)r[2]) + ")";
  m += " in " + h.tag + ", block " + std::to_string(r[3] >> 16) + ", thread " +
       std::to_string(r[3] & 0xffff);
  fail(PYC_E_INTERNAL, m);
}

namespace {

void check_cfg(const LaunchCfg& c) {
  bool vb = c.v.vec_bytes == 16 || c.v.vec_bytes == 32;
  bool un = c.v.unroll == 1 || c.v.unroll == 2 || c.v.unroll == 4;
  if (!vb) fail(PYC_E_ARG, "vec_bytes must be 16 or 32");
  if (!un) fail(PYC_E_ARG, "items_per_thread must be 1, 2 or 4");
  if (c.block < 32 || c.block > 512 || c.block % 32)
    fail(PYC_E_ARG, "block must be a multiple of 32 in [32, 512]");
}

pyc_opts opts_or_zero(const pyc_opts* o) {
  pyc_opts z{};
  if (o) z = *o;
  return z;
}

void check_opts(const pyc_opts& o) {
  if (o.block && (o.block < 32 || o.block > 512 || o.block % 32))
    fail(PYC_E_ARG, "opts.block must be 0 or a multiple of 32 in [32, 512]");
  if (o.vec_bytes && o.vec_bytes != 16 && o.vec_bytes != 32)
    fail(PYC_E_ARG, "opts.vec_bytes must be 0, 16 or 32");
  if (o.items_per_thread && o.items_per_thread != 1 && o.items_per_thread != 2 &&
      o.items_per_thread != 4)
    fail(PYC_E_ARG, "opts.items_per_thread must be 0, 1, 2 or 4");
}

void finish_handle(HandleBase& h, bool reduce) {
  h.bounds = bounds_requested(h.opts);
  if (h.bounds) h.source = bounds_defines() + h.source;
  h.min_bytes = lifted_min_bytes(h.spec);
  h.mod = get_module(h.source, h.opts.fmad != 0);
  h.tune_key = digest(h.source + (h.opts.fmad ? "|fmad" : ""));
  h.param_names.clear();
  for (auto& p : h.spec.params) h.param_names.push_back(p.name);
  tune_cache_load(h, reduce);
}

void fill_param(const HandleBase& h, int idx, pyc_param_info* info) {
  if (!info) fail(PYC_E_ARG, "info is NULL");
  if (idx < 0 || idx >= (int)h.spec.params.size()) fail(PYC_E_ARG, "parameter index out of range");
  const Param& p = h.spec.params[idx];
  info->name = h.param_names[idx].c_str();
  info->is_pointer = p.is_ptr;
  info->dtype = p.dtype;
  info->elem_bytes = type_info(p.dtype).bytes;
  info->scalar_offset = p.scalar_offset;
  info->pointer_slot = p.ptr_slot;
  info->read = p.read;
  info->written = p.written;
  info->lifted = p.lifted;
}

}  // namespace

// Launch with programmatic stream serialization: the kernel (which waits for its
// predecessor with griddepcontrol.wait before touching memory) may be scheduled
// while the previous kernel on the stream drains, hiding the launch gap between
// back-to-back launches; the order of memory effects is the stream's.
void launch_dependent(CUfunction f, unsigned grid, unsigned block, CUstream stream,
                      void** params) {
  CUlaunchAttribute at[1];
  at[0].id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
  at[0].value.programmaticStreamSerializationAllowed = 1;
  CUlaunchConfig lc{};
  lc.gridDimX = grid;
  lc.gridDimY = 1;
  lc.gridDimZ = 1;
  lc.blockDimX = block;
  lc.blockDimY = 1;
  lc.blockDimZ = 1;
  lc.sharedMemBytes = 0;
  lc.hStream = stream;
  lc.attrs = at;
  lc.numAttrs = 1;
  PYC_CU(drv().cuLaunchKernelEx(&lc, f, params, nullptr));
}

void launch_map(pyc_map* h, const LaunchCfg& cfg, int64_t n, void* const* ptrs,
                const void* scalars, CUstream stream) {
  check_cfg(cfg);
  if (n < 0) fail(PYC_E_ARG, "n must be >= 0");
  std::vector<unsigned char> args = pack_args(h->spec, ptrs, scalars);
  int64_t head = vector_head(h->spec, ptrs, cfg.v.vec_bytes, h->min_bytes, n);
  check_overlap(h->spec, ptrs, n);
  if (n == 0) return;
  CUfunction f = h->mod->function(h->kname("pyc_map", cfg.v));
  int resident = resident_ctas(f, cfg.block);
  int64_t tile = (int64_t)cfg.block * (cfg.v.vec_bytes / h->min_bytes) * cfg.v.unroll;
  int64_t nfull = head >= 0 ? (n - head) / tile : 0;
  int64_t want = nfull > 0 ? nfull : (n + cfg.block - 1) / cfg.block;
  unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, want));
  void* params[] = {args.data(), &n, &head};
  launch_dependent(f, grid, (unsigned)cfg.block, stream, params);
}

pyc_reduce::Workspace& reduce_workspace(pyc_reduce* h, CUstream stream) {
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(h->ws_mu);
  auto key = std::make_pair(ctx, stream);
  auto it = h->ws.find(key);
  if (it != h->ws.end()) return it->second;
  pyc_reduce::Workspace w;
  size_t part_bytes = (size_t)kMaxChunks * h->gen.acc_bytes;
  size_t total = part_bytes + 256;
  PYC_CU(drv().cuMemAlloc(&w.base, total));
  w.part = w.base;
  w.ticket = w.base + part_bytes;
  const CUresult r = drv().cuMemsetD8Async(w.ticket, 0, 256, stream);
  if (r != CUDA_SUCCESS) {
    drv().cuMemFree(w.base);
    ::pyc::check(r, "cuMemsetD8Async");
  }
  return h->ws.emplace(key, w).first->second;
}

void launch_reduce(pyc_reduce* h, const LaunchCfg& cfg, int64_t n, void* const* ptrs,
                   const void* scalars, void* d_out, CUstream stream) {
  check_cfg(cfg);
  if (n < 0) fail(PYC_E_ARG, "n must be >= 0");
  if (!d_out) fail(PYC_E_ARG, "d_out is NULL");
  if (reinterpret_cast<uintptr_t>(d_out) % (uintptr_t)std::min(h->gen.out_bytes, 8))
    fail(PYC_E_ARG, "d_out is not aligned to the result type");
  std::vector<unsigned char> args = pack_args(h->spec, ptrs, scalars);
  int64_t head = vector_head(h->spec, ptrs, cfg.v.vec_bytes, h->min_bytes, n);
  CUfunction f = h->mod->function(h->kname("pyc_reduce", cfg.v));
  int resident = resident_ctas(f, cfg.block);
  int64_t tile = (int64_t)cfg.block * (cfg.v.vec_bytes / h->min_bytes) * cfg.v.unroll;
  ChunkPlan cp = plan_chunks(n, head, tile, resident);
  pyc_reduce::Workspace& w = reduce_workspace(h, stream);
  void* params[] = {args.data(), &n, &cp.head, &cp.chunk, &cp.nchunks, &w.part, &w.ticket, &d_out};
  launch_dependent(f, (unsigned)cp.grid, (unsigned)cfg.block, stream, params);
}

}  // namespace pyc

using namespace pyc;

// ------------------------------------------------------------------ map

PYC_API pyc_status pyc_map_create(const char* argspec, const char* stmt, const char* name,
                                  const pyc_opts* opts, pyc_map_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (!argspec) fail(PYC_E_ARG, "argspec is NULL");
    if (!stmt) fail(PYC_E_ARG, "stmt is NULL");
    auto h = std::make_unique<pyc_map>();
    h->opts = opts_or_zero(opts);
    check_opts(h->opts);
    if (h->opts.compensated) fail(PYC_E_ARG, "opts.compensated applies to map-reduce only");
    h->preamble = h->opts.preamble ? h->opts.preamble : "";
    h->opts.preamble = nullptr;
    h->name = name ? name : "map";
    h->spec = parse_argspec(argspec);
    std::string rw = analyze_and_rewrite(h->spec, stmt, false);
    h->tag = kernel_tag(name, 'm', h->spec.canonical + "|" + rw);
    h->gen = generate_map(h->spec, rw, h->preamble, h->tag);
    h->source = h->gen.source;
    finish_handle(*h, false);
    *out = h.release();
  });
}

PYC_API pyc_status pyc_map_launch(pyc_map_t h, int64_t n, void* const* ptrs, const void* scalars,
                                  pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    const CUstream s = reinterpret_cast<CUstream>(stream);
    LaunchCfg cfg = choose_cfg(*h, n, false);
    launch_map(h, cfg, n, ptrs, scalars, s);
    // PYC_AUTOTUNE=1: a first launch at an untuned size bucket tunes it for the next
    autotune_if_due(*h, n, s, false,
                    [&](const LaunchCfg& c, int64_t nt, void* const* p, const void* sc,
                        CUdeviceptr, CUstream ls) { launch_map(h, c, nt, p, sc, ls); },
                    true);
  });
}

PYC_API pyc_status pyc_map_check_bounds(pyc_map_t h) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    check_bounds_record(*h);
  });
}

PYC_API pyc_status pyc_reduce_check_bounds(pyc_reduce_t h) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    std::shared_ptr<pyc::Module> ext;
    {
      std::lock_guard<std::mutex> lk(h->ext_mu);
      ext = h->mod_ext;
    }
    check_bounds_record(*h, ext.get());
  });
}

PYC_API int pyc_map_num_params(pyc_map_t h) { return h ? (int)h->spec.params.size() : -1; }

PYC_API pyc_status pyc_map_param(pyc_map_t h, int idx, pyc_param_info* info) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    fill_param(*h, idx, info);
  });
}

PYC_API int pyc_map_scalar_bytes(pyc_map_t h) { return h ? h->spec.scalar_bytes : -1; }

PYC_API const char* pyc_map_source(pyc_map_t h) { return h ? h->source.c_str() : ""; }

PYC_API void pyc_map_destroy(pyc_map_t h) {
  if (!h) return;
  free_host_pipe(h);
  delete h;
}

// ------------------------------------------------------------------ map-reduce

PYC_API pyc_status pyc_reduce_create(pyc_dtype out_dtype, const char* neutral,
                                     const char* reduce_expr, const char* map_expr,
                                     const char* argspec, const pyc_opts* opts,
                                     pyc_reduce_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (!argspec) fail(PYC_E_ARG, "argspec is NULL");
    auto h = std::make_unique<pyc_reduce>();
    h->opts = opts_or_zero(opts);
    check_opts(h->opts);
    h->preamble = h->opts.preamble ? h->opts.preamble : "";
    h->opts.preamble = nullptr;
    h->name = "reduce";
    h->out_dtype = out_dtype;
    (void)type_info(out_dtype);  // validates the enum
    switch (out_dtype) {
      case PYC_F32: case PYC_F64: case PYC_BF16: case PYC_F16: case PYC_I32: case PYC_I64:
      case PYC_U32: case PYC_U64: case PYC_ARGMIN_F32: case PYC_ARGMAX_F32:
        break;
      default:
        fail(PYC_E_ARG, "unsupported result type for a map-reduce");
    }
    h->spec = parse_argspec(argspec);
    std::string mexpr;
    if (map_expr) {
      mexpr = map_expr;
    } else {
      if (h->spec.num_ptrs != 1) fail(PYC_E_ARG, "map_expr may be NULL only for one array");
      for (auto& p : h->spec.params)
        if (p.is_ptr) mexpr = p.name + "[i]";
    }
    check_expression(mexpr, "map expression");
    std::string mrw = analyze_and_rewrite(h->spec, mexpr, true);
    bool arg = out_dtype == PYC_ARGMIN_F32 || out_dtype == PYC_ARGMAX_F32;
    std::string neu, red;
    if (arg) {
      h->kind = ReduceKind::Arg;
      if (h->opts.compensated) fail(PYC_E_ARG, "compensated needs an F32 result");
      if (neutral) fail(PYC_E_ARG, "ARGMIN/ARGMAX use the built-in neutral element (pass NULL)");
      bool mn = out_dtype == PYC_ARGMIN_F32;
      neu = std::string("pyc_argf32{") + (mn ? "INFINITY" : "-INFINITY") + ", 0, LLONG_MAX}";
      red = reduce_expr ? check_expression(reduce_expr, "reduce expression")
                        : (mn ? "(b.v < a.v || (b.v == a.v && b.i < a.i)) ? b : a"
                              : "(b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a");
    } else {
      if (!neutral) fail(PYC_E_ARG, "neutral is NULL");
      if (!reduce_expr) fail(PYC_E_ARG, "reduce_expr is NULL");
      neu = check_expression(neutral, "neutral expression");
      red = check_expression(reduce_expr, "reduce expression");
      if (h->opts.compensated) {
        if (out_dtype != PYC_F32) fail(PYC_E_ARG, "compensated needs an F32 result");
        std::string r;
        for (char c : red)
          if (c != ' ') r += c;
        if (r != "a+b" && r != "b+a") fail(PYC_E_ARG, "compensated needs the reduce expression a+b");
        h->kind = ReduceKind::Compensated;
      }
    }
    h->tag = kernel_tag(nullptr, 'r',
                        h->spec.canonical + "|" + std::to_string((int)out_dtype) + "|" + neu +
                            "|" + red + "|" + mrw + "|" + std::to_string((int)h->kind));
    int ordered = (arg && !reduce_expr) ? (out_dtype == PYC_ARGMIN_F32 ? 1 : 2) : 0;
    h->gen = generate_reduce(h->spec, out_dtype, h->kind, neu, red, mrw, h->preamble, h->tag,
                             ordered);
    h->source = h->gen.source;
    finish_handle(*h, true);
    h->source_ext = (h->bounds ? bounds_defines() : std::string()) + h->gen.source_ext;
    *out = h.release();
  });
}

pyc::Module& pyc_reduce::ext() {
  std::lock_guard<std::mutex> lk(ext_mu);
  if (!mod_ext) mod_ext = pyc::get_module(source_ext, opts.fmad != 0);
  return *mod_ext;
}

PYC_API pyc_status pyc_reduce_launch(pyc_reduce_t h, int64_t n, void* const* ptrs,
                                     const void* scalars, void* d_out, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    const CUstream s = reinterpret_cast<CUstream>(stream);
    LaunchCfg cfg = choose_cfg(*h, n, true);
    launch_reduce(h, cfg, n, ptrs, scalars, d_out, s);
    // PYC_AUTOTUNE=1: a first launch at an untuned size bucket tunes it for the next
    autotune_if_due(*h, n, s, true,
                    [&](const LaunchCfg& c, int64_t nt, void* const* p, const void* sc,
                        CUdeviceptr out, CUstream ls) {
                      launch_reduce(h, c, nt, p, sc, reinterpret_cast<void*>(out), ls);
                    },
                    true);
  });
}

PYC_API pyc_status pyc_reduce_batched(pyc_reduce_t h, int64_t nseg, const int64_t* seg_offsets,
                                      void* const* ptrs, const void* scalars, void* d_out,
                                      pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    reduce_batched(h, nseg, seg_offsets, ptrs, scalars, d_out, reinterpret_cast<CUstream>(stream));
  });
}

PYC_API pyc_status pyc_reduce_batched_autotune(pyc_reduce_t h, int64_t nseg,
                                               const int64_t* seg_offsets, void* const* ptrs,
                                               const void* scalars, void* d_out,
                                               pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    reduce_batched_autotune(h, nseg, seg_offsets, ptrs, scalars, d_out,
                            reinterpret_cast<CUstream>(stream));
  });
}

PYC_API int pyc_reduce_num_params(pyc_reduce_t h) { return h ? (int)h->spec.params.size() : -1; }

PYC_API pyc_status pyc_reduce_param(pyc_reduce_t h, int idx, pyc_param_info* info) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    fill_param(*h, idx, info);
  });
}

PYC_API int pyc_reduce_scalar_bytes(pyc_reduce_t h) { return h ? h->spec.scalar_bytes : -1; }
PYC_API int pyc_reduce_out_bytes(pyc_reduce_t h) { return h ? h->gen.out_bytes : -1; }
PYC_API const char* pyc_reduce_source(pyc_reduce_t h) { return h ? h->source.c_str() : ""; }

PYC_API void pyc_reduce_destroy(pyc_reduce_t h) {
  if (!h) return;
  try {
    free_plans(h);
    for (auto& kv : h->ws)
      if (kv.second.base) drv().cuMemFree(kv.second.base);
  } catch (...) {
  }
  delete h;
}
