// Parallel prefix scan (Sec. 3.2.6): C ABI and launches (see include/pyc.h).
//
// Two launches on the caller's stream, with no waiting between CTAs:
//  pass 1 folds every chunk of the input expression (the map-reduce core) and
//         the last CTA to finish turns the chunk totals into exclusive carries;
//  pass 2 scans every chunk from its carry in index order (block scans of one
//         row of vector groups at a time) and runs the output statement with
//         `item` (inclusive prefix) and `prev_item` (exclusive prefix).
// Both passes use one chunk plan, a fixed function of (n, tuning).
#include <algorithm>
#include <map>
#include <mutex>

#include "cudrv.h"
#include "handles.h"

struct pyc_scan : pyc::HandleBase {
  pyc_dtype dtype = PYC_F32;
  pyc::ScanGen gen;
  struct Workspace {
    CUdeviceptr base = 0, part = 0, ticket = 0;
  };
  std::mutex ws_mu;
  std::map<std::pair<CUcontext, CUstream>, Workspace> ws;
};

namespace pyc {

namespace {

pyc_scan::Workspace& scan_workspace(pyc_scan* h, CUstream stream) {
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(h->ws_mu);
  auto key = std::make_pair(ctx, stream);
  auto it = h->ws.find(key);
  if (it != h->ws.end()) return it->second;
  pyc_scan::Workspace w;
  size_t part_bytes = (size_t)kMaxChunks * h->gen.acc_bytes;
  PYC_CU(drv().cuMemAlloc(&w.base, part_bytes + 256));
  w.part = w.base;
  w.ticket = w.base + part_bytes;
  PYC_CU(drv().cuMemsetD8Async(w.ticket, 0, 256, stream));
  return h->ws.emplace(key, w).first->second;
}

void launch_scan(pyc_scan* h, const LaunchCfg& cfg, int64_t n, void* const* ptrs,
                 const void* scalars, CUstream stream) {
  if (cfg.block < 32 || cfg.block > 512 || cfg.block % 32)
    fail(PYC_E_ARG, "block must be a multiple of 32 in [32, 512]");
  if (n < 0) fail(PYC_E_ARG, "n must be >= 0");
  std::vector<unsigned char> args = pack_args(h->spec, ptrs, scalars);
  int64_t head = vector_head(h->spec, ptrs, cfg.v.vec_bytes, h->min_bytes, n);
  if (n == 0) return;
  CUfunction f1 = h->mod->function(h->kname("pyc_scan1", cfg.v));
  CUfunction f2 = h->mod->function(h->kname("pyc_scan2", cfg.v));
  int r1 = resident_ctas(f1, cfg.block), r2 = resident_ctas(f2, cfg.block);
  int64_t tile = (int64_t)cfg.block * (cfg.v.vec_bytes / h->min_bytes) * cfg.v.unroll;
  ChunkPlan cp = plan_chunks(n, head, tile, std::min(r1, r2));
  pyc_scan::Workspace& w = scan_workspace(h, stream);
  void* p1[] = {args.data(), &n, &cp.head, &cp.chunk, &cp.nchunks, &w.part, &w.ticket};
  PYC_CU(drv().cuLaunchKernel(f1, (unsigned)cp.grid, 1, 1, (unsigned)cfg.block, 1, 1, 0, stream,
                              p1, nullptr));
  unsigned grid2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(r2, cp.nchunks));
  void* p2[] = {args.data(), &n, &cp.head, &cp.chunk, &cp.nchunks, &w.part};
  PYC_CU(drv().cuLaunchKernel(f2, grid2, 1, 1, (unsigned)cfg.block, 1, 1, 0, stream, p2, nullptr));
}

}  // namespace

}  // namespace pyc

using namespace pyc;

PYC_API pyc_status pyc_scan_create(pyc_dtype dtype, const char* neutral, const char* scan_expr,
                                   const char* input_expr, const char* output_stmt,
                                   const char* argspec, const pyc_opts* opts, pyc_scan_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (!argspec || !neutral || !scan_expr || !input_expr || !output_stmt)
      fail(PYC_E_ARG, "neutral, scan_expr, input_expr, output_stmt and argspec are required");
    switch (dtype) {
      case PYC_F32: case PYC_F64: case PYC_I32: case PYC_I64: case PYC_U32: case PYC_U64:
        break;
      default:
        fail(PYC_E_ARG, "scan values must be F32, F64, I32, I64, U32 or U64");
    }
    auto h = std::make_unique<pyc_scan>();
    if (opts) h->opts = *opts;
    if (h->opts.compensated) fail(PYC_E_ARG, "opts.compensated applies to map-reduce only");
    if (h->opts.block && (h->opts.block < 32 || h->opts.block > 512 || h->opts.block % 32))
      fail(PYC_E_ARG, "opts.block must be 0 or a multiple of 32 in [32, 512]");
    if (h->opts.vec_bytes && h->opts.vec_bytes != 16 && h->opts.vec_bytes != 32)
      fail(PYC_E_ARG, "opts.vec_bytes must be 0, 16 or 32");
    if (h->opts.items_per_thread && h->opts.items_per_thread != 1 &&
        h->opts.items_per_thread != 2 && h->opts.items_per_thread != 4)
      fail(PYC_E_ARG, "opts.items_per_thread must be 0, 1, 2 or 4");
    h->preamble = h->opts.preamble ? h->opts.preamble : "";
    h->opts.preamble = nullptr;
    h->dtype = dtype;
    h->name = "scan";
    h->spec = parse_argspec(argspec);
    for (auto& p : h->spec.params)
      if (p.name == "item" || p.name == "prev_item")
        fail(PYC_E_PARSE, "'item' and 'prev_item' are reserved in a scan");
    check_expression(input_expr, "input expression");
    std::string neu = check_expression(neutral, "neutral expression");
    std::string red = check_expression(scan_expr, "scan expression");
    // analyse both pieces of code first, then rewrite each with the final flags
    analyze_code(h->spec, output_stmt, false);
    analyze_code(h->spec, input_expr, true);
    std::string in_rw = rewrite_lifted(h->spec, input_expr);
    std::string out_rw = rewrite_lifted(h->spec, output_stmt);
    h->tag = kernel_tag(nullptr, 's', h->spec.canonical + "|" + std::to_string((int)dtype) + "|" +
                                          neu + "|" + red + "|" + in_rw + "|" + out_rw);
    h->gen = generate_scan(h->spec, dtype, neu, red, in_rw, out_rw, h->preamble, h->tag);
    h->source = h->gen.source;
    h->min_bytes = lifted_min_bytes(h->spec);
    h->mod = get_module(h->source, h->opts.fmad != 0);
    h->tune_key = digest(h->source + (h->opts.fmad ? "|fmad" : ""));
    for (auto& p : h->spec.params) h->param_names.push_back(p.name);
    tune_cache_load(*h, true);
    *out = h.release();
  });
}

PYC_API pyc_status pyc_scan_launch(pyc_scan_t h, int64_t n, void* const* ptrs,
                                   const void* scalars, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    LaunchCfg cfg = choose_cfg(*h, n, true);
    if (cfg.v.vec_bytes != 16 && cfg.v.vec_bytes != 32) fail(PYC_E_ARG, "bad vec_bytes");
    launch_scan(h, cfg, n, ptrs, scalars, reinterpret_cast<CUstream>(stream));
  });
}

PYC_API int pyc_scan_num_params(pyc_scan_t h) { return h ? (int)h->spec.params.size() : -1; }

PYC_API pyc_status pyc_scan_param(pyc_scan_t h, int idx, pyc_param_info* info) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    if (!info) fail(PYC_E_ARG, "info is NULL");
    if (idx < 0 || idx >= (int)h->spec.params.size()) fail(PYC_E_ARG, "parameter index out of range");
    const Param& p = h->spec.params[idx];
    info->name = h->param_names[idx].c_str();
    info->is_pointer = p.is_ptr;
    info->dtype = p.dtype;
    info->elem_bytes = type_info(p.dtype).bytes;
    info->scalar_offset = p.scalar_offset;
    info->pointer_slot = p.ptr_slot;
    info->read = p.read;
    info->written = p.written;
    info->lifted = p.lifted;
  });
}

PYC_API int pyc_scan_scalar_bytes(pyc_scan_t h) { return h ? h->spec.scalar_bytes : -1; }
PYC_API const char* pyc_scan_source(pyc_scan_t h) { return h ? h->source.c_str() : ""; }

PYC_API pyc_status pyc_scan_autotune(pyc_scan_t h, int64_t n, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    CUstream s = reinterpret_cast<CUstream>(stream);
    autotune_generic(*h, n, s, true,
                     [&](const LaunchCfg& c, int64_t nt, void* const* p, const void* sc,
                         CUdeviceptr) { launch_scan(h, c, nt, p, sc, s); });
  });
}

PYC_API pyc_status pyc_scan_config(pyc_scan_t h, int64_t n, int* vec_bytes, int* unroll,
                                   int* block) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    LaunchCfg c = choose_cfg(*h, n, true);
    if (vec_bytes) *vec_bytes = c.v.vec_bytes;
    if (unroll) *unroll = c.v.unroll;
    if (block) *block = c.block;
  });
}

PYC_API void pyc_scan_destroy(pyc_scan_t h) {
  if (!h) return;
  try {
    for (auto& kv : h->ws)
      if (kv.second.base) drv().cuMemFree(kv.second.base);
  } catch (...) {
  }
  delete h;
}
