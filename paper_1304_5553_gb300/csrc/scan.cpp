// Parallel prefix scan (Sec. 3.2.6): C ABI and launches (see include/pyc.h).
//
// One launch on the caller's stream.  Persistent CTAs take tiles in index order
// from a counter.  The compute warps fold each tile (sweep 1) and hand its
// aggregate to the CTA's look-back warp, which publishes it, looks back over
// the descriptors of the tiles before it for the exclusive prefix and
// publishes the inclusive prefix; meanwhile the compute warps scan the
// previous tile (sweep 2, re-reading it from L2) and write its output.  HBM
// sees the input read once and the output written once.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "cudrv.h"
#include "handles.h"

struct pyc_scan : pyc::HandleBase {
  pyc_dtype dtype = PYC_F32;
  pyc::ScanGen gen;
  struct Workspace {
    CUdeviceptr base = 0;
    int64_t cap = 0;     // tile descriptors
    uint32_t epoch = 0;  // of the last launch
  };
  std::mutex ws_mu;
  std::map<std::pair<CUcontext, CUstream>, Workspace> ws;
};

namespace pyc {

namespace {

// Mirrors pyc_scan_params in the generated source.
struct ScanParams {
  CUdeviceptr flag, agg, inc, ctl;
  int64_t n, head, nfull, ntiles, spin_limit, stall_tile;
  uint32_t epoch, groups, tail_groups, pad;
};
static_assert(sizeof(ScanParams) == 96, "scan params layout");

constexpr int64_t kCtlBytes = 256;               // ctl[0..3] at the start of the workspace
constexpr uint32_t kEpochLimit = 1u << 30;       // flags hold epoch << 2 | state
constexpr int64_t kDefaultSpinLimit = 1 << 20;   // about a second of polling

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

// Row groups per warp in a vector tile.  A tile is read twice (fold, then
// scan), the second time from L2, and a CTA holds two tiles' input and one
// tile's output at a time, so one tile's input is kept to 5/32 of L2 over the
// resident CTAs (of 4/32, 5/32 and 6/32, the fastest for the int32 -> int64
// scan and as fast as 6/32 for the binary32 scans); within that, tiles are made
// as large as possible (fewer look-backs) while leaving at least four tiles per
// CTA.
int scan_groups(int64_t n, int64_t base, int resident, int elem_bytes, int64_t l2_bytes) {
  int64_t want = n / (4 * (int64_t)resident);
  if (elem_bytes > 0) want = std::min<int64_t>(want, l2_bytes * 5 / 32 / resident / elem_bytes);
  return (int)std::max<int64_t>(1, std::min<int64_t>(64, want / base));
}

// Workspace of (context, stream) with room for `ntiles` descriptors, and the
// parameters of the next launch (a fresh epoch).
ScanParams scan_workspace(pyc_scan* h, CUstream stream, int64_t ntiles) {
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(h->ws_mu);
  pyc_scan::Workspace& w = h->ws[std::make_pair(ctx, stream)];
  const int64_t acc = h->gen.acc_bytes;
  // descriptors (4-byte flags, or 8-byte packed words) are read in aligned
  // groups of four: cap is a multiple of 64
  auto flag_bytes = [](int64_t cap) { return align256(cap * 8); };
  if (ntiles > w.cap) {
    if (w.base) {
      // a launch in flight on this stream may still use the old descriptors
      PYC_CU(drv().cuStreamSynchronize(stream));
      drv().cuMemFree(w.base);
      w.base = 0;
      w.cap = 0;
    }
    int64_t cap = std::max<int64_t>(4096, (ntiles + 63) / 64 * 64);
    int64_t bytes = kCtlBytes + flag_bytes(cap) + 2 * align256(cap * acc);
    PYC_CU(drv().cuMemAlloc(&w.base, (size_t)bytes));
    const CUresult r = drv().cuMemsetD8Async(w.base, 0, (size_t)(kCtlBytes + flag_bytes(cap)), stream);
    if (r != CUDA_SUCCESS) {
      drv().cuMemFree(w.base);
      w.base = 0;
      ::pyc::check(r, "cuMemsetD8Async");
    }
    w.cap = cap;
    w.epoch = 0;
  }
  if (++w.epoch >= kEpochLimit) {
    // flags and ctl[3] may hold old epochs that are about to be reused
    PYC_CU(drv().cuMemsetD8Async(w.base + kCtlBytes, 0, (size_t)flag_bytes(w.cap), stream));
    PYC_CU(drv().cuMemsetD8Async(w.base + 24, 0, 8, stream));
    w.epoch = 1;
  }
  ScanParams p{};
  p.ctl = w.base;
  p.flag = w.base + kCtlBytes;
  p.agg = p.flag + flag_bytes(w.cap);
  p.inc = p.agg + align256(w.cap * acc);
  p.epoch = w.epoch;
  return p;
}

void launch_scan(pyc_scan* h, const LaunchCfg& cfg, int64_t n, void* const* ptrs,
                 const void* scalars, CUstream stream, int64_t stall_tile = -1,
                 int64_t spin_limit = kDefaultSpinLimit) {
  if (cfg.block < 32 || cfg.block > 512 || cfg.block % 32)
    fail(PYC_E_ARG, "block must be a multiple of 32 in [32, 512]");
  if (n < 0) fail(PYC_E_ARG, "n must be >= 0");
  if (spin_limit < 1) fail(PYC_E_ARG, "spin_limit must be >= 1");
  std::vector<unsigned char> args = pack_args(h->spec, ptrs, scalars);
  int64_t head = vector_head(h->spec, ptrs, cfg.v.vec_bytes, h->min_bytes, n);
  check_overlap(h->spec, ptrs, n);
  if (n == 0) return;
  CUfunction f = h->mod->function(h->kname("pyc_scan", cfg.v));
  // cfg.block compute threads and one look-back warp
  const int threads = cfg.block + 32;
  const int resident = resident_ctas(f, threads);
  // one row group per compute warp: 32 lanes x one vector of E elements x unroll rows
  const int64_t base = (int64_t)cfg.block * (cfg.v.vec_bytes / h->min_bytes) * cfg.v.unroll;
  const int groups = scan_groups(n, base, resident, h->gen.stage_elem_bytes,
                                 current_device_props().l2_bytes);
  const int64_t tile = base * groups;
  int64_t nfull = 0, tail_groups = 0, ntiles;
  if (head < 0) {
    ntiles = (n + tile - 1) / tile;
  } else {
    nfull = (n - head) / tile;
    const int64_t rest = (n - head) - nfull * tile;
    tail_groups = rest / base;
    ntiles = (head > 0 ? 1 : 0) + nfull + (tail_groups > 0 ? 1 : 0) +
             (rest - tail_groups * base > 0 ? 1 : 0);
  }
  ScanParams S = scan_workspace(h, stream, ntiles);
  S.n = n;
  S.head = head;
  S.nfull = nfull;
  S.ntiles = ntiles;
  S.spin_limit = spin_limit;
  S.stall_tile = stall_tile;
  S.groups = (uint32_t)groups;
  S.tail_groups = (uint32_t)tail_groups;
  unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, ntiles));
  void* params[] = {args.data(), &S};
  PYC_CU(drv().cuLaunchKernel(f, grid, 1, 1, (unsigned)threads, 1, 1, 0, stream, params,
                              nullptr));
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
    // opts.debug_bounds, PYC_DEBUG_BOUNDS=1 or PYC_CHECK_BOUNDS=1: the scan's own
    // bounds-checked build (debugging aid)
    bool checked = bounds_requested(h->opts);
    if (const char* c = std::getenv("PYC_CHECK_BOUNDS"))
      if (c[0] == '1') checked = true;
    if (checked) {
      std::string d = "#define PYC_CHECK 1\n";
      // test hook: narrow the array ranges, so that the checks can be seen to fire
      if (const char* k = std::getenv("PYC_DEBUG_BOUNDS_SHRINK")) {
        long long v = std::atoll(k);
        if (v > 0) d += "#define PYC_SCAN_SHRINK " + std::to_string(v) + "LL\n";
      }
      h->preamble = d + h->preamble;
    }
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
    const CUstream s = reinterpret_cast<CUstream>(stream);
    LaunchCfg cfg = choose_cfg(*h, n, true);
    if (cfg.v.vec_bytes != 16 && cfg.v.vec_bytes != 32) fail(PYC_E_ARG, "bad vec_bytes");
    launch_scan(h, cfg, n, ptrs, scalars, s);
    // PYC_AUTOTUNE=1: a first launch at an untuned size bucket tunes it for the next
    autotune_if_due(*h, n, s, true,
                    [&](const LaunchCfg& c, int64_t nt, void* const* p, const void* sc,
                        CUdeviceptr, CUstream) { launch_scan(h, c, nt, p, sc, s); });
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
                         CUdeviceptr, CUstream) { launch_scan(h, c, nt, p, sc, s); });
  });
}

PYC_API pyc_status pyc_scan_launch_test(pyc_scan_t h, int64_t n, void* const* ptrs,
                                        const void* scalars, pyc_stream_t stream,
                                        int64_t stall_tile, int64_t spin_limit) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    LaunchCfg cfg = choose_cfg(*h, n, true);
    launch_scan(h, cfg, n, ptrs, scalars, reinterpret_cast<CUstream>(stream), stall_tile,
                spin_limit);
  });
}

PYC_API pyc_status pyc_scan_sync(pyc_scan_t h, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    CUstream s = reinterpret_cast<CUstream>(stream);
    CUcontext ctx = ensure_context();
    CUdeviceptr base = 0;
    {
      std::lock_guard<std::mutex> lk(h->ws_mu);
      auto it = h->ws.find(std::make_pair(ctx, s));
      if (it != h->ws.end()) base = it->second.base;
    }
    PYC_CU(drv().cuStreamSynchronize(s));
    if (!base) return;
    unsigned long long ctl[8] = {};
    PYC_CU(drv().cuMemcpyDtoH(ctl, base, sizeof(ctl)));
    if (ctl[4]) {
      const unsigned long long zero[4] = {0, 0, 0, 0};
      PYC_CU(drv().cuMemcpyHtoD(base + 32, zero, sizeof(zero)));
      fail(PYC_E_INTERNAL, "scan bounds check " + std::to_string(ctl[4]) + " failed: index " +
                               std::to_string((long long)ctl[5]) + ", tile " +
                               std::to_string((long long)ctl[6]) + ", block " +
                               std::to_string(ctl[7] >> 16) + ", thread " +
                               std::to_string(ctl[7] & 0xffff));
    }
    const unsigned long long err = ctl[2];
    if (err) {
      // a CTA that gave up left without its share of the tile-counter reset
      const unsigned long long zero[4] = {0, 0, 0, 0};
      PYC_CU(drv().cuMemcpyHtoD(base, zero, sizeof(zero)));
      fail(PYC_E_TIMEOUT, "a scan launch on this stream gave up waiting for a tile descriptor; "
                          "its output is not valid");
    }
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
