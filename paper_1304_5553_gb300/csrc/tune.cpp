// Automated tuning (Sec. 3.3.1): every module keeps all variants (vector
// width x unroll) side by side; the tuner times each variant at each block
// size on scratch buffers for the size bucket of n, keeps the fastest for the
// handle, and appends it to a JSON-lines cache so later processes start tuned.
// Keys: (digest of the generated source, map / reduce, size bucket).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

namespace {

std::string tune_path() {
  std::string d = cache_dir();
  return d.empty() ? "" : d + "/tune.jsonl";
}

std::mutex g_file_mu;

// Minimal field extraction from one of our own JSON lines.
bool field(const std::string& line, const char* name, std::string* out) {
  std::string pat = std::string("\"") + name + "\":";
  size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  p += pat.size();
  while (p < line.size() && (line[p] == ' ' || line[p] == '\t')) ++p;  // "name": value
  if (p < line.size() && line[p] == '"') {
    size_t e = line.find('"', p + 1);
    if (e == std::string::npos) return false;
    *out = line.substr(p + 1, e - p - 1);
  } else {
    size_t e = line.find_first_of(",}", p);
    *out = line.substr(p, e - p);
  }
  return true;
}

struct Scratch {
  std::vector<CUdeviceptr> bufs;
  ~Scratch() { release(); }
  void release() {
    for (auto b : bufs)
      if (b) drv().cuMemFree(b);
    bufs.clear();
  }
  CUdeviceptr alloc(size_t bytes) {
    CUdeviceptr p;
    PYC_CU(drv().cuMemAlloc(&p, bytes));
    bufs.push_back(p);
    return p;
  }
};

template <class Launch>
double time_us(Launch&& launch, CUstream s, int reps) {
  const Driver& d = drv();
  CUevent e0, e1;
  PYC_CU(d.cuEventCreate(&e0, CU_EVENT_DEFAULT));
  PYC_CU(d.cuEventCreate(&e1, CU_EVENT_DEFAULT));
  double best = 1e30;
  try {
    launch();
    launch();
    for (int r = 0; r < reps; ++r) {
      PYC_CU(d.cuEventRecord(e0, s));
      launch();
      PYC_CU(d.cuEventRecord(e1, s));
      PYC_CU(d.cuEventSynchronize(e1));
      float ms = 0;
      PYC_CU(d.cuEventElapsedTime(&ms, e0, e1));
      best = std::min(best, (double)ms * 1000.0);
    }
  } catch (...) {
    d.cuEventDestroy(e0);
    d.cuEventDestroy(e1);
    throw;
  }
  d.cuEventDestroy(e0);
  d.cuEventDestroy(e1);
  return best;
}

// Device time of one launch, from replays of a CUDA graph of `reps` launches
// captured on the context's private stream (best of 3 replays).  The first
// launch runs outside the capture, so per-stream set-up (a reduction's
// workspace) is done before it.
template <class Launch>
double time_graph_us(Launch&& launch, int reps) {
  const Driver& d = drv();
  CUstream cs = capture_stream();
  launch(cs);
  PYC_CU(d.cuStreamSynchronize(cs));
  struct Res {
    CUgraph g = nullptr;
    CUgraphExec ge = nullptr;
    CUevent e0 = nullptr, e1 = nullptr;
    ~Res() {
      const Driver& d = drv();
      if (ge) d.cuGraphExecDestroy(ge);
      if (g) d.cuGraphDestroy(g);
      if (e0) d.cuEventDestroy(e0);
      if (e1) d.cuEventDestroy(e1);
    }
  } r;
  PYC_CU(d.cuStreamBeginCapture(cs, CU_STREAM_CAPTURE_MODE_THREAD_LOCAL));
  try {
    for (int k = 0; k < reps; ++k) launch(cs);
  } catch (...) {
    CUgraph t = nullptr;
    d.cuStreamEndCapture(cs, &t);
    if (t) d.cuGraphDestroy(t);
    throw;
  }
  PYC_CU(d.cuStreamEndCapture(cs, &r.g));
  PYC_CU(d.cuGraphInstantiateWithFlags(&r.ge, r.g, 0));
  PYC_CU(d.cuEventCreate(&r.e0, CU_EVENT_DEFAULT));
  PYC_CU(d.cuEventCreate(&r.e1, CU_EVENT_DEFAULT));
  PYC_CU(d.cuGraphLaunch(r.ge, cs));
  double best = 1e30;
  for (int k = 0; k < 3; ++k) {
    PYC_CU(d.cuEventRecord(r.e0, cs));
    PYC_CU(d.cuGraphLaunch(r.ge, cs));
    PYC_CU(d.cuEventRecord(r.e1, cs));
    PYC_CU(d.cuEventSynchronize(r.e1));
    float ms = 0;
    PYC_CU(d.cuEventElapsedTime(&ms, r.e0, r.e1));
    best = std::min(best, (double)ms * 1000.0 / reps);
  }
  return best;
}

template <class H, class Launch>
void autotune(H* h, int64_t n, CUstream stream, bool reduce, Launch&& launch_one,
              bool graph_timing) {
  if (n <= 0) fail(PYC_E_ARG, "autotune needs n > 0");
  // Representative size: n itself up to 2^28 elements (a variant's rank at a
  // quarter of the size can differ from its rank at the size that runs), with
  // the scratch arrays held to 6 GiB together, halved while the device cannot
  // hold them (down to 2^20 elements).
  const int64_t kMinTune = (int64_t)1 << 20;
  const int64_t kScratchCap = (int64_t)6 << 30;
  int64_t per_elem = 0;
  for (auto& p : h->spec.params)
    if (p.is_ptr) per_elem += type_info(p.dtype).bytes;
  int64_t nt = std::min<int64_t>(n, (int64_t)1 << 28);
  while (nt > kMinTune && per_elem * nt > kScratchCap) nt = (nt + 1) / 2;
  Scratch sc;
  std::vector<void*> ptrs(h->spec.num_ptrs ? h->spec.num_ptrs : 1, nullptr);
  for (;;) {
    try {
      for (auto& p : h->spec.params)
        if (p.is_ptr) {
          size_t bytes = (size_t)nt * type_info(p.dtype).bytes + 256;
          CUdeviceptr b = sc.alloc(bytes);
          PYC_CU(drv().cuMemsetD8Async(b, 0, bytes, stream));
          ptrs[p.ptr_slot] = reinterpret_cast<void*>(b);
        }
      break;
    } catch (const Error& e) {
      if (e.status != PYC_E_NOMEM || nt <= kMinTune) throw;
      sc.release();
      nt = (nt + 1) / 2;
    }
  }
  std::vector<unsigned char> scal(h->spec.scalar_bytes + 8, 0);
  CUdeviceptr out = sc.alloc(256);
  LaunchCfg best;
  double best_us = 1e30;
  const int blocks[] = {128, 256, 512};
  for (const Variant& v : all_variants()) {
    if (h->opts.vec_bytes && v.vec_bytes != h->opts.vec_bytes) continue;
    if (h->opts.items_per_thread && v.unroll != h->opts.items_per_thread) continue;
    for (int b : blocks) {
      if (h->opts.block && b != h->opts.block) continue;
      LaunchCfg c;
      c.v = v;
      c.block = b;
      double us =
          time_us([&] { launch_one(c, nt, ptrs.data(), scal.data(), out, stream); }, stream, 5);
      // short kernels: a single launch's sample includes the host's launch latency
      if (graph_timing && us < 40.0)
        us = time_graph_us(
            [&](CUstream cs) { launch_one(c, nt, ptrs.data(), scal.data(), out, cs); }, 20);
      if (std::getenv("PYC_TUNE_LOG"))
        std::fprintf(stderr, "pyc tune %s %s n=%lld vec=%d unroll=%d block=%d %.2f us\n",
                     reduce ? "reduce" : "map", h->tag.c_str(), (long long)nt, v.vec_bytes,
                     v.unroll, b, us);
      if (us < best_us) {
        best_us = us;
        best = c;
      }
    }
  }
  int bucket = size_bucket(n);
  {
    std::lock_guard<std::mutex> lk(h->tune.mu);
    h->tune.by_bucket[bucket] = best;
  }
  log_event("tuned %s %s for size bucket %d (n = %lld): vec%d_u%d_b%d, %.2f us", reduce ? "reduce" : "map",
            h->tag.c_str(), bucket, (long long)n, best.v.vec_bytes, best.v.unroll, best.block,
            best_us);
  tune_cache_store(*h, reduce, bucket, best, best_us);
}

}  // namespace

void autotune_generic(HandleBase& h, int64_t n, CUstream stream, bool reduce,
                      const TuneLaunch& launch_one, bool graph_timing) {
  autotune(&h, n, stream, reduce, launch_one, graph_timing);
}

void autotune_if_due(HandleBase& h, int64_t n, CUstream stream, bool reduce,
                     const TuneLaunch& launch_one, bool graph_timing) {
  const char* e = std::getenv("PYC_AUTOTUNE");
  if (!e || e[0] != '1' || n <= 0) return;
  if (h.opts.block && h.opts.vec_bytes && h.opts.items_per_thread) return;  // nothing to choose
  auto tuned = [&] {
    std::lock_guard<std::mutex> lk(h.tune.mu);
    return h.tune.by_bucket.count(size_bucket(n)) > 0;
  };
  if (tuned()) return;
  // tuning allocates and synchronises: never inside a stream capture
  CUstreamCaptureStatus cap = CU_STREAM_CAPTURE_STATUS_NONE;
  if (stream) PYC_CU(drv().cuStreamIsCapturing(stream, &cap));
  if (cap != CU_STREAM_CAPTURE_STATUS_NONE) return;
  std::unique_lock<std::mutex> busy(h.tune.tuning, std::try_to_lock);
  if (!busy.owns_lock() || tuned()) return;  // another thread tunes (or did): launch as is
  autotune(&h, n, stream, reduce, launch_one, graph_timing);
}

void tune_cache_load(HandleBase& h, bool reduce) {
  std::string path = tune_path();
  if (path.empty()) return;
  std::lock_guard<std::mutex> flk(g_file_mu);
  std::ifstream f(path);
  if (!f) return;
  std::string line;
  const char* kind = reduce ? "reduce" : "map";
  std::lock_guard<std::mutex> lk(h.tune.mu);
  while (std::getline(f, line)) {
    std::string key, k, b, vb, u, blk;
    if (!field(line, "key", &key) || key != h.tune_key) continue;
    if (!field(line, "kind", &k) || k != kind) continue;
    if (!field(line, "bucket", &b) || !field(line, "vec_bytes", &vb) ||
        !field(line, "unroll", &u) || !field(line, "block", &blk))
      continue;
    LaunchCfg c;
    c.v.vec_bytes = std::atoi(vb.c_str());
    c.v.unroll = std::atoi(u.c_str());
    c.block = std::atoi(blk.c_str());
    std::string ln;
    c.lean = field(line, "lean", &ln) && ln == "1" && c.v.vec_bytes == 16 ? 1 : 0;
    bool ok = (c.v.vec_bytes == 16 || c.v.vec_bytes == 32) &&
              (c.v.unroll == 1 || c.v.unroll == 2 || c.v.unroll == 4) && c.block >= 32 &&
              c.block <= 512 && c.block % 32 == 0;
    if (ok) h.tune.by_bucket[std::atoi(b.c_str())] = c;  // later lines win
  }
}

void tune_cache_store(const HandleBase& h, bool reduce, int bucket, const LaunchCfg& c,
                      double us) {
  std::string path = tune_path();
  if (path.empty()) return;
  std::string dev;
  try {
    dev = current_device_props().name;
  } catch (...) {
  }
  for (auto& ch : dev)
    if (ch == '"' || ch == '\\') ch = ' ';
  std::ostringstream o;
  o << "{\"key\":\"" << h.tune_key << "\",\"kind\":\"" << (reduce ? "reduce" : "map")
    << "\",\"bucket\":" << bucket << ",\"vec_bytes\":" << c.v.vec_bytes
    << ",\"unroll\":" << c.v.unroll << ",\"block\":" << c.block << ",\"lean\":" << c.lean
    << ",\"us\":" << us
    << ",\"device\":\"" << dev << "\"}\n";
  std::lock_guard<std::mutex> flk(g_file_mu);
  std::ofstream f(path, std::ios::app);
  if (f) f << o.str();
}

}  // namespace pyc

using namespace pyc;

PYC_API pyc_status pyc_map_config(pyc_map_t h, int64_t n, int* vec_bytes, int* unroll,
                                  int* block) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    LaunchCfg c = choose_cfg(*h, n, false);
    if (vec_bytes) *vec_bytes = c.v.vec_bytes;
    if (unroll) *unroll = c.v.unroll;
    if (block) *block = c.block;
  });
}

PYC_API pyc_status pyc_reduce_config(pyc_reduce_t h, int64_t n, int* vec_bytes, int* unroll,
                                     int* block) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    LaunchCfg c = choose_cfg(*h, n, true);
    if (vec_bytes) *vec_bytes = c.v.vec_bytes;
    if (unroll) *unroll = c.v.unroll;
    if (block) *block = c.block;
  });
}

PYC_API pyc_status pyc_reduce_batched_config(pyc_reduce_t h, int* vec_bytes, int* unroll,
                                             int* block, int* reg_cap) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    LaunchCfg c = batched_cfg(*h, true);
    if (vec_bytes) *vec_bytes = c.v.vec_bytes;
    if (unroll) *unroll = c.v.unroll;
    if (block) *block = c.block;
    if (reg_cap) *reg_cap = c.lean ? kLeanRegs : 0;
  });
}

PYC_API pyc_status pyc_map_autotune(pyc_map_t h, int64_t n, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    CUstream s = reinterpret_cast<CUstream>(stream);
    autotune(h, n, s, false,
             [&](const LaunchCfg& c, int64_t nt, void* const* p, const void* sc, CUdeviceptr,
                 CUstream ls) { launch_map(h, c, nt, p, sc, ls); },
             true);
  });
}

PYC_API pyc_status pyc_reduce_autotune(pyc_reduce_t h, int64_t n, pyc_stream_t stream) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    CUstream s = reinterpret_cast<CUstream>(stream);
    autotune(h, n, s, true,
             [&](const LaunchCfg& c, int64_t nt, void* const* p, const void* sc, CUdeviceptr out,
                 CUstream ls) { launch_reduce(h, c, nt, p, sc, reinterpret_cast<void*>(out), ls); },
             true);
  });
}
