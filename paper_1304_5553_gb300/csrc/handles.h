// Handle objects behind the opaque pyc_map_t / pyc_reduce_t pointers, and the
// launch-configuration helpers shared by launches, the batched reducer, the
// tuner and the server.
#pragma once

#include <cuda.h>

#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "codegen.h"
#include "common.h"
#include "kcache.h"
#include "spec.h"

namespace pyc {

// One tuned (or chosen) launch configuration.
struct LaunchCfg {
  Variant v{16, 4};
  int block = 256;
  int lean = 0;  // batched reductions: 1 = the register-lean build (16-byte variants)
};

// Size buckets for tuning: bucket b holds n with bit length in [2b, 2b+1].
int size_bucket(int64_t n);

// Per-handle tuning results by size bucket.
struct TuneTable {
  std::mutex mu;
  std::map<int, LaunchCfg> by_bucket;
  std::mutex tuning;  // held while a launch tunes the handle (PYC_AUTOTUNE)
};

struct BatchPlan;  // batched reducer plan (batched.cpp)
struct HostPipe;   // staging for host-array maps (hostpipe.cpp)

struct HandleBase {
  ArgSpec spec;
  std::string name;
  pyc_opts opts{};
  std::string preamble;
  std::string source;
  std::shared_ptr<Module> mod;
  int min_bytes = 4;
  TuneTable tune;
  std::string tune_key;  // digest of the source: key of the persistent tuning cache
  std::vector<std::string> param_names;  // stable storage for pyc_param_info.name
  std::string tag;                       // kernel-name tag of this spec
  bool bounds = false;                   // bounds-checked build (opts.debug_bounds)
  // Kernel function name, e.g. kname("pyc_map", v) = "pyc_map_<tag>_v16_u4".
  std::string kname(const char* kind, const Variant& v) const {
    return std::string(kind) + "_" + tag + "_" + variant_suffix(v);
  }
  // Batched reduction kernel of a configuration (the lean build's suffix included).
  std::string rbatch_name(const LaunchCfg& c) const {
    return kname("pyc_rbatch", c.v) + (c.lean ? "_r" + std::to_string(kLeanRegs) : "");
  }
};

// Identifier-safe kernel tag: the sanitised name, or "<prefix><8 hex digits>"
// of the spec text when no name is given.
std::string kernel_tag(const char* name, char prefix, const std::string& spec_text);

}  // namespace pyc

struct pyc_map : pyc::HandleBase {
  pyc::MapGen gen;
  std::mutex pipe_mu;
  pyc::HostPipe* pipe = nullptr;  // created by the first pyc_map_launch_host
};

struct pyc_reduce : pyc::HandleBase {
  pyc_reduce();
  ~pyc_reduce();  // defined where BatchPlan is complete
  pyc_dtype out_dtype = PYC_F32;
  pyc::ReduceKind kind = pyc::ReduceKind::Plain;
  pyc::ReduceGen gen;
  // workspace (partials + ticket) per (context, stream)
  struct Workspace {
    CUdeviceptr base = 0;
    CUdeviceptr part = 0;
    CUdeviceptr ticket = 0;
  };
  std::mutex ws_mu;
  std::map<std::pair<CUcontext, CUstream>, Workspace> ws;
  std::mutex plan_mu;
  std::vector<std::unique_ptr<pyc::BatchPlan>> plans;  // most recent last
  // The extra module (sharded reduction, record combine, register-lean batched
  // kernels), compiled on first use: most handles never need it.
  std::string source_ext;
  std::mutex ext_mu;
  std::shared_ptr<pyc::Module> mod_ext;
  pyc::Module& ext();
  // Module holding the batched kernel of a configuration.
  pyc::Module& batched_module(const pyc::LaunchCfg& c) { return c.lean ? ext() : *mod; }
  // Set-up of pyc_reduce_launch_static for the context it was last called in:
  // kernel handles of every variant and resident CTAs per (variant, block / 32).
  std::mutex static_mu;
  CUcontext static_ctx = nullptr;
  CUfunction static_fn[6] = {};
  int static_resident[6][17] = {};
};

namespace pyc {

// Bounds-checked builds: whether opts (or $PYC_DEBUG_BOUNDS=1) ask for one, and
// the defines placed before the generated source of such a build.
bool bounds_requested(const pyc_opts& o);
std::string bounds_defines();
// Synchronise the context, then read and clear the violations recorded by a
// checked handle's kernels in the current context -- every unit of its module
// and of `extra` (a map-reduce handle's second module, if compiled): returns
// normally if there were none, else fails with PYC_E_INTERNAL describing the
// first one found.
void check_bounds_record(HandleBase& h, pyc::Module* extra = nullptr);

// Maximum number of chunks of one reduction (bounds the partial workspace).
constexpr int64_t kMaxChunks = 4096;

// Configuration for a launch of n elements: explicit options first, then the
// tuned value of n's bucket, then the built-in default.
LaunchCfg choose_cfg(HandleBase& h, int64_t n, bool reduce);

// Device-side argument struct bytes from the caller's pointers and scalars.
std::vector<unsigned char> pack_args(const ArgSpec& spec, void* const* ptrs, const void* scalars);

// First element index at which every lifted array is vec_bytes-aligned, or -1
// if their alignments are incompatible.  Throws PYC_E_ARG on a null lifted
// array (when n > 0) or an array not aligned to its element size.
int64_t vector_head(const ArgSpec& spec, void* const* ptrs, int vec_bytes, int min_bytes,
                    int64_t n);

// A written array that overlaps another array in part is undefined behaviour
// (only exact aliasing -- the same pointer and element size -- is allowed); for
// arrays indexed as name[i] over [0, n) it is detectable: PYC_E_ARG.
void check_overlap(const ArgSpec& spec, void* const* ptrs, int64_t n);

// Resident CTAs of `f` at `block` threads on the current device.
// CTAs of f that fit on the device at once (dyn_smem: dynamic shared bytes per CTA).
int resident_ctas(CUfunction f, int block, int dyn_smem = 0);

// Chunking of a single reduction of n elements (head from vector_head).
struct ChunkPlan {
  int64_t head = -1;
  int64_t chunk = 0;
  int64_t nchunks = 0;
  int grid = 1;
};
ChunkPlan plan_chunks(int64_t n, int64_t head, int64_t tile, int resident);

// The handle's workspace (partials + ticket) for the current context and
// `stream`, allocated and zeroed by its first use.
pyc_reduce::Workspace& reduce_workspace(pyc_reduce* h, CUstream stream);

// Enqueue one reduction (used by pyc_reduce_launch and the tuner).
void launch_reduce(pyc_reduce* h, const LaunchCfg& cfg, int64_t n, void* const* ptrs,
                   const void* scalars, void* d_out, CUstream stream);
// Enqueue one map.
void launch_map(pyc_map* h, const LaunchCfg& cfg, int64_t n, void* const* ptrs,
                const void* scalars, CUstream stream);

// Times every (variant, block) candidate of a handle with `launch_one` on
// scratch buffers for n's size bucket and keeps the fastest (tune.cpp).
// launch_one(cfg, n, ptrs, scalars, out, stream) enqueues one launch on stream.
// With graph_timing, kernels shorter than ~40 us are timed as replays of a CUDA
// graph of 20 launches (on the context's private capture stream), so that the
// host's per-launch latency is not part of the sample.
using TuneLaunch = std::function<void(const LaunchCfg&, int64_t, void* const*, const void*,
                                      CUdeviceptr, CUstream)>;
void autotune_generic(HandleBase& h, int64_t n, CUstream stream, bool reduce,
                      const TuneLaunch& launch_one, bool graph_timing = false);

// With the environment variable PYC_AUTOTUNE=1, tunes the size bucket of n
// after a launch when it has no tuned configuration yet, the handle's options
// leave something to choose, the stream is not being captured and no other
// thread is tuning the handle; otherwise does nothing.
void autotune_if_due(HandleBase& h, int64_t n, CUstream stream, bool reduce,
                     const TuneLaunch& launch_one, bool graph_timing = false);

// One private non-blocking stream per context, used for graph capture.
CUstream capture_stream();

// Persistent tuning cache (JSON lines in the kernel cache directory).
void tune_cache_load(HandleBase& h, bool reduce);
void tune_cache_store(const HandleBase& h, bool reduce, int bucket, const LaunchCfg& c,
                      double us);

// Work lists of batched launches (worklist.cpp), shared by the segmented
// reducer and the server.  Each task is one independent map / reduction over
// its own (already offset) arrays.
constexpr int64_t kSmallTask = 2048;       // reductions up to this length: one warp each
constexpr int64_t kChunkElems = 1 << 16;   // chunk length of long tasks (rounded to tiles)

struct ReduceTaskIn {
  void* const* ptrs;
  const void* scalars;
  int64_t n;
  void* out;
};
struct ReduceItem {
  int32_t task, chunk, count, pad;  // chunk < 0: warp bundle of `count` short tasks
};
// Writes task records (short tasks first, then long ones, longest first) and
// work items; returns the number of partial slots the list needs.  Long tasks
// are cut into chunks of kChunkElems elements (rounded to whole tiles); with
// spread > 0 into about `spread` chunks of at least min_chunk elements each
// instead, capped at that length.  A task's chunking depends on its own length
// and the configuration only, so its result does not depend on the other tasks.
int64_t write_reduce_work(const pyc_reduce* h, const LaunchCfg& cfg,
                          const std::vector<ReduceTaskIn>& in, std::vector<unsigned char>& tasks,
                          std::vector<ReduceItem>& items, int64_t spread = 0,
                          int64_t min_chunk = 0);

struct MapTaskIn {
  void* const* ptrs;
  const void* scalars;
  int64_t n;
};
struct MapItem {
  int32_t task, chunk;
};
void write_map_work(const pyc_map* h, const LaunchCfg& cfg, const std::vector<MapTaskIn>& in,
                    std::vector<unsigned char>& tasks, std::vector<MapItem>& items,
                    int64_t spread = 0, int64_t min_chunk = 0);

// Batched reducer (batched.cpp).  The configuration of batched launches (the
// segmented reducer and the server's batches) is tuned separately from single
// launches and kept under this pseudo size bucket.
constexpr int kBatchedBucket = -1;
LaunchCfg batched_cfg(HandleBase& h, bool reduce);
void reduce_batched(pyc_reduce* h, int64_t nseg, const int64_t* offsets, void* const* ptrs,
                    const void* scalars, void* d_out, CUstream stream);
void reduce_batched_autotune(pyc_reduce* h, int64_t nseg, const int64_t* offsets,
                             void* const* ptrs, const void* scalars, void* d_out,
                             CUstream stream);
void free_plans(pyc_reduce* h);
void free_host_pipe(pyc_map* h);

}  // namespace pyc
