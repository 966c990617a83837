// Segmented (batched) map-reduce: many independent reductions in one
// persistent launch over a work list, replayed as a CUDA graph.
//
// Plan (built once per segment table, pointers, scalars and output): every
// segment becomes a task over its own offset pointers, and the work list is
// written by write_reduce_work (short segments one warp each, long ones in
// chunks with a per-segment ticket).  CTAs pull items from an atomic counter,
// which the last CTA to leave resets, so replays need no memset.
// The launch is captured once into a graph on a private stream and replayed on
// the caller's stream; while the caller's stream is itself being captured the
// kernel is launched directly so it becomes part of the caller's graph.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

namespace {
constexpr size_t kMaxPlans = 8;
}  // namespace

struct BatchPlan {
  std::string key;
  CUcontext ctx = nullptr;
  CUdeviceptr mem = 0;
  CUdeviceptr tasks = 0, items = 0, tickets = 0, ctl = 0, part = 0;
  int nitems = 0;
  int grid = 1;
  LaunchCfg cfg;
  CUfunction f = nullptr;
  CUgraph graph = nullptr;
  CUgraphExec exec = nullptr;

  void launch_direct(CUstream s) {
    void* params[] = {&tasks, &items, &nitems, &part, &tickets, &ctl};
    PYC_CU(drv().cuLaunchKernel(f, (unsigned)grid, 1, 1, (unsigned)cfg.block, 1, 1, 0, s, params,
                                nullptr));
  }
  void release() {
    const Driver& d = drv();
    if (exec) d.cuGraphExecDestroy(exec);
    if (graph) d.cuGraphDestroy(graph);
    if (mem) d.cuMemFree(mem);
    exec = nullptr;
    graph = nullptr;
    mem = 0;
  }
};

CUstream capture_stream() {
  static std::mutex mu;
  static std::map<CUcontext, CUstream> streams;
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(mu);
  auto it = streams.find(ctx);
  if (it != streams.end()) return it->second;
  CUstream s;
  PYC_CU(drv().cuStreamCreate(&s, CU_STREAM_NON_BLOCKING));
  streams[ctx] = s;
  return s;
}

namespace {

std::unique_ptr<BatchPlan> build_plan(pyc_reduce* h, int64_t nseg, const int64_t* off,
                                      void* const* ptrs, const void* scalars, void* d_out,
                                      const LaunchCfg& cfg) {
  const ArgSpec& spec = h->spec;
  const ReduceGen& g = h->gen;
  auto plan = std::make_unique<BatchPlan>();
  plan->cfg = cfg;
  plan->ctx = ensure_context();
  // every segment becomes a task over its own offset pointers
  const size_t np = spec.num_ptrs ? spec.num_ptrs : 1;
  std::vector<void*> tptrs((size_t)nseg * np, nullptr);
  std::vector<ReduceTaskIn> in((size_t)nseg);
  for (int64_t s = 0; s < nseg; ++s) {
    void** tp = &tptrs[(size_t)s * np];
    for (auto& p : spec.params)
      if (p.is_ptr)
        tp[p.ptr_slot] = static_cast<char*>(ptrs[p.ptr_slot]) + off[s] * type_info(p.dtype).bytes;
    in[s] = {tp, scalars, off[s + 1] - off[s], static_cast<char*>(d_out) + s * g.out_bytes};
  }
  std::vector<unsigned char> tasks;
  std::vector<ReduceItem> items;
  int64_t slots = write_reduce_work(h, cfg, in, tasks, items);
  plan->nitems = (int)items.size();

  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t b_tasks = up(tasks.size()), b_items = up(items.size() * sizeof(ReduceItem));
  size_t b_tickets = up((size_t)nseg * 4), b_ctl = 256;
  size_t b_part = up((size_t)std::max<int64_t>(slots, 1) * g.acc_bytes);
  const Driver& d = drv();
  PYC_CU(d.cuMemAlloc(&plan->mem, b_tasks + b_items + b_tickets + b_ctl + b_part));
  try {
    plan->tasks = plan->mem;
    plan->items = plan->tasks + b_tasks;
    plan->tickets = plan->items + b_items;
    plan->ctl = plan->tickets + b_tickets;
    plan->part = plan->ctl + b_ctl;
    if (!tasks.empty()) PYC_CU(d.cuMemcpyHtoD(plan->tasks, tasks.data(), tasks.size()));
    if (!items.empty())
      PYC_CU(d.cuMemcpyHtoD(plan->items, items.data(), items.size() * sizeof(ReduceItem)));
    PYC_CU(d.cuMemsetD8(plan->tickets, 0, b_tickets + b_ctl));

    plan->f = h->batched_module(cfg).function(h->rbatch_name(cfg));
    int resident = resident_ctas(plan->f, cfg.block);
    plan->grid = std::max(1, std::min(resident, plan->nitems));

    CUstream cs = capture_stream();
    PYC_CU(d.cuStreamBeginCapture(cs, CU_STREAM_CAPTURE_MODE_THREAD_LOCAL));
    try {
      plan->launch_direct(cs);
    } catch (...) {
      CUgraph tmp = nullptr;
      d.cuStreamEndCapture(cs, &tmp);
      if (tmp) d.cuGraphDestroy(tmp);
      throw;
    }
    PYC_CU(d.cuStreamEndCapture(cs, &plan->graph));
    PYC_CU(d.cuGraphInstantiateWithFlags(&plan->exec, plan->graph, 0));
    log_event("segmented plan for %lld segments: %d work items, %zu bytes on the device, %s",
              (long long)nseg, plan->nitems, b_tasks + b_items + b_tickets + b_ctl + b_part,
              h->rbatch_name(cfg).c_str());
  } catch (...) {
    // a copy, a compilation (the register-lean module is built on first use) or
    // the graph failed: the plan's memory goes back before the error surfaces
    plan->release();
    throw;
  }
  return plan;
}

}  // namespace

namespace {

// Everything that can be rejected before any GPU work: the plan's cache key and
// the task records read ptrs[] and the scalar block, so NULLs stop here.
void check_batched_args(pyc_reduce* h, int64_t nseg, const int64_t* off, void* const* ptrs,
                        const void* scalars, void* d_out) {
  if (nseg < 0) fail(PYC_E_ARG, "nseg must be >= 0");
  if (nseg > (int64_t)INT32_MAX / 2) fail(PYC_E_ARG, "too many segments");
  if (nseg == 0) return;
  if (!off) fail(PYC_E_ARG, "seg_offsets is NULL");
  if (!d_out) fail(PYC_E_ARG, "d_out is NULL");
  if (h->spec.num_ptrs > 0 && !ptrs) fail(PYC_E_ARG, "ptrs is NULL but the spec declares arrays");
  if (h->spec.scalar_bytes > 0 && !scalars)
    fail(PYC_E_ARG, "scalars is NULL but the spec declares scalar parameters");
  if (reinterpret_cast<uintptr_t>(d_out) % (uintptr_t)std::min(h->gen.out_bytes, 8))
    fail(PYC_E_ARG, "d_out is not aligned to the result type");
  if (off[0] < 0) fail(PYC_E_ARG, "seg_offsets[0] must be >= 0");
  for (int64_t s = 0; s < nseg; ++s)
    if (off[s + 1] < off[s]) fail(PYC_E_ARG, "seg_offsets must be non-decreasing");
}

}  // namespace

LaunchCfg batched_cfg(HandleBase& h, bool reduce) {
  LaunchCfg c;
  bool tuned = false;
  {
    std::lock_guard<std::mutex> lk(h.tune.mu);
    auto it = h.tune.by_bucket.find(kBatchedBucket);
    if (it != h.tune.by_bucket.end()) {
      c = it->second;
      tuned = true;
    }
  }
  if (!tuned) {
    if (reduce) {
      c.v = Variant{16, 1};  // short segments are one warp each: small tiles
      c.block = 256;
    } else {
      c = choose_cfg(h, (int64_t)1 << 26, false);
    }
  }
  if (h.opts.block) c.block = h.opts.block;
  if (h.opts.vec_bytes) c.v.vec_bytes = h.opts.vec_bytes;
  if (h.opts.items_per_thread) c.v.unroll = h.opts.items_per_thread;
  // a configuration fixed by options is the regular build; only 16-byte
  // reductions have a lean one
  if (!reduce || c.v.vec_bytes != 16 || h.opts.block || h.opts.vec_bytes ||
      h.opts.items_per_thread)
    c.lean = 0;
  return c;
}

void reduce_batched(pyc_reduce* h, int64_t nseg, const int64_t* off, void* const* ptrs,
                    const void* scalars, void* d_out, CUstream stream) {
  check_batched_args(h, nseg, off, ptrs, scalars, d_out);
  if (nseg == 0) return;
  LaunchCfg cfg = batched_cfg(*h, true);

  // key: everything the plan bakes in
  std::string k;
  CUcontext ctx = ensure_context();
  k.append(reinterpret_cast<const char*>(&ctx), sizeof(ctx));
  k.append(reinterpret_cast<const char*>(&cfg), sizeof(cfg));
  k.append(reinterpret_cast<const char*>(&d_out), sizeof(d_out));
  k.append(reinterpret_cast<const char*>(off), (size_t)(nseg + 1) * 8);
  if (h->spec.num_ptrs) k.append(reinterpret_cast<const char*>(ptrs), (size_t)h->spec.num_ptrs * 8);
  if (h->spec.scalar_bytes && scalars)
    k.append(reinterpret_cast<const char*>(scalars), (size_t)h->spec.scalar_bytes);
  std::string key = digest(k) + std::to_string(k.size());

  BatchPlan* plan = nullptr;
  {
    std::lock_guard<std::mutex> lk(h->plan_mu);
    for (size_t j = 0; j < h->plans.size(); ++j)
      if (h->plans[j]->key == key) {
        std::unique_ptr<BatchPlan> p = std::move(h->plans[j]);
        h->plans.erase(h->plans.begin() + (long)j);
        h->plans.push_back(std::move(p));
        plan = h->plans.back().get();
        break;
      }
    if (!plan) {
      std::unique_ptr<BatchPlan> p = build_plan(h, nseg, off, ptrs, scalars, d_out, cfg);
      p->key = key;
      h->plans.push_back(std::move(p));
      while (h->plans.size() > kMaxPlans) {
        h->plans.front()->release();
        h->plans.erase(h->plans.begin());
      }
      plan = h->plans.back().get();
    }
  }
  CUstreamCaptureStatus cap = CU_STREAM_CAPTURE_STATUS_NONE;
  if (stream) PYC_CU(drv().cuStreamIsCapturing(stream, &cap));
  if (cap == CU_STREAM_CAPTURE_STATUS_ACTIVE)
    plan->launch_direct(stream);
  else
    PYC_CU(drv().cuGraphLaunch(plan->exec, stream));
}

}  // namespace pyc

pyc_reduce::pyc_reduce() = default;
pyc_reduce::~pyc_reduce() = default;

namespace pyc {

// Times every (variant, block) candidate on the caller's segment table (one
// plan and graph each, three replays, best kept) and keeps the fastest as the
// handle's batched configuration (also persisted in the tuning cache).
void reduce_batched_autotune(pyc_reduce* h, int64_t nseg, const int64_t* off, void* const* ptrs,
                             const void* scalars, void* d_out, CUstream stream) {
  check_batched_args(h, nseg, off, ptrs, scalars, d_out);
  if (nseg == 0) fail(PYC_E_ARG, "autotune needs nseg > 0");
  const Driver& d = drv();
  CUevent e0, e1;
  PYC_CU(d.cuEventCreate(&e0, CU_EVENT_DEFAULT));
  PYC_CU(d.cuEventCreate(&e1, CU_EVENT_DEFAULT));
  LaunchCfg best;
  double best_us = 1e30;
  try {
    for (const Variant& v : all_variants()) {
      if (h->opts.vec_bytes && v.vec_bytes != h->opts.vec_bytes) continue;
      if (h->opts.items_per_thread && v.unroll != h->opts.items_per_thread) continue;
      static const int kBlocks[3] = {128, 256, 512};
      for (int lb = 0; lb < 6; ++lb) {
        const int b = kBlocks[lb % 3];
        const int lean = lb / 3;
        if (lean && v.vec_bytes != 16) continue;  // only the 16-byte variants have it
        if (h->opts.block && b != h->opts.block) continue;
        LaunchCfg c;
        c.v = v;
        c.block = b;
        c.lean = lean;
        std::unique_ptr<BatchPlan> plan = build_plan(h, nseg, off, ptrs, scalars, d_out, c);
        double us = 1e30;
        try {
          PYC_CU(d.cuGraphLaunch(plan->exec, stream));
          for (int r = 0; r < 3; ++r) {
            PYC_CU(d.cuEventRecord(e0, stream));
            PYC_CU(d.cuGraphLaunch(plan->exec, stream));
            PYC_CU(d.cuEventRecord(e1, stream));
            PYC_CU(d.cuEventSynchronize(e1));
            float ms = 0;
            PYC_CU(d.cuEventElapsedTime(&ms, e0, e1));
            us = std::min(us, (double)ms * 1000.0);
          }
        } catch (...) {
          plan->release();
          throw;
        }
        plan->release();
        if (std::getenv("PYC_TUNE_LOG"))
          std::fprintf(stderr, "pyc tune batched %s nseg=%lld vec=%d unroll=%d block=%d lean=%d %.2f us\n",
                       h->tag.c_str(), (long long)nseg, v.vec_bytes, v.unroll, b, lean, us);
        if (us < best_us) {
          best_us = us;
          best = c;
        }
      }
    }
  } catch (...) {
    d.cuEventDestroy(e0);
    d.cuEventDestroy(e1);
    throw;
  }
  d.cuEventDestroy(e0);
  d.cuEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(h->tune.mu);
    h->tune.by_bucket[kBatchedBucket] = best;
  }
  tune_cache_store(*h, true, kBatchedBucket, best, best_us);
}

// Host-side view of the work plan pyc_reduce_batched builds for a segment
// table: the same task construction as build_plan (tasks over each segment's
// offset pointers) and the same work list writer, with a stand-in output base
// so that each task record names its segment.  Nothing touches a GPU.
void reduce_batched_plan(pyc_reduce* h, int64_t nseg, const int64_t* off, void* const* ptrs,
                         const void* scalars, int64_t* task_info, int32_t* items_out,
                         int64_t items_cap, int64_t* n_items, int64_t* n_slots) {
  char* const base = reinterpret_cast<char*>((uintptr_t)1 << 20);  // never written
  check_batched_args(h, nseg, off, ptrs, scalars, base);
  if (n_items) *n_items = 0;
  if (n_slots) *n_slots = 0;
  if (nseg == 0) return;
  const LaunchCfg cfg = batched_cfg(*h, true);
  const ArgSpec& spec = h->spec;
  const ReduceGen& g = h->gen;
  const size_t np = spec.num_ptrs ? spec.num_ptrs : 1;
  std::vector<void*> tptrs((size_t)nseg * np, nullptr);
  std::vector<ReduceTaskIn> in((size_t)nseg);
  for (int64_t s = 0; s < nseg; ++s) {
    void** tp = &tptrs[(size_t)s * np];
    for (auto& p : spec.params)
      if (p.is_ptr)
        tp[p.ptr_slot] = static_cast<char*>(ptrs[p.ptr_slot]) + off[s] * type_info(p.dtype).bytes;
    in[s] = {tp, scalars, off[s + 1] - off[s], base + s * g.out_bytes};
  }
  std::vector<unsigned char> tasks;
  std::vector<ReduceItem> items;
  const int64_t slots = write_reduce_work(h, cfg, in, tasks, items);
  if (items_out && (int64_t)items.size() > items_cap)
    fail(PYC_E_ARG, "items_cap " + std::to_string(items_cap) + " < " +
                        std::to_string(items.size()) + " work items");
  if (n_items) *n_items = (int64_t)items.size();
  if (n_slots) *n_slots = slots;
  if (items_out)
    for (size_t k = 0; k < items.size(); ++k) {
      items_out[4 * k] = items[k].task;
      items_out[4 * k + 1] = items[k].chunk;
      items_out[4 * k + 2] = items[k].count;
      items_out[4 * k + 3] = 0;
    }
  if (task_info)
    for (int64_t t = 0; t < nseg; ++t) {
      const unsigned char* rec = &tasks[(size_t)t * g.task_bytes];
      int64_t n, head, chunk;
      char* out;
      int32_t nchunks, slot0;
      std::memcpy(&n, rec + g.task_off_n, 8);
      std::memcpy(&head, rec + g.task_off_head, 8);
      std::memcpy(&chunk, rec + g.task_off_chunk, 8);
      std::memcpy(&out, rec + g.task_off_out, 8);
      std::memcpy(&nchunks, rec + g.task_off_nchunks, 4);
      std::memcpy(&slot0, rec + g.task_off_slot0, 4);
      int64_t* ti = task_info + 6 * t;
      ti[0] = (int64_t)((out - base) / g.out_bytes);
      ti[1] = n;
      ti[2] = head;
      ti[3] = chunk;
      ti[4] = nchunks;
      ti[5] = slot0;
    }
}

void free_plans(pyc_reduce* h) {
  std::lock_guard<std::mutex> lk(h->plan_mu);
  for (auto& p : h->plans) p->release();
  h->plans.clear();
}

}  // namespace pyc

using namespace pyc;

PYC_API pyc_status pyc_reduce_batched_plan(pyc_reduce_t h, int64_t nseg,
                                           const int64_t* seg_offsets, void* const* ptrs,
                                           const void* scalars, int64_t* task_info,
                                           int32_t* items, int64_t items_cap, int64_t* n_items,
                                           int64_t* n_slots) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    reduce_batched_plan(h, nseg, seg_offsets, ptrs, scalars, task_info, items, items_cap, n_items,
                        n_slots);
  });
}
