// Serving loop: continuous batching of map and map-reduce requests.
//
// A client thread submits requests (a handle, n, device pointers, scalars).
// One scheduler thread per server, in a loop:
//  1. retires launched batches whose completion event has fired (results of
//     reductions are copied back to pinned host memory by the batch itself);
//  2. admits queued requests in arrival order while the logical bytes of
//     admitted, unreleased requests stay within the memory budget and the
//     arena can hold the outputs the server allocates for them;
//  3. groups the admitted requests by handle and launches each group as one
//     batched kernel (one work item per chunk, short reductions one warp each)
//     on the next of several streams, as long as a batch slot is free.
// Requests that arrive while others run are admitted as memory and slots free
// up, and batches on different streams overlap on the device.  A request's
// result depends only on the request itself (its work list and the handle's
// fixed batch configuration), never on the rest of its batch.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <thread>
#include <unordered_map>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Best-fit allocator over one device allocation, 256-byte granules, with
// coalescing of neighbouring free ranges.
class Arena {
 public:
  void init(int64_t bytes) {
    cap_ = bytes;
    free_by_off_[0] = bytes;
    free_by_size_.insert({bytes, 0});
  }
  bool alloc(int64_t bytes, int64_t* off) {
    bytes = round_up(std::max<int64_t>(bytes, 1), 256);
    auto it = free_by_size_.lower_bound({bytes, -1});
    if (it == free_by_size_.end()) return false;
    int64_t sz = it->first, o = it->second;
    free_by_size_.erase(it);
    free_by_off_.erase(o);
    if (sz > bytes) {
      free_by_off_[o + bytes] = sz - bytes;
      free_by_size_.insert({sz - bytes, o + bytes});
    }
    used_[o] = bytes;
    in_use_ += bytes;
    *off = o;
    return true;
  }
  void release(int64_t o) {
    auto u = used_.find(o);
    if (u == used_.end()) return;
    int64_t sz = u->second;
    used_.erase(u);
    in_use_ -= sz;
    auto next = free_by_off_.lower_bound(o);
    if (next != free_by_off_.end() && o + sz == next->first) {
      free_by_size_.erase({next->second, next->first});
      sz += next->second;
      next = free_by_off_.erase(next);
    }
    if (next != free_by_off_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        free_by_size_.erase({prev->second, prev->first});
        o = prev->first;
        sz += prev->second;
        free_by_off_.erase(prev);
      }
    }
    free_by_off_[o] = sz;
    free_by_size_.insert({sz, o});
  }
  int64_t in_use() const { return in_use_; }

 private:
  int64_t cap_ = 0, in_use_ = 0;
  std::map<int64_t, int64_t> free_by_off_;
  std::set<std::pair<int64_t, int64_t>> free_by_size_;
  std::map<int64_t, int64_t> used_;
};

enum ReqState { kQueued, kAdmitted, kLaunched, kDone, kFailed };

struct SReq {
  uint64_t id = 0;
  int kind = 0;
  pyc_map* mh = nullptr;
  pyc_reduce* rh = nullptr;
  int64_t n = 0;
  std::vector<void*> ptrs;
  std::vector<unsigned char> scalars;
  int64_t deadline_ns = 0;
  int64_t bytes = 0;
  bool counted = false;         // bytes are included in the admitted total
  std::vector<int> alloc_slots;  // pointer slots the server allocates
  std::vector<int64_t> out_offs;
  int state = kQueued;
  pyc_result res{};
  HandleBase* handle() const { return mh ? static_cast<HandleBase*>(mh) : rh; }
};

constexpr int64_t kSlotDevBytes = 16 << 20;
constexpr int64_t kSlotHostBytes = 16 << 20;
constexpr int64_t kCtlBytes = 256;
// Work lists up to this size are read by the batch kernel from page-locked host
// memory instead of being copied to the device first.
constexpr int64_t kDirectListBytes = 8192;
// A request is cut into about kServeSpread chunks of at least kServeMinChunk
// elements (at most the work list's usual chunk length), so that one request
// arriving alone runs on many CTAs: a function of its own length only, so a
// reduction's bits are the same alone and in any batch.
constexpr int64_t kServeSpread = 256;
constexpr int64_t kServeMinChunk = 4096;
// Chunks of one batch at most (work items and partial slots of a slot).
constexpr int64_t kBatchChunks = (int64_t)1 << 17;

struct Slot {
  CUdeviceptr dev = 0;
  unsigned char* host = nullptr;
  CUevent ev = nullptr;
  bool busy = false;
  // host execution (pyc_server_create_host): the batch's requests, and per
  // request its status and result, filled by the executor thread; done is set
  // under the server lock once every request has been computed
  std::vector<SReq*> host_reqs;
  std::vector<int> host_status;
  std::vector<std::array<unsigned char, 16>> host_vals;
  bool host_done = false;
};

struct Batch {
  int kind = 0;
  HandleBase* h = nullptr;
  std::vector<SReq*> reqs;
  int slot = -1;
  int64_t res_host_off = 0;
  int out_bytes = 0;
};

// Offset (bytes, below 256) at which a server-allocated output starts inside
// its arena block (256-byte granules): the address of the request's first given
// array modulo 256, rounded down to the output's element size.  Arrays at equal
// addresses modulo the vector width take the vector path together; inputs at
// arbitrary element offsets would otherwise leave a 256-byte-aligned output
// alone and the whole request element-wise.
int64_t align_shift(const HandleBase& h, void* const* ptrs, int64_t out_eb) {
  for (auto& q : h.spec.params)
    if (q.is_ptr && q.lifted && ptrs[q.ptr_slot]) {
      const int64_t m = (int64_t)(reinterpret_cast<uintptr_t>(ptrs[q.ptr_slot]) % 256);
      return m / out_eb * out_eb;
    }
  return 0;
}

// Launch configuration the server uses for a handle's batches: fixed per
// handle so that a request's result never depends on its batch.
LaunchCfg batch_cfg(HandleBase& h, bool reduce) { return batched_cfg(h, reduce); }

}  // namespace

}  // namespace pyc

struct pyc_server {
  pyc_server_cfg cfg{};
  CUcontext ctx = nullptr;
  std::vector<CUstream> streams;
  int next_stream = 0;
  CUdeviceptr arena_mem = 0;
  pyc::Arena arena;
  std::vector<pyc::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::unordered_map<uint64_t, std::unique_ptr<pyc::SReq>> reqs;
  std::deque<pyc::SReq*> queue;
  std::vector<pyc::SReq*> admitted;
  std::deque<pyc::Batch> inflight;  // touched by the scheduler thread only
  std::deque<uint64_t> finished;    // ids finished since the last take (during a replay)
  bool track_finished = false;
  std::atomic<uint64_t> nfinished{0};  // requests finished so far (wakes pollers)
  std::atomic<uint64_t> nevents{0};    // submissions + releases (wakes the scheduler)
  uint64_t next_id = 1;
  int64_t admitted_bytes = 0;
  pyc_server_stats stats{};
  bool stop = false;
  std::string fatal;
  std::thread th;
  // host execution (test hook): batches run on exec_th through host_exec
  pyc_host_exec_fn host_exec = nullptr;
  void* host_user = nullptr;
  std::vector<unsigned char> host_arena;
  std::mutex exec_mu;
  std::condition_variable exec_cv;
  std::deque<int> exec_queue;  // slots whose batches wait for the executor
  bool exec_stop = false;
  std::thread exec_th;
};

namespace pyc {

namespace {

void finish_req(pyc_server* s, SReq* r, int status, int64_t t) {
  r->res.status = status;
  r->res.t_done_ns = t;
  r->state = status == PYC_OK ? kDone : kFailed;
  if (status == PYC_OK)
    ++s->stats.completed;
  else
    ++s->stats.failed;
  if (s->track_finished) s->finished.push_back(r->id);
  ++s->nfinished;
}

// Slot layout.  Device: [ctl][tickets][results][tasks][items][partials].  The
// ticket and control words sit at fixed offsets so they stay zero between
// batches (the kernels reset what they use); results sit at a fixed offset so
// output pointers are known before the work list is written.  Host (pinned):
// [tasks][items] staged from offset 0, results copied back to a fixed offset.
struct SlotLayout {
  int64_t res = 0, tasks = 0, items = 0, part = 0, dev_end = 0;
  int64_t task_bytes = 0, item_bytes = 0, res_bytes = 0;
  int64_t host_res = 0;
};

SlotLayout layout(int max_batch, int64_t task_bytes, int64_t item_bytes, int64_t part_bytes,
                  int64_t res_bytes) {
  SlotLayout L;
  L.task_bytes = task_bytes;
  L.item_bytes = item_bytes;
  L.res_bytes = res_bytes;
  L.res = kCtlBytes + round_up((int64_t)max_batch * 4, 256);
  L.tasks = L.res + round_up((int64_t)max_batch * 16, 256);
  L.items = L.tasks + task_bytes;
  L.part = round_up(L.items + item_bytes, 256);
  L.dev_end = L.part + part_bytes;
  L.host_res = kSlotHostBytes - round_up((int64_t)max_batch * 16, 256);
  return L;
}

// Builds and enqueues one batch (without the server lock: it reads only the
// batch's immutable request fields and its own slot).
void launch_batch(pyc_server* s, Batch& b) {
  if (s->host_exec) {
    // hand the batch to the executor thread (its slot is this batch's alone)
    Slot& hs = s->slots[b.slot];
    hs.host_reqs = b.reqs;
    hs.host_status.assign(b.reqs.size(), PYC_E_INTERNAL);
    hs.host_vals.assign(b.reqs.size(), {});
    hs.host_done = false;
    b.out_bytes = b.kind == PYC_REQ_REDUCE ? static_cast<pyc_reduce*>(b.h)->gen.out_bytes : 0;
    {
      std::lock_guard<std::mutex> lk(s->exec_mu);
      s->exec_queue.push_back(b.slot);
    }
    s->exec_cv.notify_one();
    return;
  }
  const Driver& d = drv();
  Slot& sl = s->slots[b.slot];
  CUstream st = s->streams[s->next_stream];
  s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
  const bool reduce = b.kind == PYC_REQ_REDUCE;
  LaunchCfg cfg = batch_cfg(*b.h, reduce);
  std::vector<unsigned char> tasks;
  int nitems = 0;
  SlotLayout L;
  CUfunction f;
  // results go straight to the slot's page-locked host area (the kernel writes
  // them over the chip-to-chip link; no copy back after the kernel)
  const int64_t host_res = layout(s->cfg.max_batch, 0, 0, 0, 0).host_res;
  if (reduce) {
    pyc_reduce* h = static_cast<pyc_reduce*>(b.h);
    std::vector<ReduceTaskIn> in;
    std::vector<ReduceItem> items;
    for (size_t k = 0; k < b.reqs.size(); ++k)
      in.push_back({b.reqs[k]->ptrs.data(), b.reqs[k]->scalars.data(), b.reqs[k]->n,
                    static_cast<void*>(sl.host + host_res + (int64_t)k * h->gen.out_bytes)});
    int64_t nslots = write_reduce_work(h, cfg, in, tasks, items, kServeSpread, kServeMinChunk);
    L = layout(s->cfg.max_batch, (int64_t)tasks.size(), (int64_t)(items.size() * sizeof(ReduceItem)),
               round_up(std::max<int64_t>(nslots, 1) * h->gen.acc_bytes, 256),
               (int64_t)b.reqs.size() * h->gen.out_bytes);
    if (L.dev_end > kSlotDevBytes || L.task_bytes + L.item_bytes > L.host_res)
      fail(PYC_E_INTERNAL, "batch does not fit its slot");
    std::memcpy(sl.host, tasks.data(), tasks.size());
    if (!items.empty())
      std::memcpy(sl.host + tasks.size(), items.data(), items.size() * sizeof(ReduceItem));
    nitems = (int)items.size();
    f = h->batched_module(cfg).function(h->rbatch_name(cfg));
    b.res_host_off = L.host_res;
    b.out_bytes = h->gen.out_bytes;
  } else {
    pyc_map* h = static_cast<pyc_map*>(b.h);
    std::vector<MapTaskIn> in;
    std::vector<MapItem> items;
    for (SReq* r : b.reqs) in.push_back({r->ptrs.data(), r->scalars.data(), r->n});
    write_map_work(h, cfg, in, tasks, items, kServeSpread, kServeMinChunk);
    L = layout(s->cfg.max_batch, (int64_t)tasks.size(), (int64_t)(items.size() * sizeof(MapItem)),
               0, 0);
    if (L.dev_end > kSlotDevBytes || L.task_bytes + L.item_bytes > L.host_res)
      fail(PYC_E_INTERNAL, "batch does not fit its slot");
    std::memcpy(sl.host, tasks.data(), tasks.size());
    if (!items.empty())
      std::memcpy(sl.host + tasks.size(), items.data(), items.size() * sizeof(MapItem));
    nitems = (int)items.size();
    f = h->mod->function(h->kname("pyc_mbatch", cfg.v));
  }
  if (nitems > 0) {
    // a small work list is read by the kernel from the page-locked slot itself;
    // a larger one (read by many CTAs) is copied to the device first
    const bool direct = L.task_bytes + L.item_bytes <= kDirectListBytes;
    if (!direct)
      PYC_CU(d.cuMemcpyHtoDAsync(sl.dev + L.tasks, sl.host, (size_t)(L.task_bytes + L.item_bytes),
                                 st));
    int grid = std::max(1, std::min(resident_ctas(f, cfg.block), nitems));
    CUdeviceptr tasks_d = direct ? reinterpret_cast<CUdeviceptr>(sl.host) : sl.dev + L.tasks;
    CUdeviceptr items_d = tasks_d + (CUdeviceptr)(L.items - L.tasks), ctl = sl.dev;
    CUdeviceptr tickets = sl.dev + kCtlBytes, part = sl.dev + L.part;
    if (reduce) {
      void* params[] = {&tasks_d, &items_d, &nitems, &part, &tickets, &ctl};
      PYC_CU(d.cuLaunchKernel(f, (unsigned)grid, 1, 1, (unsigned)cfg.block, 1, 1, 0, st, params,
                              nullptr));
    } else {
      void* params[] = {&tasks_d, &items_d, &nitems, &ctl};
      PYC_CU(d.cuLaunchKernel(f, (unsigned)grid, 1, 1, (unsigned)cfg.block, 1, 1, 0, st, params,
                              nullptr));
    }
  }
  PYC_CU(d.cuEventRecord(sl.ev, st));
}

// Retire the batch (results to the requests, slot freed).  Caller holds mu.
void retire(pyc_server* s, Batch& b, int status) {
  Slot& sl = s->slots[b.slot];
  const int64_t t = now_ns();
  for (size_t k = 0; k < b.reqs.size(); ++k) {
    SReq* r = b.reqs[k];
    int st = status;
    if (s->host_exec && st == PYC_OK) {
      st = sl.host_status[k];
      if (st == PYC_OK && b.kind == PYC_REQ_REDUCE)
        std::memcpy(r->res.value, sl.host_vals[k].data(), (size_t)b.out_bytes);
    } else if (st == PYC_OK && b.kind == PYC_REQ_REDUCE) {
      std::memcpy(r->res.value, sl.host + b.res_host_off + (int64_t)k * b.out_bytes, b.out_bytes);
    }
    if (st == PYC_OK && b.kind == PYC_REQ_MAP && !r->alloc_slots.empty())
      r->res.d_out = r->ptrs[r->alloc_slots[0]];
    finish_req(s, r, st, t);
  }
  sl.host_reqs.clear();
  sl.busy = false;
  ++s->stats.batches;
}

// The executor thread of a host-executed server: computes each handed-over
// batch through host_exec, request by request, then marks its slot done.
void host_executor(pyc_server* s) {
  for (;;) {
    int slot;
    {
      std::unique_lock<std::mutex> lk(s->exec_mu);
      s->exec_cv.wait(lk, [&] { return s->exec_stop || !s->exec_queue.empty(); });
      if (s->exec_queue.empty()) return;  // stopping, nothing left
      slot = s->exec_queue.front();
      s->exec_queue.pop_front();
    }
    Slot& sl = s->slots[slot];
    for (size_t k = 0; k < sl.host_reqs.size(); ++k) {
      SReq* r = sl.host_reqs[k];
      pyc_request q{};
      q.kind = r->kind;
      q.handle = r->kind == PYC_REQ_MAP ? static_cast<void*>(r->mh) : static_cast<void*>(r->rh);
      q.n = r->n;
      q.ptrs = r->ptrs.data();
      q.scalars = r->scalars.data();
      q.deadline_us = 0;
      sl.host_status[k] = s->host_exec(s->host_user, &q, sl.host_vals[k].data());
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      sl.host_done = true;
    }
    ++s->nevents;
    s->cv_sched.notify_one();
  }
}

void scheduler(pyc_server* s) {
  if (!s->host_exec) drv().cuCtxSetCurrent(s->ctx);
  std::unique_lock<std::mutex> lk(s->mu);
  uint64_t seen = 0;
  auto notify = [&] {
    uint64_t f = s->nfinished.load();
    if (f != seen) {
      seen = f;
      s->cv_done.notify_all();
    }
  };
  for (;;) {
    // 1. retire finished batches
    for (auto it = s->inflight.begin(); it != s->inflight.end();) {
      CUresult q = s->host_exec ? (s->slots[it->slot].host_done ? CUDA_SUCCESS : CUDA_ERROR_NOT_READY)
                                : drv().cuEventQuery(s->slots[it->slot].ev);
      if (q == CUDA_ERROR_NOT_READY) {
        ++it;
        continue;
      }
      if (q != CUDA_SUCCESS && s->fatal.empty()) s->fatal = "a batch failed on the device";
      retire(s, *it, q == CUDA_SUCCESS ? PYC_OK : PYC_E_CUDA);
      it = s->inflight.erase(it);
    }
    notify();
    if (s->stop && s->queue.empty() && s->admitted.empty() && s->inflight.empty()) break;
    // an injected stall (pyc_test_inject): the scheduler is late to admit
    if (const int64_t ms = take_injected_stall_ms()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::milliseconds(ms));
      lk.lock();
    }
    // 2. admission in arrival order
    const int64_t t = now_ns();
    while (!s->queue.empty() && !s->stop) {
      SReq* r = s->queue.front();
      if (r->deadline_ns && t > r->deadline_ns) {
        s->queue.pop_front();
        finish_req(s, r, PYC_E_TIMEOUT, t);
        continue;
      }
      if (take_injected(PYC_INJECT_ADMIT)) {  // an injected rejection (pyc_test_inject)
        s->queue.pop_front();
        finish_req(s, r, PYC_E_NOMEM, t);
        continue;
      }
      if (s->admitted_bytes + r->bytes > s->cfg.mem_budget_bytes) break;
      bool ok = true;
      for (int slot : r->alloc_slots) {
        int64_t off;
        const Param* p = nullptr;
        for (auto& q : r->mh->spec.params)
          if (q.is_ptr && q.ptr_slot == slot) p = &q;
        const int64_t eb = type_info(p->dtype).bytes;
        const int64_t shift = align_shift(*r->mh, r->ptrs.data(), eb);
        if (!s->arena.alloc(r->n * eb + shift, &off)) {
          ok = false;
          break;
        }
        r->out_offs.push_back(off);
        r->ptrs[slot] = reinterpret_cast<void*>(s->arena_mem + off + shift);
      }
      if (!ok) {
        for (int64_t off : r->out_offs) s->arena.release(off);
        r->out_offs.clear();
        if (s->admitted_bytes == 0 && s->inflight.empty()) {  // can never fit
          s->queue.pop_front();
          finish_req(s, r, PYC_E_NOMEM, t);
          continue;
        }
        break;
      }
      s->queue.pop_front();
      r->state = kAdmitted;
      r->res.t_admit_ns = t;
      r->counted = true;
      s->admitted_bytes += r->bytes;
      s->stats.peak_admitted_bytes = std::max(s->stats.peak_admitted_bytes, s->admitted_bytes);
      s->admitted.push_back(r);
    }
    notify();
    // 3. batches: group admitted requests by handle, in arrival order.  While
    //    num_streams batches are already running, admitted requests wait and
    //    accumulate into larger batches, unless a full batch is ready.
    std::vector<Batch> to_launch;
    while (!s->admitted.empty()) {
      int free_slot = -1;
      for (size_t k = 0; k < s->slots.size(); ++k)
        if (!s->slots[k].busy) {
          free_slot = (int)k;
          break;
        }
      if (free_slot < 0) break;
      if ((int)(s->inflight.size() + to_launch.size()) >= s->cfg.num_streams &&
          (int)s->admitted.size() < s->cfg.max_batch)
        break;
      Batch bt;
      bt.h = s->admitted.front()->handle();
      bt.kind = s->admitted.front()->kind;
      std::vector<SReq*> rest;
      int64_t chunks = 0;
      for (SReq* r : s->admitted) {
        // an upper bound on the request's chunks under kServeSpread / kServeMinChunk
        const int64_t rc =
            std::min(r->n / kServeMinChunk, std::max(kServeSpread, r->n / kChunkElems)) + 2;
        if (r->handle() == bt.h && (int)bt.reqs.size() < s->cfg.max_batch &&
            (bt.reqs.empty() || chunks + rc <= kBatchChunks)) {
          bt.reqs.push_back(r);
          chunks += rc;
        } else {
          rest.push_back(r);
        }
      }
      s->admitted.swap(rest);
      bt.slot = free_slot;
      s->slots[free_slot].busy = true;
      to_launch.push_back(std::move(bt));
    }
    if (!to_launch.empty()) {
      // build and enqueue outside the lock: submitters and pollers go on
      std::vector<int> ok(to_launch.size(), 0);
      std::vector<std::string> err(to_launch.size());
      lk.unlock();
      for (size_t k = 0; k < to_launch.size(); ++k) {
        try {
          launch_batch(s, to_launch[k]);
          ok[k] = 1;
        } catch (const std::exception& e) {
          err[k] = e.what();
        }
      }
      lk.lock();
      const int64_t tl = now_ns();
      for (size_t k = 0; k < to_launch.size(); ++k) {
        Batch& bt = to_launch[k];
        if (ok[k]) {
          for (SReq* r : bt.reqs) {
            r->state = kLaunched;
            r->res.t_launch_ns = tl;
            r->res.batch_size = (int32_t)bt.reqs.size();
          }
          s->inflight.push_back(std::move(bt));
        } else {
          if (s->fatal.empty()) s->fatal = err[k];
          s->slots[bt.slot].busy = false;
          for (SReq* r : bt.reqs) finish_req(s, r, PYC_E_CUDA, tl);
        }
      }
    }
    notify();
    // 4. wait: briefly while work is in flight (poll its events), else until
    //    a submission, a release or shutdown
    // (spinning with yields: a timed sleep or a condition-variable wake-up
    //  costs tens of microseconds of latency)
    if (!s->inflight.empty()) {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      const uint64_t ev0 = s->nevents.load();
      lk.unlock();
      const int64_t t_end = now_ns() + 200000;
      while (s->nevents.load() == ev0 && now_ns() < t_end) std::this_thread::yield();
      lk.lock();
      if (s->nevents.load() == ev0 && !s->stop)
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

int64_t request_bytes(const HandleBase& h, int64_t n, int out_bytes) {
  int64_t b = out_bytes;
  for (auto& p : h.spec.params)
    if (p.is_ptr) b += n * type_info(p.dtype).bytes;
  return b;
}

}  // namespace

}  // namespace pyc

using namespace pyc;

namespace pyc {
namespace {
// The configuration with defaults filled in (arena: at most `arena_cap` bytes
// by default); PYC_E_ARG on a bad one.
pyc_server_cfg server_cfg(const pyc_server_cfg* cfg, int64_t arena_cap) {
  if (!cfg) fail(PYC_E_ARG, "cfg is NULL");
  pyc_server_cfg c = *cfg;
  if (c.mem_budget_bytes <= 0) fail(PYC_E_ARG, "mem_budget_bytes must be > 0");
  if (c.num_streams <= 0) c.num_streams = 4;
  if (c.max_batch <= 0) c.max_batch = 256;
  if (c.max_inflight <= 0) c.max_inflight = 8;
  if (c.max_queue <= 0) c.max_queue = 1 << 20;
  if (c.arena_bytes <= 0) c.arena_bytes = std::min<int64_t>(c.mem_budget_bytes, arena_cap);
  if (c.num_streams > 64 || c.max_inflight > 256 || c.max_batch > 4096)
    fail(PYC_E_ARG, "num_streams <= 64, max_inflight <= 256, max_batch <= 4096");
  return c;
}
}  // namespace
}  // namespace pyc

PYC_API pyc_status pyc_server_create(const pyc_server_cfg* cfg, pyc_server_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    const pyc_server_cfg c = server_cfg(cfg, (int64_t)8 << 30);
    auto s = std::make_unique<pyc_server>();
    s->cfg = c;
    s->ctx = ensure_context();
    const Driver& d = drv();
    try {
      for (int k = 0; k < c.num_streams; ++k) {
        CUstream st;
        PYC_CU(d.cuStreamCreate(&st, CU_STREAM_NON_BLOCKING));
        s->streams.push_back(st);
      }
      PYC_CU(d.cuMemAlloc(&s->arena_mem, (size_t)c.arena_bytes));
      s->arena.init(c.arena_bytes);
      s->slots.resize(c.max_inflight);
      for (auto& sl : s->slots) {
        PYC_CU(d.cuMemAlloc(&sl.dev, (size_t)kSlotDevBytes));
        PYC_CU(d.cuMemsetD8(sl.dev, 0, (size_t)kSlotDevBytes));
        void* hp = nullptr;
        PYC_CU(d.cuMemAllocHost(&hp, (size_t)kSlotHostBytes));
        sl.host = static_cast<unsigned char*>(hp);
        PYC_CU(d.cuEventCreate(&sl.ev, CU_EVENT_DISABLE_TIMING));
      }
    } catch (...) {
      for (auto& sl : s->slots) {
        if (sl.dev) d.cuMemFree(sl.dev);
        if (sl.host) d.cuMemFreeHost(sl.host);
        if (sl.ev) d.cuEventDestroy(sl.ev);
      }
      if (s->arena_mem) d.cuMemFree(s->arena_mem);
      for (CUstream st : s->streams) d.cuStreamDestroy(st);
      throw;
    }
    pyc_server* raw = s.get();
    s->th = std::thread([raw] { scheduler(raw); });
    log_event("server created: budget %lld bytes, arena %lld bytes, %d streams, batches of "
              "up to %d, %d in flight", (long long)c.mem_budget_bytes, (long long)c.arena_bytes,
              c.num_streams, c.max_batch, c.max_inflight);
    *out = s.release();
  });
}

PYC_API pyc_status pyc_server_create_host(const pyc_server_cfg* cfg, pyc_host_exec_fn exec,
                                          void* user, pyc_server_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (!exec) fail(PYC_E_ARG, "exec is NULL");
    const pyc_server_cfg c = server_cfg(cfg, (int64_t)256 << 20);
    auto s = std::make_unique<pyc_server>();
    s->cfg = c;
    s->host_exec = exec;
    s->host_user = user;
    // 256-byte aligned, as a device allocation is: outputs keep their inputs' alignment
    s->host_arena.assign((size_t)c.arena_bytes + 256, 0);
    s->arena_mem = (reinterpret_cast<CUdeviceptr>(s->host_arena.data()) + 255) & ~(CUdeviceptr)255;
    s->arena.init(c.arena_bytes);
    s->slots.resize(c.max_inflight);
    pyc_server* raw = s.get();
    s->exec_th = std::thread([raw] { host_executor(raw); });
    s->th = std::thread([raw] { scheduler(raw); });
    log_event("server created with host-executed batches: budget %lld bytes, batches of up to "
              "%d, %d in flight", (long long)c.mem_budget_bytes, c.max_batch, c.max_inflight);
    *out = s.release();
  });
}

PYC_API pyc_status pyc_server_submit(pyc_server_t s, const pyc_request* req, uint64_t* id) {
  return guarded([&] {
    if (!s || !req || !id) fail(PYC_E_ARG, "server, request and id must not be NULL");
    auto r = std::make_unique<SReq>();
    r->kind = req->kind;
    r->n = req->n;
    if (r->n < 0) fail(PYC_E_ARG, "n must be >= 0");
    if (r->n > ((int64_t)1 << 34)) fail(PYC_E_ARG, "request too large for the server (n > 2^34)");
    HandleBase* h = nullptr;
    int out_bytes = 0;
    if (req->kind == PYC_REQ_MAP) {
      r->mh = static_cast<pyc_map*>(req->handle);
      h = r->mh;
    } else if (req->kind == PYC_REQ_REDUCE) {
      r->rh = static_cast<pyc_reduce*>(req->handle);
      h = r->rh;
      if (h) out_bytes = r->rh->gen.out_bytes;
    } else {
      fail(PYC_E_ARG, "kind must be PYC_REQ_MAP or PYC_REQ_REDUCE");
    }
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    const ArgSpec& spec = h->spec;
    if (spec.num_ptrs > 0 && !req->ptrs) fail(PYC_E_ARG, "ptrs is NULL");
    if (spec.scalar_bytes > 0 && !req->scalars) fail(PYC_E_ARG, "scalars is NULL");
    r->ptrs.assign(req->ptrs, req->ptrs + spec.num_ptrs);
    r->ptrs.resize(std::max(1, spec.num_ptrs));
    r->scalars.assign(spec.scalar_bytes + 8, 0);
    if (spec.scalar_bytes)
      std::memcpy(r->scalars.data(), req->scalars, (size_t)spec.scalar_bytes);
    // every array is checked here, so that a bad one fails its own request
    // rather than the batch it would join
    for (auto& p : spec.params) {
      if (!p.is_ptr) continue;
      if (const void* a = r->ptrs[p.ptr_slot]) {
        if (reinterpret_cast<uintptr_t>(a) % (uintptr_t)type_info(p.dtype).bytes)
          fail(PYC_E_ARG, "array '" + p.name + "' is not aligned to its element size");
        continue;
      }
      bool server_out = req->kind == PYC_REQ_MAP && p.lifted && p.written && !p.read;
      if (server_out)
        r->alloc_slots.push_back(p.ptr_slot);
      else if (r->n > 0)
        fail(PYC_E_ARG, "array '" + p.name + "' is NULL (only written-only map outputs may be)");
    }
    check_overlap(spec, r->ptrs.data(), r->n);  // NULL (server-allocated) outputs skipped
    r->bytes = request_bytes(*h, r->n, out_bytes);
    if (r->bytes > s->cfg.mem_budget_bytes)
      fail(PYC_E_NOMEM, "request needs " + std::to_string(r->bytes) +
                            " bytes, more than the whole memory budget");
    r->res.t_submit_ns = now_ns();
    r->deadline_ns = req->deadline_us > 0 ? r->res.t_submit_ns + req->deadline_us * 1000 : 0;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop) fail(PYC_E_BUSY, "server is shutting down");
      if ((int64_t)s->queue.size() >= s->cfg.max_queue) fail(PYC_E_BUSY, "queue full");
      r->id = s->next_id++;
      *id = r->id;
      s->queue.push_back(r.get());
      s->reqs[r->id] = std::move(r);
      ++s->stats.submitted;
    }
    ++s->nevents;
    s->cv_sched.notify_one();
  });
}

PYC_API pyc_status pyc_server_poll(pyc_server_t s, uint64_t id, pyc_result* res,
                                   int64_t timeout_us) {
  pyc_status status = PYC_OK;
  pyc_status g = guarded([&] {
    if (!s || !res) fail(PYC_E_ARG, "server and res must not be NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) fail(PYC_E_NOTFOUND, "unknown request id");
    SReq* r = it->second.get();
    auto done = [&] { return r->state == kDone || r->state == kFailed; };
    if (!done() && timeout_us > 0)
      s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
    if (!done()) {
      status = PYC_E_TIMEOUT;
      return;
    }
    *res = r->res;
  });
  return g != PYC_OK ? g : status;
}

PYC_API pyc_status pyc_server_release(pyc_server_t s, uint64_t id) {
  return guarded([&] {
    if (!s) fail(PYC_E_ARG, "server is NULL");
    {
      std::lock_guard<std::mutex> lk(s->mu);
      auto it = s->reqs.find(id);
      if (it == s->reqs.end()) fail(PYC_E_NOTFOUND, "unknown request id");
      SReq* r = it->second.get();
      if (r->state != kDone && r->state != kFailed) fail(PYC_E_BUSY, "request not finished");
      for (int64_t off : r->out_offs) s->arena.release(off);
      if (r->counted) s->admitted_bytes -= r->bytes;
      s->reqs.erase(it);
    }
    ++s->nevents;
    s->cv_sched.notify_one();
  });
}

PYC_API pyc_status pyc_server_get_stats(pyc_server_t s, pyc_server_stats* st) {
  return guarded([&] {
    if (!s || !st) fail(PYC_E_ARG, "server and stats must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    st->admitted_bytes = s->admitted_bytes;
    st->queued = (int64_t)s->queue.size();
    st->arena_in_use = s->arena.in_use();
  });
}

PYC_API void pyc_server_destroy(pyc_server_t s) {
  if (!s) return;
  log_event("server destroyed: %lld requests completed, %lld failed, %lld batches",
            (long long)s->stats.completed, (long long)s->stats.failed,
            (long long)s->stats.batches);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    int64_t t = now_ns();
    for (SReq* r : s->queue) finish_req(s, r, PYC_E_BUSY, t);
    s->queue.clear();
    for (SReq* r : s->admitted) finish_req(s, r, PYC_E_BUSY, t);
    s->admitted.clear();
  }
  ++s->nevents;
  s->cv_sched.notify_all();
  s->cv_done.notify_all();
  if (s->th.joinable()) s->th.join();
  if (s->host_exec) {  // every batch has been retired: the executor is idle
    {
      std::lock_guard<std::mutex> lk(s->exec_mu);
      s->exec_stop = true;
    }
    s->exec_cv.notify_all();
    if (s->exec_th.joinable()) s->exec_th.join();
    delete s;
    return;
  }
  try {
    const Driver& d = drv();
    d.cuCtxSetCurrent(s->ctx);
    for (CUstream st : s->streams) d.cuStreamSynchronize(st);
    for (auto& sl : s->slots) {
      d.cuMemFree(sl.dev);
      d.cuMemFreeHost(sl.host);
      d.cuEventDestroy(sl.ev);
    }
    d.cuMemFree(s->arena_mem);
    for (CUstream st : s->streams) d.cuStreamDestroy(st);
  } catch (...) {
  }
  delete s;
}

// ------------------------------------------------------------------ replay

namespace {

void replay_server(pyc_server* s, int64_t nreq, const pyc_request* reqs, const int64_t* arr,
                   pyc_result* results) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->track_finished = true;
    s->finished.clear();
  }
  std::vector<uint64_t> ids(nreq, 0);
  std::unordered_map<uint64_t, int64_t> index;
  const int64_t t0 = now_ns();
  int64_t next = 0, done = 0;
  // Submissions go in bursts, with finished requests collected and released in
  // between: a client that submitted everything before releasing anything would
  // hold the budget with finished requests and stall admission (with 50,000
  // requests due at once, about 34 ms of submissions).
  constexpr int kBurst = 64;
  while (done < nreq) {
    // submit what is due, up to a burst
    for (int burst = 0; burst < kBurst && next < nreq && (!arr || now_ns() >= t0 + arr[next]);
         ++burst) {
      uint64_t id;
      pyc_status st = pyc_server_submit(s, &reqs[next], &id);
      int64_t t_arr = arr ? t0 + arr[next] : t0;
      if (st != PYC_OK) {
        results[next] = pyc_result{};
        results[next].status = st;
        results[next].t_submit_ns = t_arr;
        results[next].t_done_ns = now_ns();
        ++done;
      } else {
        ids[next] = id;
        index[id] = next;
      }
      ++next;
    }
    // collect finished requests, release them
    std::vector<uint64_t> fin;
    {
      // spin (yielding) until something finishes or the next arrival is due; no
      // waiting while requests are due already
      const uint64_t f0 = s->nfinished.load();
      const bool due = next < nreq && (!arr || now_ns() >= t0 + arr[next]);
      const int64_t t_end = due ? 0 : std::min<int64_t>(now_ns() + 200000,
                                                       next < nreq && arr ? t0 + arr[next]
                                                                          : INT64_MAX);
      while (s->nfinished.load() == f0 && now_ns() < t_end) std::this_thread::yield();
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->finished.empty()) {
        fin.push_back(s->finished.front());
        s->finished.pop_front();
      }
    }
    if (!fin.empty()) {
      // copy results and release, all under one lock
      std::lock_guard<std::mutex> lk(s->mu);
      for (uint64_t id : fin) {
        auto it = index.find(id);
        auto rq = s->reqs.find(id);
        if (it == index.end() || rq == s->reqs.end()) continue;
        int64_t k = it->second;
        SReq* r = rq->second.get();
        results[k] = r->res;
        results[k].t_submit_ns = arr ? t0 + arr[k] : t0;  // latency from the arrival
        for (int64_t off : r->out_offs) s->arena.release(off);
        if (r->counted) s->admitted_bytes -= r->bytes;
        s->reqs.erase(rq);
        index.erase(it);
        ++done;
      }
      ++s->nevents;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->track_finished = false;
  s->finished.clear();
}

// The per-request baseline: each request launched alone, as it arrives, with
// the single-launch kernels on one stream; no batching.
void replay_direct(pyc_server* s, int64_t nreq, const pyc_request* reqs, const int64_t* arr,
                   pyc_result* results) {
  const Driver& d = drv();
  CUstream st = s->streams[0];
  const int kEvents = 4096;
  struct Out {
    int64_t k;
    std::vector<int64_t> offs;
    void* out = nullptr;  // first server-allocated output
    CUdeviceptr val = 0;
  };
  // the replay's events, result buffer and the arena blocks of launched
  // requests go back however the replay ends (an error included)
  struct Held {
    pyc_server* s;
    CUstream st;
    std::vector<CUevent> evs;
    CUdeviceptr vals = 0;
    std::deque<Out> pending;  // launched, in stream order
    ~Held() {
      const Driver& dd = drv();
      dd.cuStreamSynchronize(st);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Out& o : pending)
          for (int64_t off : o.offs) s->arena.release(off);
      }
      for (CUevent e : evs)
        if (e) dd.cuEventDestroy(e);
      if (vals) dd.cuMemFree(vals);
    }
  } held{s, st, std::vector<CUevent>(kEvents, nullptr)};
  std::vector<CUevent>& evs = held.evs;
  std::deque<Out>& pending = held.pending;
  for (auto& e : evs) PYC_CU(d.cuEventCreate(&e, CU_EVENT_DISABLE_TIMING));
  CUdeviceptr& vals = held.vals;
  PYC_CU(d.cuMemAlloc(&vals, (size_t)kEvents * 16));
  std::vector<unsigned char> host_val(16);
  const int64_t t0 = now_ns();
  int64_t next = 0, done = 0;
  auto retire_front = [&](bool wait) {
    Out& o = pending.front();
    CUevent e = evs[o.k % kEvents];
    if (wait)
      PYC_CU(d.cuEventSynchronize(e));
    else if (d.cuEventQuery(e) != CUDA_SUCCESS)
      return false;
    pyc_result& r = results[o.k];
    r.t_done_ns = now_ns();
    r.status = PYC_OK;
    r.batch_size = 1;
    if (reqs[o.k].kind == PYC_REQ_REDUCE) {
      int ob = static_cast<pyc_reduce*>(reqs[o.k].handle)->gen.out_bytes;
      PYC_CU(d.cuMemcpyDtoH(r.value, o.val, (size_t)ob));
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int64_t off : o.offs) s->arena.release(off);
    }
    pending.pop_front();
    ++done;
    return true;
  };
  while (done < nreq) {
    if (next < nreq && (!arr || now_ns() >= t0 + arr[next])) {
      if ((int64_t)pending.size() >= kEvents - 1) {
        retire_front(true);
        continue;
      }
      const pyc_request& q = reqs[next];
      pyc_result& r = results[next];
      r = pyc_result{};
      r.t_submit_ns = arr ? t0 + arr[next] : t0;
      Out o;
      o.k = next;
      HandleBase* h = q.kind == PYC_REQ_MAP ? static_cast<HandleBase*>(static_cast<pyc_map*>(q.handle))
                                            : static_cast<pyc_reduce*>(q.handle);
      std::vector<void*> ptrs(q.ptrs, q.ptrs + h->spec.num_ptrs);
      bool ok = true;
      for (auto& p : h->spec.params)
        if (p.is_ptr && !ptrs[p.ptr_slot] && q.kind == PYC_REQ_MAP) {
          int64_t off;
          const int64_t eb = type_info(p.dtype).bytes;
          const int64_t shift = align_shift(*h, ptrs.data(), eb);
          std::lock_guard<std::mutex> lk(s->mu);
          if (!s->arena.alloc(q.n * eb + shift, &off)) {
            ok = false;
            break;
          }
          o.offs.push_back(off);
          ptrs[p.ptr_slot] = reinterpret_cast<void*>(s->arena_mem + off + shift);
          if (!o.out) o.out = ptrs[p.ptr_slot];
        }
      if (!ok) {  // arena full: wait for the oldest launch, then retry
        {
          std::lock_guard<std::mutex> lk(s->mu);
          for (int64_t off : o.offs) s->arena.release(off);
        }
        if (pending.empty()) fail(PYC_E_NOMEM, "arena too small for one request");
        retire_front(true);
        continue;
      }
      r.t_admit_ns = r.t_launch_ns = now_ns();
      if (q.kind == PYC_REQ_MAP) {
        pyc_map* h2 = static_cast<pyc_map*>(q.handle);
        launch_map(h2, choose_cfg(*h2, q.n, false), q.n, ptrs.data(), q.scalars, st);
        if (o.out) r.d_out = o.out;
      } else {
        pyc_reduce* h2 = static_cast<pyc_reduce*>(q.handle);
        o.val = vals + (next % kEvents) * 16;
        launch_reduce(h2, choose_cfg(*h2, q.n, true), q.n, ptrs.data(), q.scalars,
                      reinterpret_cast<void*>(o.val), st);
      }
      PYC_CU(d.cuEventRecord(evs[next % kEvents], st));
      pending.push_back(std::move(o));
      ++next;
      continue;
    }
    if (!pending.empty() && retire_front(false)) continue;
    if (!pending.empty() && (next >= nreq)) {
      retire_front(true);
      continue;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(2));
  }
}

}  // namespace

PYC_API pyc_status pyc_server_replay(pyc_server_t s, int64_t nreq, const pyc_request* reqs,
                                     const int64_t* arrival_ns, int mode, pyc_result* results) {
  return guarded([&] {
    if (!s || (nreq > 0 && (!reqs || !results))) fail(PYC_E_ARG, "NULL argument");
    if (nreq < 0) fail(PYC_E_ARG, "nreq must be >= 0");
    if (arrival_ns)
      for (int64_t k = 1; k < nreq; ++k)
        if (arrival_ns[k] < arrival_ns[k - 1]) fail(PYC_E_ARG, "arrival times must not decrease");
    if (s->host_exec && mode != PYC_REPLAY_SERVER)
      fail(PYC_E_ARG, "a host-executed server replays through the serving loop only");
    if (!s->host_exec) ensure_context();
    if (mode == PYC_REPLAY_SERVER)
      replay_server(s, nreq, reqs, arrival_ns, results);
    else if (mode == PYC_REPLAY_DIRECT)
      replay_direct(s, nreq, reqs, arrival_ns, results);
    else
      fail(PYC_E_ARG, "mode must be PYC_REPLAY_SERVER or PYC_REPLAY_DIRECT");
  });
}
