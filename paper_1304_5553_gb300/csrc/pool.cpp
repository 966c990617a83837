// Memory pools (Sec. 3.2.6): blocks handed back by the program are retained and
// reused for later requests of the same size class instead of returning them to
// the driver, whose allocation calls are expensive.  One pool kind per memory:
// device (cuMemAlloc), page-locked host (cuMemAllocHost) and ordinary host memory.
//
// Reuse is stream-ordered: a block freed with stream s is reusable at once by a
// request on s (later work on s runs after the work that used the block), and by
// requests on other streams once an event recorded on s at the free has
// completed.  Retained blocks go back to the system on trim, on destroy, when
// the retained bytes pass max_retained, and when a system allocation fails (then
// the allocation is retried once).
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

namespace {

struct Block {
  void* ptr = nullptr;
  int64_t size = 0;
  CUstream stream = nullptr;
  CUevent event = nullptr;  // recorded on `stream` at the free (device / pinned)
};

}  // namespace

}  // namespace pyc

struct pyc_pool {
  pyc_pool_kind kind = PYC_POOL_DEVICE;
  pyc_pool_cfg cfg{};
  std::mutex mu;
  CUcontext ctx = nullptr;
  std::map<int64_t, std::vector<pyc::Block>> retained;  // by size class, oldest first
  std::unordered_map<void*, int64_t> live;
  std::vector<CUevent> spare_events;
  pyc_pool_stats st{};
};

namespace pyc {

namespace {

bool uses_cuda(const pyc_pool* p) { return p->kind != PYC_POOL_HOST; }

void* system_alloc(pyc_pool* p, int64_t bytes, bool* oom) {
  *oom = false;
  if (p->kind == PYC_POOL_HOST) {
    if (take_injected(PYC_INJECT_ALLOC)) {  // (device kinds: in the driver wrapper)
      *oom = true;
      return nullptr;
    }
    void* q = std::aligned_alloc(256, (size_t)((bytes + 255) / 256 * 256));
    *oom = q == nullptr;
    return q;
  }
  CUresult r;
  void* q = nullptr;
  if (p->kind == PYC_POOL_DEVICE) {
    CUdeviceptr d = 0;
    r = drv().cuMemAlloc(&d, (size_t)bytes);
    q = reinterpret_cast<void*>(d);
  } else {
    r = drv().cuMemAllocHost(&q, (size_t)bytes);
  }
  if (r == CUDA_ERROR_OUT_OF_MEMORY) {
    *oom = true;
    return nullptr;
  }
  check(r, p->kind == PYC_POOL_DEVICE ? "cuMemAlloc" : "cuMemAllocHost");
  return q;
}

void system_free(pyc_pool* p, void* q) {
  if (p->kind == PYC_POOL_HOST) {
    std::free(q);
  } else if (p->kind == PYC_POOL_DEVICE) {
    drv().cuMemFree(reinterpret_cast<CUdeviceptr>(q));
  } else {
    drv().cuMemFreeHost(q);
  }
}

// Give a retained block back to the system (after the work that used it).
void release(pyc_pool* p, Block& b) {
  if (b.event) {
    PYC_CU(drv().cuEventSynchronize(b.event));
    p->spare_events.push_back(b.event);
    b.event = nullptr;
  }
  system_free(p, b.ptr);
  p->st.system_bytes -= b.size;
  p->st.retained_bytes -= b.size;
  p->st.retained_blocks -= 1;
  p->st.system_frees += 1;
}

// Release retained blocks, the largest class first (fewest driver calls per
// byte) and the oldest block within a class, until `want` bytes are gone (or
// all, want < 0).
void release_retained(pyc_pool* p, int64_t want) {
  int64_t freed = 0;
  while ((want < 0 || freed < want) && p->st.retained_blocks > 0) {
    auto it = std::prev(p->retained.end());
    while (it->second.empty()) {
      if (it == p->retained.begin()) return;
      --it;
    }
    Block b = it->second.front();
    it->second.erase(it->second.begin());
    freed += b.size;
    release(p, b);
  }
}

bool reusable(const Block& b, CUstream s) {
  if (!b.event || b.stream == s) return true;
  CUresult r = drv().cuEventQuery(b.event);
  if (r == CUDA_SUCCESS) return true;
  if (r != CUDA_ERROR_NOT_READY) check(r, "cuEventQuery");
  return false;
}

}  // namespace

}  // namespace pyc

using namespace pyc;

PYC_API int64_t pyc_pool_block_size(int64_t bytes) {
  if (bytes <= 512) return 512;
  // 8 classes per octave: 2^e * (1 + k/8), so at most 1/8 of a block is unused
  int e = 63 - __builtin_clzll((unsigned long long)(bytes - 1));
  int64_t step = (int64_t)1 << (e - 3);
  return (bytes + step - 1) / step * step;
}

PYC_API pyc_status pyc_pool_create(pyc_pool_kind kind, const pyc_pool_cfg* cfg, pyc_pool_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (kind != PYC_POOL_DEVICE && kind != PYC_POOL_PINNED && kind != PYC_POOL_HOST)
      fail(PYC_E_ARG, "unknown pool kind");
    auto p = std::make_unique<pyc_pool>();
    p->kind = kind;
    if (cfg) p->cfg = *cfg;
    if (p->cfg.max_bytes < 0 || p->cfg.max_retained < 0) fail(PYC_E_ARG, "negative limit");
    if (uses_cuda(p.get())) p->ctx = ensure_context();
    *out = p.release();
  });
}

PYC_API pyc_status pyc_pool_alloc(pyc_pool_t p, int64_t bytes, pyc_stream_t stream, void** ptr) {
  return guarded([&] {
    if (!p || !ptr) fail(PYC_E_ARG, "pool or ptr is NULL");
    *ptr = nullptr;
    if (bytes <= 0) fail(PYC_E_ARG, "bytes must be > 0");
    const int64_t sz = pyc_pool_block_size(bytes);
    CUstream s = reinterpret_cast<CUstream>(stream);
    if (uses_cuda(p)) ensure_context();
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->retained.find(sz);
    if (it != p->retained.end()) {
      auto& v = it->second;
      for (size_t k = v.size(); k-- > 0;) {  // the most recently freed first
        if (!reusable(v[k], s)) continue;
        Block b = v[k];
        v.erase(v.begin() + (ptrdiff_t)k);
        if (b.event) p->spare_events.push_back(b.event);
        p->live.emplace(b.ptr, sz);
        p->st.retained_bytes -= sz;
        p->st.retained_blocks -= 1;
        p->st.live_bytes += sz;
        p->st.live_blocks += 1;
        p->st.hits += 1;
        *ptr = b.ptr;
        return;
      }
    }
    if (p->cfg.max_bytes && p->st.system_bytes + sz > p->cfg.max_bytes) {
      release_retained(p, p->st.system_bytes + sz - p->cfg.max_bytes);
      if (p->st.system_bytes + sz > p->cfg.max_bytes)
        fail(PYC_E_NOMEM, "pool limit of " + std::to_string(p->cfg.max_bytes) + " bytes reached");
    }
    bool oom = false;
    void* q = system_alloc(p, sz, &oom);
    if (oom) {  // give the retained blocks back and try once more
      release_retained(p, -1);
      q = system_alloc(p, sz, &oom);
      if (oom) fail(PYC_E_NOMEM, "out of memory allocating " + std::to_string(sz) + " bytes");
    }
    p->live.emplace(q, sz);
    p->st.system_bytes += sz;
    p->st.system_allocs += 1;
    p->st.live_bytes += sz;
    p->st.live_blocks += 1;
    p->st.misses += 1;
    *ptr = q;
  });
}

PYC_API pyc_status pyc_pool_free(pyc_pool_t p, void* ptr, pyc_stream_t stream) {
  return guarded([&] {
    if (!p) fail(PYC_E_ARG, "pool is NULL");
    if (!ptr) return;
    CUstream s = reinterpret_cast<CUstream>(stream);
    if (uses_cuda(p)) ensure_context();
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->live.find(ptr);
    if (it == p->live.end()) fail(PYC_E_ARG, "pointer was not allocated by this pool (or freed twice)");
    Block b;
    b.ptr = ptr;
    b.size = it->second;
    b.stream = s;
    p->live.erase(it);
    if (uses_cuda(p)) {
      if (p->spare_events.empty()) {
        CUevent e = nullptr;
        PYC_CU(drv().cuEventCreate(&e, CU_EVENT_DISABLE_TIMING));
        p->spare_events.push_back(e);
      }
      b.event = p->spare_events.back();
      p->spare_events.pop_back();
      PYC_CU(drv().cuEventRecord(b.event, s));
    }
    p->retained[b.size].push_back(b);
    p->st.live_bytes -= b.size;
    p->st.live_blocks -= 1;
    p->st.retained_bytes += b.size;
    p->st.retained_blocks += 1;
    if (p->cfg.max_retained && p->st.retained_bytes > p->cfg.max_retained)
      release_retained(p, p->st.retained_bytes - p->cfg.max_retained);
  });
}

PYC_API pyc_status pyc_pool_trim(pyc_pool_t p) {
  return guarded([&] {
    if (!p) fail(PYC_E_ARG, "pool is NULL");
    if (uses_cuda(p)) ensure_context();
    std::lock_guard<std::mutex> lk(p->mu);
    release_retained(p, -1);
  });
}

PYC_API pyc_status pyc_pool_get_stats(pyc_pool_t p, pyc_pool_stats* out) {
  return guarded([&] {
    if (!p || !out) fail(PYC_E_ARG, "pool or out is NULL");
    std::lock_guard<std::mutex> lk(p->mu);
    *out = p->st;
  });
}

PYC_API void pyc_pool_destroy(pyc_pool_t p) {
  if (!p) return;
  try {
    if (uses_cuda(p)) ensure_context();
    std::lock_guard<std::mutex> lk(p->mu);
    release_retained(p, -1);
    for (auto& kv : p->live) system_free(p, kv.first);
    for (CUevent e : p->spare_events) drv().cuEventDestroy(e);
  } catch (...) {
  }
  delete p;
}
