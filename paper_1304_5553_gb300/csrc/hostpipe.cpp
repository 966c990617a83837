// Map over host arrays: pyc_map_launch_host.
//
// When every array is page-locked host memory mapped into the device's address
// space at the same address (unified addressing), the kernel runs directly on
// the host arrays: its loads and stores cross the chip-to-chip link with no
// staging copies (on a GB300 board faster than the copy engines: one
// host-to-device stream of kernel loads ~211 GB/s against ~197 GB/s, and loads
// and stores together ~336 GB/s).  Otherwise the arrays are streamed through
// device staging buffers in chunks.  Three
// streams overlap the work: chunk k's host-to-device copies, chunk k-1's kernel
// and chunk k-2's device-to-host copies run at the same time, ordered by events
// per staging slot.  Arrays the statement reads are copied in; arrays it writes
// are copied back (an array it may leave unwritten is also copied in, so the
// unwritten elements come back unchanged).  Only elementwise specs qualify:
// every array must be accessed as name[i] alone, because a chunk sees only its
// own slice.
#include <algorithm>
#include <cstring>

#include "cudrv.h"
#include "handles.h"

namespace pyc {

namespace {

constexpr int kStages = 3;
constexpr int64_t kPipeChunk = (int64_t)1 << 22;  // elements per chunk

}  // namespace

struct HostPipe {
  CUcontext ctx = nullptr;
  bool staged = false;  // staging buffers allocated
  CUstream s_in = nullptr, s_run = nullptr, s_out = nullptr;
  CUevent in_done[kStages] = {}, run_done[kStages] = {}, out_done[kStages] = {};
  std::vector<CUdeviceptr> buf;  // [stage * num_ptrs + slot]
  CUdeviceptr mem = 0;
  bool used[kStages] = {};

  void release() {
    const Driver& d = drv();
    for (int k = 0; k < kStages; ++k) {
      if (in_done[k]) d.cuEventDestroy(in_done[k]);
      if (run_done[k]) d.cuEventDestroy(run_done[k]);
      if (out_done[k]) d.cuEventDestroy(out_done[k]);
    }
    if (s_in) d.cuStreamDestroy(s_in);
    if (s_run) d.cuStreamDestroy(s_run);
    if (s_out) d.cuStreamDestroy(s_out);
    if (mem) d.cuMemFree(mem);
    *this = HostPipe();
  }
};

void free_host_pipe(pyc_map* h) {
  if (h->pipe) {
    try {
      h->pipe->release();
    } catch (...) {
    }
    delete h->pipe;
    h->pipe = nullptr;
  }
}

namespace {

HostPipe* get_pipe(pyc_map* h) {
  CUcontext ctx = ensure_context();
  if (h->pipe && h->pipe->ctx == ctx) return h->pipe;
  free_host_pipe(h);
  const Driver& d = drv();
  auto* p = new HostPipe();
  try {
    p->ctx = ctx;
    PYC_CU(d.cuStreamCreate(&p->s_in, CU_STREAM_NON_BLOCKING));
    PYC_CU(d.cuStreamCreate(&p->s_run, CU_STREAM_NON_BLOCKING));
    PYC_CU(d.cuStreamCreate(&p->s_out, CU_STREAM_NON_BLOCKING));
    for (int k = 0; k < kStages; ++k) {
      PYC_CU(d.cuEventCreate(&p->in_done[k], CU_EVENT_DISABLE_TIMING));
      PYC_CU(d.cuEventCreate(&p->run_done[k], CU_EVENT_DISABLE_TIMING));
      PYC_CU(d.cuEventCreate(&p->out_done[k], CU_EVENT_DISABLE_TIMING));
    }
  } catch (...) {
    p->release();
    delete p;
    throw;
  }
  h->pipe = p;
  return p;
}

// The staging buffers: three chunks of every array, allocated on first use.
void ensure_staging(const pyc_map* h, HostPipe* p) {
  if (p->staged) return;
  const ArgSpec& spec = h->spec;
  int64_t per_stage = 0;
  std::vector<int64_t> off(spec.num_ptrs, 0);
  for (auto& q : spec.params)
    if (q.is_ptr) {
      off[q.ptr_slot] = per_stage;
      per_stage += (kPipeChunk * type_info(q.dtype).bytes + 255) / 256 * 256;
    }
  PYC_CU(drv().cuMemAlloc(&p->mem, (size_t)std::max<int64_t>(per_stage * kStages, 256)));
  p->buf.assign((size_t)kStages * std::max(1, spec.num_ptrs), 0);
  for (int k = 0; k < kStages; ++k)
    for (int j = 0; j < spec.num_ptrs; ++j)
      p->buf[(size_t)k * spec.num_ptrs + j] = p->mem + k * per_stage + off[j];
  p->staged = true;
}

// True if [ptr, ptr + bytes) lies inside one allocation the driver knows that
// is mapped into the device's address space at the same address (page-locked
// host memory under unified addressing).  Pageable memory is not.
bool device_mapped(const void* ptr, int64_t bytes) {
  const Driver& d = drv();
  const CUdeviceptr a = reinterpret_cast<CUdeviceptr>(ptr);
  CUdeviceptr dp = 0, start = 0;
  size_t size = 0;
  if (d.cuPointerGetAttribute(&dp, CU_POINTER_ATTRIBUTE_DEVICE_POINTER, a) != CUDA_SUCCESS ||
      dp != a)
    return false;
  if (d.cuPointerGetAttribute(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, a) != CUDA_SUCCESS ||
      d.cuPointerGetAttribute(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, a) != CUDA_SUCCESS)
    return false;
  return a >= start && a + (CUdeviceptr)bytes <= start + (CUdeviceptr)size;
}

}  // namespace

}  // namespace pyc

using namespace pyc;

PYC_API pyc_status pyc_map_launch_host(pyc_map_t h, int64_t n, void* const* host_ptrs,
                                       const void* scalars) {
  return guarded([&] {
    if (!h) fail(PYC_E_ARG, "handle is NULL");
    if (n < 0) fail(PYC_E_ARG, "n must be >= 0");
    const ArgSpec& spec = h->spec;
    for (auto& q : spec.params)
      if (q.is_ptr && q.used && !q.lifted)
        fail(PYC_E_ARG, "array '" + q.name + "' is not accessed as " + q.name +
                            "[i] alone; host launches need an elementwise statement");
    if (n == 0) return;
    if (spec.num_ptrs > 0 && !host_ptrs) fail(PYC_E_ARG, "host_ptrs is NULL");
    for (auto& q : spec.params)
      if (q.is_ptr && q.used && !host_ptrs[q.ptr_slot])
        fail(PYC_E_ARG, "array '" + q.name + "' is NULL");
    check_overlap(spec, host_ptrs, n);
    std::lock_guard<std::mutex> lk(h->pipe_mu);
    HostPipe* p = get_pipe(h);
    const Driver& d = drv();
    bool direct = true;
    for (auto& q : spec.params)
      if (q.is_ptr && q.used)
        direct = direct && device_mapped(host_ptrs[q.ptr_slot], n * type_info(q.dtype).bytes);
    if (direct) {
      // one launch on the host arrays themselves
      launch_map(h, choose_cfg(*h, n, false), n, host_ptrs, scalars, p->s_run);
      PYC_CU(d.cuStreamSynchronize(p->s_run));
      return;
    }
    ensure_staging(h, p);
    const LaunchCfg cfg = choose_cfg(*h, kPipeChunk, false);
    const int np = spec.num_ptrs;
    std::vector<void*> dptrs(std::max(1, np), nullptr);
    for (int k = 0; k < kStages; ++k) p->used[k] = false;
    const int64_t nchunks = (n + kPipeChunk - 1) / kPipeChunk;
    for (int64_t c = 0; c < nchunks; ++c) {
      const int st = (int)(c % kStages);
      const int64_t lo = c * kPipeChunk, len = std::min(kPipeChunk, n - lo);
      // the stage's buffers are free once its previous chunk has been copied out
      if (p->used[st]) PYC_CU(d.cuStreamWaitEvent(p->s_in, p->out_done[st], 0));
      for (auto& q : spec.params) {
        if (!q.is_ptr) continue;
        const int64_t eb = type_info(q.dtype).bytes;
        CUdeviceptr dbuf = p->buf[(size_t)st * np + q.ptr_slot];
        dptrs[q.ptr_slot] = reinterpret_cast<void*>(dbuf);
        if (q.used && q.read)
          PYC_CU(d.cuMemcpyHtoDAsync(dbuf, static_cast<const char*>(host_ptrs[q.ptr_slot]) + lo * eb,
                                     (size_t)(len * eb), p->s_in));
      }
      PYC_CU(d.cuEventRecord(p->in_done[st], p->s_in));
      PYC_CU(d.cuStreamWaitEvent(p->s_run, p->in_done[st], 0));
      launch_map(h, cfg, len, dptrs.data(), scalars, p->s_run);
      PYC_CU(d.cuEventRecord(p->run_done[st], p->s_run));
      PYC_CU(d.cuStreamWaitEvent(p->s_out, p->run_done[st], 0));
      for (auto& q : spec.params) {
        if (!q.is_ptr || !q.used || !q.written) continue;
        const int64_t eb = type_info(q.dtype).bytes;
        PYC_CU(d.cuMemcpyDtoHAsync(static_cast<char*>(host_ptrs[q.ptr_slot]) + lo * eb,
                                   p->buf[(size_t)st * np + q.ptr_slot], (size_t)(len * eb),
                                   p->s_out));
      }
      PYC_CU(d.cuEventRecord(p->out_done[st], p->s_out));
      p->used[st] = true;
    }
    PYC_CU(d.cuStreamSynchronize(p->s_out));
    PYC_CU(d.cuStreamSynchronize(p->s_run));
  });
}
