// Run-time loading of the CUDA driver (see cudrv.h).
#include "cudrv.h"

#include <dlfcn.h>

#include <cstdlib>
#include <map>
#include <mutex>

#include "common.h"

namespace pyc {

namespace {

Driver g_drv;
bool g_loaded = false;
std::string g_load_error;
std::once_flag g_once;

// Stringise a name after macro expansion: cuda.h maps e.g. cuMemAlloc to
// cuMemAlloc_v2, so this yields the exact exported symbol whose signature the
// header declares -- the binding a link against libcuda would make.  (A
// version-keyed lookup is not used: for some entry points, e.g.
// cuCtxGetDevice, the CUDA 13 table returns a newer form with an extra
// argument that the header does not remap.)
#define PYC_XSTR(x) PYC_STR(x)
#define PYC_STR(x) #x

// The driver's allocation entry points, called through these wrappers so that
// pyc_test_inject can make the next allocations fail as the driver does when
// memory runs out.
decltype(&::cuMemAlloc) g_real_mem_alloc = nullptr;
decltype(&::cuMemAllocHost) g_real_mem_alloc_host = nullptr;

CUresult CUDAAPI mem_alloc_or_injected(CUdeviceptr* p, size_t bytes) {
  if (take_injected(PYC_INJECT_ALLOC)) return CUDA_ERROR_OUT_OF_MEMORY;
  return g_real_mem_alloc(p, bytes);
}

CUresult CUDAAPI mem_alloc_host_or_injected(void** p, size_t bytes) {
  if (take_injected(PYC_INJECT_ALLOC)) return CUDA_ERROR_OUT_OF_MEMORY;
  return g_real_mem_alloc_host(p, bytes);
}

void load_driver() {
  void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_GLOBAL);
  if (!h) h = dlopen("libcuda.so", RTLD_NOW | RTLD_GLOBAL);
  if (!h) {
    g_load_error = "CUDA driver (libcuda.so.1) not found: no GPU driver on this machine";
    return;
  }
  std::string missing;
  auto resolve = [&](void** slot, const char* name) {
    *slot = dlsym(h, name);
    if (!*slot) missing += std::string(missing.empty() ? "" : ", ") + name;
  };
  Driver& d = g_drv;
#define PYC_DRV_FN(name) resolve(reinterpret_cast<void**>(&d.name), PYC_XSTR(name));
#include "cudrv_fns.inc"
#undef PYC_DRV_FN
  if (!missing.empty()) {
    g_load_error = "CUDA driver lacks entry points: " + missing;
    return;
  }
  g_real_mem_alloc = d.cuMemAlloc;
  g_real_mem_alloc_host = d.cuMemAllocHost;
  d.cuMemAlloc = &mem_alloc_or_injected;
  d.cuMemAllocHost = &mem_alloc_host_or_injected;
  CUresult r = d.cuInit(0);
  if (r != CUDA_SUCCESS) {
    const char* s = nullptr;
    d.cuGetErrorString(r, &s);
    g_load_error = std::string("cuInit failed: ") + (s ? s : "unknown error");
    return;
  }
  g_loaded = true;
}

}  // namespace

const Driver& drv() {
  std::call_once(g_once, load_driver);
  if (!g_loaded) fail(PYC_E_CUDA, g_load_error);
  return g_drv;
}

void check(CUresult r, const char* what) {
  if (r == CUDA_SUCCESS) return;
  const char* name = nullptr;
  const char* s = nullptr;
  if (g_loaded) {
    g_drv.cuGetErrorName(r, &name);
    g_drv.cuGetErrorString(r, &s);
  }
  pyc_status st = (r == CUDA_ERROR_OUT_OF_MEMORY) ? PYC_E_NOMEM : PYC_E_CUDA;
  fail(st, std::string(what) + " failed: " + (name ? name : "?") + " (" + (s ? s : "?") + ")");
}

CUcontext ensure_context() {
  const Driver& d = drv();
  CUcontext ctx = nullptr;
  PYC_CU(d.cuCtxGetCurrent(&ctx));
  if (ctx) return ctx;
  int ordinal = 0;
  if (const char* e = std::getenv("CUDA_DEVICE")) ordinal = std::atoi(e);
  CUdevice dev;
  PYC_CU(d.cuDeviceGet(&dev, ordinal));
  PYC_CU(d.cuDevicePrimaryCtxRetain(&ctx, dev));
  PYC_CU(d.cuCtxSetCurrent(ctx));
  return ctx;
}

const DeviceProps& current_device_props() {
  static std::mutex mu;
  static std::map<int, DeviceProps> cache;
  const Driver& d = drv();
  ensure_context();
  CUdevice dev;
  PYC_CU(d.cuCtxGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find((int)dev);
  if (it != cache.end()) return it->second;
  DeviceProps p;
  p.device = (int)dev;
  PYC_CU(d.cuDeviceGetAttribute(&p.sm_count, CU_DEVICE_ATTRIBUTE_MULTIPROCESSOR_COUNT, dev));
  PYC_CU(d.cuDeviceGetAttribute(&p.cc_major, CU_DEVICE_ATTRIBUTE_COMPUTE_CAPABILITY_MAJOR, dev));
  PYC_CU(d.cuDeviceGetAttribute(&p.cc_minor, CU_DEVICE_ATTRIBUTE_COMPUTE_CAPABILITY_MINOR, dev));
  PYC_CU(d.cuDeviceGetAttribute(&p.max_threads_per_sm,
                                CU_DEVICE_ATTRIBUTE_MAX_THREADS_PER_MULTIPROCESSOR, dev));
  PYC_CU(d.cuDeviceGetAttribute(&p.l2_bytes, CU_DEVICE_ATTRIBUTE_L2_CACHE_SIZE, dev));
  char name[256] = {0};
  PYC_CU(d.cuDeviceGetName(name, sizeof(name) - 1, dev));
  p.name = name;
  return cache.emplace((int)dev, p).first->second;
}

}  // namespace pyc
