// CUDA driver API, loaded at run time.
//
// The library is usable without a GPU for everything up to a launch
// (parsing, source generation, run-time compilation, caching), so it does not
// link libcuda: the driver is opened with dlopen on first use and every entry
// point is resolved by the exact (versioned) symbol its cuda.h declaration
// names.
#pragma once

#include <cuda.h>

#include <string>

namespace pyc {

struct Driver {
#define PYC_DRV_FN(name) decltype(&::name) name = nullptr;
#include "cudrv_fns.inc"
#undef PYC_DRV_FN
};

// Loaded driver table; throws Error(PYC_E_CUDA) if no driver is present.
const Driver& drv();

// Throws Error(PYC_E_CUDA) naming `what` if r is not CUDA_SUCCESS.
void check(CUresult r, const char* what);

// Make sure a context is current on this thread (the primary context of
// device $CUDA_DEVICE, default 0, when none is); returns it.
CUcontext ensure_context();

struct DeviceProps {
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  int max_threads_per_sm = 0;
  int l2_bytes = 0;
  std::string name;
};

// Properties of the device of the current context (cached per device).
const DeviceProps& current_device_props();

}  // namespace pyc

#define PYC_CU(call) ::pyc::check((call), #call)
