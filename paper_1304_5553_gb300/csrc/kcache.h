// Run-time compilation and the kernel cache (Sec. 2, Fig. 1): the generated
// source is hashed; the in-memory table and then the on-disk cache are
// consulted; NVRTC compiles only on a miss.  A changed kernel therefore
// recompiles while every other kernel loads at once.
#pragma once

#include <cuda.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

namespace pyc {

// A compiled module (sm_103a CUBIN) and its per-context loaded copies.
class Module {
 public:
  explicit Module(std::string cubin) : cubin_(std::move(cubin)) {}
  ~Module();
  // Function `name` in the current context (loads the module on first use).
  CUfunction function(const std::string& name);
  // Device address and size of the module-scope variable `name` in the current
  // context (loads the module on first use).
  CUdeviceptr global(const std::string& name, size_t* bytes);
  const std::string& cubin() const { return cubin_; }

 private:
  std::string cubin_;
  std::mutex mu_;
  std::map<CUcontext, CUmodule> loaded_;
  std::map<std::pair<CUcontext, std::string>, CUfunction> funcs_;
};

// Compile `source` (or fetch it from a cache).  `fmad` selects FMA
// contraction.  Throws Error(PYC_E_COMPILE) with the NVRTC log on failure.
std::shared_ptr<Module> get_module(const std::string& source, bool fmad);

// Hex digest used as the cache key (128-bit, two independent FNV-1a lanes).
std::string digest(const std::string& data);

struct CacheStats {
  long long compiled = 0, disk_hits = 0, mem_hits = 0;
};
CacheStats cache_stats();

// Directory of the on-disk cache ("" when disabled).
std::string cache_dir();

}  // namespace pyc
