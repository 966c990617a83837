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

// Separates the units of a generated source: the text before the first mark
// is common to every unit, and each unit (common text + its own text) is an
// NVRTC program of its own, so the units of one source compile in parallel.
// A source without the mark is one unit.
constexpr const char* kUnitMark = "\n//@@pyc-unit\n";

// A compiled module: one sm_103a CUBIN per unit and the per-context loaded
// copies (a unit is loaded when a kernel it holds is first asked for).
class Module {
 public:
  // own_text[u]: unit u's own text, where its kernels' names appear as "name("
  Module(std::vector<std::string> cubins, std::vector<std::string> own_text);
  ~Module();
  // Function `name` in the current context.
  CUfunction function(const std::string& name);
  // Device address of the module-scope variable `name` in every unit that
  // defines it, in the current context (loads every unit); *bytes its size.
  std::vector<CUdeviceptr> globals(const std::string& name, size_t* bytes);
  size_t units() const { return cubins_.size(); }

 private:
  CUmodule unit(CUcontext ctx, size_t u);  // mu_ held
  std::vector<std::string> cubins_, own_;
  std::mutex mu_;
  std::map<CUcontext, std::vector<CUmodule>> loaded_;
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
