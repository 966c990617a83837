// NVRTC driver and kernel cache (see kcache.h).
#include <chrono>
#include "kcache.h"

#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <future>
#include <sstream>
#include <thread>

#include "common.h"
#include "cudrv.h"

namespace pyc {

namespace {

// NVRTC entry points, resolved with dlopen so that the library loads on
// machines without the toolkit (compilation then fails with a clear error).
struct Nvrtc {
  decltype(&::nvrtcVersion) version = nullptr;
  decltype(&::nvrtcCreateProgram) create = nullptr;
  decltype(&::nvrtcCompileProgram) compile = nullptr;
  decltype(&::nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&::nvrtcGetProgramLog) log = nullptr;
  decltype(&::nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&::nvrtcGetCUBIN) cubin = nullptr;
  decltype(&::nvrtcDestroyProgram) destroy = nullptr;
  decltype(&::nvrtcGetErrorString) error_string = nullptr;
  int major = 0, minor = 0;
};

Nvrtc g_nv;
bool g_nv_ok = false;
std::string g_nv_err;
std::once_flag g_nv_once;

void load_nvrtc() {
  const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", nullptr};
  void* h = nullptr;
  for (int j = 0; names[j] && !h; ++j) h = dlopen(names[j], RTLD_NOW | RTLD_LOCAL);
  if (!h) {
    std::string home;
    if (const char* c = std::getenv("CUDA_HOME")) home = c;
    if (home.empty()) home = "/usr/local/cuda";
    h = dlopen((home + "/lib64/libnvrtc.so").c_str(), RTLD_NOW | RTLD_LOCAL);
  }
  if (!h) {
    g_nv_err = "NVRTC (libnvrtc.so.13) not found";
    return;
  }
  bool ok = true;
  auto sym = [&](auto& slot, const char* name) {
    slot = reinterpret_cast<std::remove_reference_t<decltype(slot)>>(dlsym(h, name));
    if (!slot) ok = false;
  };
  sym(g_nv.version, "nvrtcVersion");
  sym(g_nv.create, "nvrtcCreateProgram");
  sym(g_nv.compile, "nvrtcCompileProgram");
  sym(g_nv.log_size, "nvrtcGetProgramLogSize");
  sym(g_nv.log, "nvrtcGetProgramLog");
  sym(g_nv.cubin_size, "nvrtcGetCUBINSize");
  sym(g_nv.cubin, "nvrtcGetCUBIN");
  sym(g_nv.destroy, "nvrtcDestroyProgram");
  sym(g_nv.error_string, "nvrtcGetErrorString");
  if (!ok) {
    g_nv_err = "NVRTC library lacks required entry points";
    return;
  }
  g_nv.version(&g_nv.major, &g_nv.minor);
  g_nv_ok = true;
}

const Nvrtc& nvrtc() {
  std::call_once(g_nv_once, load_nvrtc);
  if (!g_nv_ok) fail(PYC_E_COMPILE, g_nv_err);
  return g_nv;
}

std::atomic<long long> g_compiled{0}, g_disk{0}, g_mem{0};

std::mutex g_cache_mu;
std::map<std::string, std::weak_ptr<Module>> g_mem_cache;
// keys being loaded or compiled right now: a second thread asking for the same
// key waits for the first one's result instead of compiling it again
std::map<std::string, std::shared_future<std::shared_ptr<Module>>> g_inflight;
// keep recently used modules alive even when no handle holds them; never
// destroyed, so no driver call runs during static destruction at exit
std::vector<std::shared_ptr<Module>>* g_recent = new std::vector<std::shared_ptr<Module>>();

const char* kArch = "sm_103a";
const char* kLibTag = "pyc-0.1-t2";

std::string read_file(const std::string& path, bool* ok) {
  std::ifstream f(path, std::ios::binary);
  if (!f) {
    *ok = false;
    return {};
  }
  std::ostringstream ss;
  ss << f.rdbuf();
  *ok = true;
  return ss.str();
}

void mkdirs(const std::string& path) {
  std::string cur;
  for (size_t j = 0; j < path.size(); ++j) {
    cur += path[j];
    if ((path[j] == '/' && j > 0) || j + 1 == path.size()) mkdir(cur.c_str(), 0755);
  }
}

// On-disk record: magic, key text length + text, number of units, then each
// unit's cubin length + bytes.  The full key text (source + options) is
// compared on read, so a hash collision can never return the wrong binary.
std::string pack_record(const std::string& key_text, const std::vector<std::string>& cubins) {
  std::string r = "PYCK2\n";
  r += std::to_string(key_text.size()) + "\n" + key_text;
  r += std::to_string(cubins.size()) + "\n";
  for (const auto& c : cubins) r += std::to_string(c.size()) + "\n" + c;
  return r;
}

bool unpack_record(const std::string& r, const std::string& key_text,
                   std::vector<std::string>* cubins) {
  if (r.compare(0, 6, "PYCK2\n") != 0) return false;
  size_t p = 6;
  auto number = [&](size_t* v) {
    const size_t nl = r.find('\n', p);
    if (nl == std::string::npos || nl == p || nl - p > 19) return false;
    for (size_t q = p; q < nl; ++q)
      if (r[q] < '0' || r[q] > '9') return false;
    *v = std::strtoull(r.c_str() + p, nullptr, 10);
    p = nl + 1;
    return true;
  };
  size_t klen = 0, count = 0;
  if (!number(&klen) || klen != key_text.size() || p + klen > r.size() ||
      r.compare(p, klen, key_text) != 0)
    return false;
  p += klen;
  if (!number(&count) || count == 0 || count > 1024) return false;
  std::vector<std::string> out;
  for (size_t u = 0; u < count; ++u) {
    size_t clen = 0;
    if (!number(&clen) || clen > r.size() - p) return false;
    out.push_back(r.substr(p, clen));
    p += clen;
  }
  if (p != r.size()) return false;
  *cubins = std::move(out);
  return true;
}

// The units of `source` (see kUnitMark): each unit's full text and its own part.
void split_units(const std::string& source, std::vector<std::string>* text,
                 std::vector<std::string>* own) {
  const std::string mark = kUnitMark;
  size_t p = source.find(mark);
  if (p == std::string::npos) {
    text->push_back(source);
    own->push_back(source);
    return;
  }
  const std::string common = source.substr(0, p);
  while (p != std::string::npos) {
    const size_t b = p + mark.size();
    const size_t e = source.find(mark, b);
    std::string mine = source.substr(b, e == std::string::npos ? std::string::npos : e - b);
    text->push_back(common + mine);
    own->push_back(std::move(mine));
    p = e;
  }
}

std::string compile_nvrtc(const std::string& source, bool fmad) {
  if (take_injected(PYC_INJECT_COMPILE))
    fail(PYC_E_COMPILE, "compilation failed: injected by pyc_test_inject (no compiler log)");
  const Nvrtc& nv = nvrtc();
  nvrtcProgram prog;
  nvrtcResult r = nv.create(&prog, source.c_str(), "pyc_kernel.cu", 0, nullptr, nullptr);
  if (r != NVRTC_SUCCESS) fail(PYC_E_COMPILE, std::string("nvrtcCreateProgram: ") + nv.error_string(r));
  std::string arch = std::string("-arch=") + kArch;
  const char* opts[] = {arch.c_str(), "-std=c++17", fmad ? "--fmad=true" : "--fmad=false",
                        "-lineinfo", "-DNDEBUG"};
  r = nv.compile(prog, 5, opts);
  size_t ls = 0;
  nv.log_size(prog, &ls);
  std::string log(ls, '\0');
  if (ls) nv.log(prog, &log[0]);
  if (r != NVRTC_SUCCESS) {
    nv.destroy(&prog);
    fail(PYC_E_COMPILE, std::string("run-time compilation failed (") + nv.error_string(r) +
                            "):\n" + log);
  }
  size_t cs = 0;
  nv.cubin_size(prog, &cs);
  std::string cubin(cs, '\0');
  nv.cubin(prog, &cubin[0]);
  nv.destroy(&prog);
  return cubin;
}

// Compile every unit, up to one thread per unit and hardware thread; the first
// failure (in unit order) is rethrown after all threads have finished.
std::vector<std::string> compile_units(const std::vector<std::string>& text, bool fmad) {
  const size_t n = text.size();
  std::vector<std::string> cubins(n);
  if (n == 1) {
    cubins[0] = compile_nvrtc(text[0], fmad);
    return cubins;
  }
  std::vector<std::exception_ptr> errs(n);
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t u; (u = next.fetch_add(1)) < n;) {
      try {
        cubins[u] = compile_nvrtc(text[u], fmad);
      } catch (...) {
        errs[u] = std::current_exception();
      }
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(n, std::min(hw, 16u));
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  for (auto& e : errs)
    if (e) std::rethrow_exception(e);
  return cubins;
}

}  // namespace

std::string digest(const std::string& data) {
  uint64_t h1 = 1469598103934665603ULL, h2 = 0x9E3779B97F4A7C15ULL;
  for (unsigned char c : data) {
    h1 = (h1 ^ c) * 1099511628211ULL;
    h2 = (h2 ^ c) * 0x100000001B3ULL + 0x632BE59BD9B4E019ULL;
    h2 ^= h2 >> 29;
  }
  char buf[40];
  std::snprintf(buf, sizeof(buf), "%016llx%016llx", (unsigned long long)h1,
                (unsigned long long)h2);
  return buf;
}

std::string cache_dir() {
  if (const char* d = std::getenv("PYC_CACHE_DIR")) return d;  // "" disables
  std::string base;
  if (const char* x = std::getenv("XDG_CACHE_HOME")) base = x;
  if (base.empty()) {
    if (const char* h = std::getenv("HOME")) base = std::string(h) + "/.cache";
  }
  if (base.empty()) return "";
  return base + "/pyc";
}

namespace {
std::shared_ptr<Module> load_or_compile(const std::string& key, const std::string& key_text,
                                        const std::string& source, bool fmad);
}  // namespace

std::shared_ptr<Module> get_module(const std::string& source, bool fmad) {
  int maj = 0, mnr = 0;
  {
    const Nvrtc& nv = nvrtc();
    maj = nv.major;
    mnr = nv.minor;
  }
  std::string key_text = std::string(kLibTag) + "|" + kArch + "|nvrtc" + std::to_string(maj) +
                         "." + std::to_string(mnr) + "|fmad=" + (fmad ? "1" : "0") + "\n" + source;
  std::string key = digest(key_text);
  std::promise<std::shared_ptr<Module>> promise;
  {
    std::unique_lock<std::mutex> lk(g_cache_mu);
    auto it = g_mem_cache.find(key);
    if (it != g_mem_cache.end()) {
      if (auto m = it->second.lock()) {
        ++g_mem;
        return m;
      }
    }
    auto fl = g_inflight.find(key);
    if (fl != g_inflight.end()) {
      std::shared_future<std::shared_ptr<Module>> pending = fl->second;
      lk.unlock();
      ++g_mem;
      return pending.get();  // the other thread's module, or its error rethrown
    }
    g_inflight.emplace(key, promise.get_future().share());
  }
  try {
    auto m = load_or_compile(key, key_text, source, fmad);
    {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      g_mem_cache[key] = m;
      g_recent->push_back(m);
      if (g_recent->size() > 64) g_recent->erase(g_recent->begin());
      g_inflight.erase(key);
    }
    promise.set_value(m);
    return m;
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      g_inflight.erase(key);
    }
    promise.set_exception(std::current_exception());
    throw;
  }
}

namespace {

// Disk-cache lookup, else NVRTC compilation (written back to the disk cache).
std::shared_ptr<Module> load_or_compile(const std::string& key, const std::string& key_text,
                                        const std::string& source, bool fmad) {
  std::string dir = cache_dir();
  std::string path = dir.empty() ? "" : dir + "/" + key + ".pyck";
  std::vector<std::string> text, own, cubins;
  split_units(source, &text, &own);
  bool have = false;
  if (!path.empty()) {
    bool ok = false;
    std::string rec = read_file(path, &ok);
    if (ok && unpack_record(rec, key_text, &cubins) && cubins.size() == text.size()) {
      have = true;
      ++g_disk;
      log_event("loaded %zu kernel units from the disk cache (%s)", cubins.size(), key.c_str());
    }
  }
  if (!have) {
    const auto t0 = std::chrono::steady_clock::now();
    cubins = compile_units(text, fmad);
    ++g_compiled;
    log_event("compiled %zu kernel units with NVRTC in %.0f ms (%s)", cubins.size(),
              std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                  .count(),
              key.c_str());
    if (!path.empty()) {
      mkdirs(dir);
      std::string tmp = path + ".tmp" + std::to_string(getpid());
      {
        std::ofstream f(tmp, std::ios::binary);
        std::string rec = pack_record(key_text, cubins);
        f.write(rec.data(), (std::streamsize)rec.size());
      }
      std::rename(tmp.c_str(), path.c_str());  // atomic publish
    }
  }
  return std::make_shared<Module>(std::move(cubins), std::move(own));
}

}  // namespace

CacheStats cache_stats() {
  CacheStats s;
  s.compiled = g_compiled;
  s.disk_hits = g_disk;
  s.mem_hits = g_mem;
  return s;
}

Module::Module(std::vector<std::string> cubins, std::vector<std::string> own_text)
    : cubins_(std::move(cubins)), own_(std::move(own_text)) {}

Module::~Module() {
  // Modules are unloaded only if the driver is present and the context lives;
  // errors at teardown are ignored on purpose.
  for (auto& kv : loaded_)
    for (CUmodule m : kv.second) {
      if (!m) continue;
      try {
        drv().cuModuleUnload(m);
      } catch (...) {
      }
    }
}

CUmodule Module::unit(CUcontext ctx, size_t u) {
  auto& mods = loaded_[ctx];
  if (mods.empty()) mods.assign(cubins_.size(), nullptr);
  if (!mods[u]) PYC_CU(drv().cuModuleLoadData(&mods[u], cubins_[u].data()));
  return mods[u];
}

std::vector<CUdeviceptr> Module::globals(const std::string& name, size_t* bytes) {
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(mu_);
  std::vector<CUdeviceptr> out;
  for (size_t u = 0; u < cubins_.size(); ++u) {
    CUdeviceptr p = 0;
    size_t b = 0;
    const CUresult r = drv().cuModuleGetGlobal(&p, &b, unit(ctx, u), name.c_str());
    if (r == CUDA_ERROR_NOT_FOUND) continue;
    PYC_CU(r);
    if (bytes) *bytes = b;
    out.push_back(p);
  }
  return out;
}

CUfunction Module::function(const std::string& name) {
  CUcontext ctx = ensure_context();
  std::lock_guard<std::mutex> lk(mu_);
  auto fk = std::make_pair(ctx, name);
  auto fit = funcs_.find(fk);
  if (fit != funcs_.end()) return fit->second;
  // the unit whose own text defines the kernel, else every unit in turn
  const std::string call = name + "(";
  std::vector<size_t> order;
  for (size_t u = 0; u < own_.size(); ++u)
    if (own_[u].find(call) != std::string::npos) order.push_back(u);
  for (size_t u = 0; u < cubins_.size(); ++u) order.push_back(u);
  CUresult last = CUDA_ERROR_NOT_FOUND;
  for (size_t u : order) {
    CUfunction f;
    last = drv().cuModuleGetFunction(&f, unit(ctx, u), name.c_str());
    if (last == CUDA_SUCCESS) {
      funcs_[fk] = f;
      return f;
    }
    if (last != CUDA_ERROR_NOT_FOUND) break;
  }
  PYC_CU(last);
  return nullptr;
}

}  // namespace pyc

PYC_API void pyc_cache_stats(int64_t* compiled, int64_t* disk_hits, int64_t* mem_hits) {
  pyc::CacheStats s = pyc::cache_stats();
  if (compiled) *compiled = s.compiled;
  if (disk_hits) *disk_hits = s.disk_hits;
  if (mem_hits) *mem_hits = s.mem_hits;
}
