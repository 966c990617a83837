// Thread-local error text, element-type tables and the injected-failure
// counters of pyc_test_inject.
#include "common.h"

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>

namespace pyc {

namespace {
thread_local std::string t_last_error;
std::atomic<int64_t> g_inject[4];  // pending failures by pyc_inject_kind

int64_t take_one(std::atomic<int64_t>& c, bool all) {
  int64_t v = c.load();
  while (v > 0)
    if (c.compare_exchange_weak(v, all ? 0 : v - 1)) return all ? v : 1;
  return 0;
}
}  // namespace

bool take_injected(pyc_inject_kind k) {
  return k != PYC_INJECT_STALL_MS && (int)k >= 0 && (int)k < 4 &&
         take_one(g_inject[(int)k], false) > 0;
}

int64_t take_injected_stall_ms() { return take_one(g_inject[PYC_INJECT_STALL_MS], true); }

void set_last_error(const std::string& m) { t_last_error = m; }

void log_event(const char* fmt, ...) {
  static const bool on = [] {
    const char* e = std::getenv("PYC_LOG");
    return e && e[0] == '1';
  }();
  if (!on) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  std::fprintf(stderr, "pyc: %s\n", buf);
}
void clear_last_error() { t_last_error.clear(); }

const TypeInfo& type_info(pyc_dtype t) {
  static const TypeInfo table[] = {
      {PYC_F32, 4, "float"},
      {PYC_F64, 8, "double"},
      {PYC_BF16, 2, "pyc_bf16"},
      {PYC_F16, 2, "pyc_f16"},
      {PYC_I32, 4, "int"},
      {PYC_I64, 8, "long long"},
      {PYC_ARGMIN_F32, 16, "pyc_argf32"},
      {PYC_ARGMAX_F32, 16, "pyc_argf32"},
      {PYC_U8, 1, "unsigned char"},
      {PYC_I8, 1, "signed char"},
      {PYC_U32, 4, "unsigned int"},
      {PYC_U64, 8, "unsigned long long"},
      {PYC_I16, 2, "short"},
      {PYC_U16, 2, "unsigned short"},
  };
  int k = (int)t;
  if (k < 0 || k >= (int)(sizeof(table) / sizeof(table[0])))
    fail(PYC_E_ARG, "unknown dtype " + std::to_string(k));
  return table[k];
}

bool is_float_type(pyc_dtype t) {
  return t == PYC_F32 || t == PYC_F64 || t == PYC_BF16 || t == PYC_F16;
}

}  // namespace pyc

PYC_API const char* pyc_last_error(void) { return pyc::t_last_error.c_str(); }

PYC_API const char* pyc_version(void) { return "pyc 0.1 (sm_103a)"; }

PYC_API pyc_status pyc_test_inject(pyc_inject_kind what, int64_t value) {
  return pyc::guarded([&] {
    if ((int)what < 0 || (int)what > 3) pyc::fail(PYC_E_ARG, "unknown injection kind");
    if (value < 0) pyc::fail(PYC_E_ARG, "value must be >= 0");
    pyc::g_inject[(int)what].store(value);
  });
}
