// Internal helpers shared by the library's translation units: status
// exceptions, the thread-local last-error message, and element-type tables.
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>

#include "pyc.h"

#define PYC_API extern "C" __attribute__((visibility("default")))

namespace pyc {

// Thrown inside the library; converted to a pyc_status at the C boundary.
struct Error : std::runtime_error {
  pyc_status status;
  Error(pyc_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] inline void fail(pyc_status s, const std::string& m) { throw Error(s, m); }

void set_last_error(const std::string& m);

// One line on stderr ("pyc: ...") for the library's slow or stateful events --
// compilations, disk-cache loads, tuning results, segmented plans, server
// lifetimes -- when the environment variable PYC_LOG=1 was set at the first
// call; otherwise nothing.
void log_event(const char* fmt, ...) __attribute__((format(printf, 1, 2)));
void clear_last_error();

// Runs f(); maps exceptions to a status and records the message.
template <class F>
pyc_status guarded(F&& f) {
  try {
    clear_last_error();
    f();
    return PYC_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return PYC_E_NOMEM;
  } catch (const std::exception& e) {
    set_last_error(std::string("internal error: ") + e.what());
    return PYC_E_INTERNAL;
  }
}

// Element types that may appear in an argument list.
struct TypeInfo {
  pyc_dtype dtype;
  int bytes;
  const char* device_name;  // spelling used in generated source
};

const TypeInfo& type_info(pyc_dtype t);
bool is_float_type(pyc_dtype t);

// Failures injected by pyc_test_inject (host side only): take_injected
// consumes one pending failure of the kind and says whether there was one;
// take_injected_stall_ms consumes the pending scheduler stall (0 if none).
bool take_injected(pyc_inject_kind k);
int64_t take_injected_stall_ms();

}  // namespace pyc
