// Per-thread error text of the C ABI (fptc_last_error_message), and the guard
// that keeps C++ exceptions from crossing it.
#pragma once

#include <exception>
#include <new>

#include "fptc.h"

namespace fptc {
void set_error(const char *fmt, ...) noexcept;
void clear_error() noexcept;

// Runs the body of a C ABI entry point: a C++ exception (host memory
// exhausted, a worker thread that could not start) becomes a status and a
// message instead of crossing the C boundary.
template <class F>
fptc_status guarded(F &&body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc &) {
    set_error("host memory exhausted");
    return FPTC_ERR_OUT_OF_MEMORY;
  } catch (const std::exception &e) {
    set_error("host error: %s", e.what());
    return FPTC_ERR_INVALID_ARGUMENT;
  } catch (...) {
    set_error("host error");
    return FPTC_ERR_INVALID_ARGUMENT;
  }
}
}  // namespace fptc
