// Per-thread error text of the C ABI (fptc_last_error_message).
#pragma once

namespace fptc {
void set_error(const char *fmt, ...);
void clear_error();
}  // namespace fptc
