// ac_internal.h -- helpers shared by the translation units of the library
// (not part of the C ABI).
#pragma once

namespace acgb {

// Record the thread's last error message (read by ac_last_error) and
// return `code`.
int set_last_error(int code, const char *fmt, ...);

}  // namespace acgb
