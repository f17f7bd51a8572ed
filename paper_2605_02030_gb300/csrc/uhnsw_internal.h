// Internal declarations shared by the host files of the library.
#pragma once

#include <cstdarg>
#include <cstdint>

#include "uhnsw.h"

namespace uhnsw_internal {

void clear_error();
int fail(int code, const char* fmt, ...);

}  // namespace uhnsw_internal
