// Internal declarations shared by the host files of the library.
#pragma once

#include <cstdarg>
#include <cstdint>

#include "uhnsw.h"

namespace uhnsw_internal {

void clear_error();
int fail(int code, const char* fmt, ...);

// Bytes of search state one query holds while it runs (the per-query shared
// memory of the kernel `opts` selects, at beam ef and k results); a negative
// UHNSW_E* code on bad arguments.
int64_t query_state_bytes(const uhnsw_index* idx, int32_t ef, int32_t k,
                          const uhnsw_search_opts* opts);

}  // namespace uhnsw_internal
