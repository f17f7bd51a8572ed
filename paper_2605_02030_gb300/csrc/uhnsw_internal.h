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

// A built graph (CSR per level) from padded adjacency tables: layer 0
// [n][M0], upper rows [rows][M] with the row of (v, l) at up_off[v] + l - 1,
// -1 after the last link.  nullptr when host memory runs out.
uhnsw_built* make_built(int64_t n, int32_t M, int32_t M0, const int32_t* levels, int32_t entry,
                        int32_t top, const int32_t* ell0, const int32_t* up_off,
                        const int32_t* up_adj);

// The base-metric code of L_p: 1-4 when p is one of their p (their own
// closed forms), else UHNSW_BASE_LP.
inline int32_t base_metric_of_p(float p) {
  return p == 1.f ? UHNSW_BASE_L1 : p == 2.f ? UHNSW_BASE_L2 : p == 0.5f ? UHNSW_BASE_L05
         : p == 1.5f ? UHNSW_BASE_L15 : UHNSW_BASE_LP;
}

// The GPU HNSW construction under base metric `metric`; bp is the p of
// UHNSW_BASE_LP (ignored for the other codes).  Arguments and errors as
// uhnsw_build_graph_gpu.
int build_graph_gpu(const float* base, int64_t n, int32_t d, int32_t metric, float bp, int32_t M,
                    int32_t ef_construction, const int32_t* levels, uhnsw_built** out);

}  // namespace uhnsw_internal
