// Warp-per-query search kernel instantiations for float traversal rows.
#include "wsearch_inst.cuh"

namespace uhnsw_dev {

#define WLAUNCH_CALL(T, TEAM, CPL, U) wlaunch_one<T, TEAM, CPL, U>(a, grid, smem, st)
#define WOCC_CALL(T, TEAM, CPL, U) wocc_one<T, TEAM, CPL, U>(smem)

cudaError_t launch_wsearch_f32(WarpShape sh, const QueryArgs& a, int grid, size_t smem,
                               cudaStream_t st) {
#define FAIL_VALUE cudaErrorInvalidValue
  UHNSW_WSHAPE_SWITCH(float, sh, WLAUNCH_CALL);
#undef FAIL_VALUE
}

int wocc_f32(WarpShape sh, size_t smem) {
#define FAIL_VALUE 0
  UHNSW_WSHAPE_SWITCH(float, sh, WOCC_CALL);
#undef FAIL_VALUE
}

}  // namespace uhnsw_dev
