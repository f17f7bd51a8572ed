// Search kernel instantiations for __half traversal rows.
#include "search_inst.cuh"

namespace uhnsw_dev {

#define LAUNCH_CALL(T, TEAM, CPL, B) launch_one<T, TEAM, CPL, B>(a, grid, smem, st)
#define OCC_CALL(T, TEAM, CPL, B) occupancy_one<T, TEAM, CPL, B>(smem)

cudaError_t launch_search_f16(TeamShape sh, const QueryArgs& a, int grid, int block, size_t smem,
                              cudaStream_t st) {
#define FAIL_VALUE cudaErrorInvalidValue
  UHNSW_SHAPE_SWITCH(__half, sh, block, LAUNCH_CALL);
#undef FAIL_VALUE
}

int occupancy_f16(TeamShape sh, int block, size_t smem) {
#define FAIL_VALUE 0
  UHNSW_SHAPE_SWITCH(__half, sh, block, OCC_CALL);
#undef FAIL_VALUE
}

}  // namespace uhnsw_dev
