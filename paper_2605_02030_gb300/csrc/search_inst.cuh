// Instantiation of the search kernel for one storage type: the team shapes
// below cover rows of up to UHNSW_MAX_DIM elements.
#pragma once

#include "launch.h"

namespace uhnsw_dev {

template <typename T, int TEAM, int CPL, int BLOCK>
cudaError_t launch_one(const QueryArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = uhnsw_search_kernel<T, TEAM, CPL, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, BLOCK, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int TEAM, int CPL, int BLOCK>
int occupancy_one(size_t smem) {
  auto kern = uhnsw_search_kernel<T, TEAM, CPL, BLOCK>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem) != cudaSuccess) return 0;
  return nb;
}

// Calls F<TEAM, CPL, BLOCK>() for the compiled (shape, block) pair.
#define UHNSW_SHAPE_SWITCH(T, SH, BLK, CALL)                                              \
  do {                                                                                    \
    const int key_ = (SH).team * 1000 + (SH).cpl;                                         \
    if ((BLK) != 128) return FAIL_VALUE;                                                  \
    switch (key_) {                                                                       \
      case 8001: return CALL(T, 8, 1, 128);                                               \
      case 16001: return CALL(T, 16, 1, 128);                                             \
      case 16002: return CALL(T, 16, 2, 128);                                             \
      case 32001: return CALL(T, 32, 1, 128);                                             \
      case 32002: return CALL(T, 32, 2, 128);                                             \
      case 32004: return CALL(T, 32, 4, 128);                                             \
      case 32008: return CALL(T, 32, 8, 128);                                             \
      case 32016: return CALL(T, 32, 16, 128);                                            \
      default: return FAIL_VALUE;                                                         \
    }                                                                                     \
  } while (0)

}  // namespace uhnsw_dev
