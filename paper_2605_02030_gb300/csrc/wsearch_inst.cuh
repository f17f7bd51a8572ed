// Instantiation of the warp-per-query search kernel for one storage type.
#pragma once

#include "launch.h"

namespace uhnsw_dev {

template <typename T, int TEAM, int CPL, int U>
cudaError_t wlaunch_one(const QueryArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = uhnsw_wsearch_kernel<T, TEAM, CPL, U, kWarpsPerBlock>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int TEAM, int CPL, int U>
int wocc_one(size_t smem) {
  auto kern = uhnsw_wsearch_kernel<T, TEAM, CPL, U, kWarpsPerBlock>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kWarpsPerBlock * 32, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

// Calls CALL(T, TEAM, CPL, U) for the compiled warp shape.
#define UHNSW_WSHAPE_SWITCH(T, SH, CALL)                                     \
  do {                                                                       \
    const int key_ = (SH).team * 1000 + (SH).cpl * 10 + (SH).u;              \
    switch (key_) {                                                          \
      case 4032: return CALL(T, 4, 3, 2);                                    \
      case 8014: return CALL(T, 8, 1, 4);                                    \
      case 8022: return CALL(T, 8, 2, 2);                                    \
      case 8023: return CALL(T, 8, 2, 3);                                    \
      case 16022: return CALL(T, 16, 2, 2);                                  \
      case 16024: return CALL(T, 16, 2, 4);                                  \
      case 32022: return CALL(T, 32, 2, 2);                                  \
      case 32042: return CALL(T, 32, 4, 2);                                  \
      case 32081: return CALL(T, 32, 8, 1);                                  \
      case 32161: return CALL(T, 32, 16, 1);                                 \
      default: return FAIL_VALUE;                                            \
    }                                                                        \
  } while (0)

}  // namespace uhnsw_dev
