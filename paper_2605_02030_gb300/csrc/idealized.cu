// Idealized recall of candidate sets (Section 3.2): how many of a query's
// exact L_p top-K lie among the exact top-t under the base metric of the
// graph it is routed to, for every t up to t_max.  The paper uses this
// experiment to choose t; uhnsw_plan_t turns the curves into a t per p.
#include <cuda_runtime.h>

#include "launch.h"

namespace uhnsw_dev {

// The p of the base metric each query's graph is built under (same routing
// rule as the search kernels: p equal to a graph's base p selects it, else
// p <= cutoff selects the first graph).
__global__ void base_p_kernel(const float* p, int64_t nq, float gp0, float gp1, float cutoff,
                              float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = p[i];
    const int slot = v == gp0 ? 0 : v == gp1 ? 1 : (v <= cutoff ? 0 : 1);
    out[i] = slot == 0 ? gp0 : gp1;
  }
}

// One block per query: the position of each of the K true ids in the base
// top-T list, then counts[t] = number of true ids at positions <= t.
__global__ void recall_curve_kernel(const int64_t* ids_k, const int64_t* ids_t, int64_t nq, int K,
                                    int T, int32_t* counts) {
  extern __shared__ int32_t hist[];
  for (int64_t i = blockIdx.x; i < nq; i += gridDim.x) {
    for (int t = threadIdx.x; t < T; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const int64_t* bt = ids_t + i * T;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      const int64_t id = ids_k[i * K + j];
      if (id < 0) continue;
      for (int t = 0; t < T; ++t)
        if (bt[t] == id) {
          atomicAdd(&hist[t], 1);
          break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int t = 0; t < T; ++t) {
        acc += hist[t];
        counts[i * T + t] = acc;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_base_p(const float* p, int64_t nq, float gp0, float gp1, float cutoff,
                          float* out, cudaStream_t st) {
  int64_t blocks = (nq + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  base_p_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, nq, gp0, gp1, cutoff, out);
  return cudaGetLastError();
}

cudaError_t launch_recall_curve(const int64_t* ids_k, const int64_t* ids_t, int64_t nq, int K,
                                int T, int32_t* counts, cudaStream_t st) {
  int64_t blocks = nq < 4096 ? nq : 4096;
  recall_curve_kernel<<<(unsigned)blocks, 128, (size_t)T * 4, st>>>(ids_k, ids_t, nq, K, T,
                                                                    counts);
  return cudaGetLastError();
}

}  // namespace uhnsw_dev
