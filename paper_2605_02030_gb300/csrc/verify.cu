// Verification-only kernel launch and the storage conversion kernel.
#include <cuda_runtime.h>

#include "launch.h"

namespace uhnsw_dev {

cudaError_t launch_wverify(const QueryArgs& a, cudaStream_t st) {
  const WVerifyLayout L(a.d_pad, a.k_max, a.vcap);
  constexpr int warps = 4;
  const size_t smem = (size_t)L.total * warps;
  auto kern = uhnsw_wverify_kernel<warps>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.nq + warps - 1) / warps);
  kern<<<grid, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

// FP32 master rows -> FP16 / BF16 traversal rows (round to nearest even).
__global__ void convert_kernel(const float* __restrict__ src, void* dst, int dt, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = src[i];
    if (dt == UHNSW_F16) reinterpret_cast<__half*>(dst)[i] = __float2half_rn(x);
    else reinterpret_cast<__nv_bfloat16*>(dst)[i] = __float2bfloat16_rn(x);
  }
}

// Counts the elements whose FP16 / BF16 copy differs from the FP32 value.
__global__ void inexact_kernel(const float* __restrict__ src, const void* dst, int dt,
                               int64_t count, unsigned long long* bad) {
  unsigned long long mine = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float back = dt == UHNSW_F16 ? __half2float(reinterpret_cast<const __half*>(dst)[i])
                                       : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(dst)[i]);
    mine += back != src[i];
  }
  if (mine) atomicAdd(bad, mine);
}

cudaError_t launch_inexact_count(const float* src, const void* dst, uhnsw_dtype dt, int64_t count,
                                 unsigned long long* bad, cudaStream_t st) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  inexact_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, (int)dt, count, bad);
  return cudaGetLastError();
}

cudaError_t launch_convert(const float* src, void* dst, uhnsw_dtype dt, int64_t count,
                           cudaStream_t st) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  convert_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, (int)dt, count);
  return cudaGetLastError();
}

bool pick_shape(uhnsw_dtype dt, int chunks, TeamShape* out) {
  static const TeamShape f32[] = {{8, 1}, {16, 2}, {32, 2}, {32, 4}, {32, 8}, {32, 16}};
  static const TeamShape f16[] = {{8, 1}, {16, 1}, {32, 1}, {32, 2}, {32, 4}, {32, 8}};
  const TeamShape* list = dt == UHNSW_F32 ? f32 : f16;
  const int cnt = 6;
  for (int i = 0; i < cnt; ++i)
    if (list[i].team * list[i].cpl >= chunks) {
      *out = list[i];
      return true;
    }
  return false;
}

// Beam ef' of a query exactly as the search kernels derive it.
__device__ __forceinline__ int query_beam(bool direct, int k, int ef, int t) {
  int tt = direct ? k : (t > 0 ? t : ef);
  if (tt < k) tt = k;
  return max(ef, tt);
}

__device__ __forceinline__ int beam_bucket(const BeamBuckets& bb, int efp) {
  for (int b = 0; b < bb.n; ++b)
    if (efp <= bb.bound[b]) return b;
  return bb.n - 1;  // beyond every bound: the query fails validation there
}

// Code route of a query: graph slot (with the same rule as the search
// kernels' route_query) and the p form of its verification (none for a
// direct query, then p = 0.5, p = 1.5, general p).  Queries of one route run
// the same instructions, so grouping them keeps the code that the warps of an
// SM execute at the same time small.
__device__ __forceinline__ int query_route(float p, float cutoff, float gp0, float gp1) {
  const int slot = p == gp0 ? 0 : p == gp1 ? 1 : (p <= cutoff ? 0 : 1);
  const bool direct = p == (slot == 0 ? gp0 : gp1);
  const int form = direct ? 0 : p == 0.5f ? 1 : p == 1.5f ? 2 : 3;
  return slot * 4 + form;
}

__device__ __forceinline__ int query_bin(const BeamBuckets& bb, const float* p, const int32_t* k,
                                         const int32_t* ef, const int32_t* tq, int64_t i,
                                         int k_max, int ef_default, int t, float cutoff, float gp0,
                                         float gp1) {
  const bool direct = p[i] == gp0 || p[i] == gp1;
  const int b = beam_bucket(bb, query_beam(direct, k ? k[i] : k_max, ef ? ef[i] : ef_default,
                                           tq ? tq[i] : t));
  return b * kRoutes + query_route(p[i], cutoff, gp0, gp1);
}

// Counting sort of the query indices by (beam bucket, route): counts, then
// slots.  ws[0..64): counts per bin, ws[64..128): cursors; info[2b] = first
// slot of bucket b, info[2b+1] = its count.
__global__ void bucket_count_kernel(const float* p, const int32_t* k, const int32_t* ef,
                                    const int32_t* tq, int64_t nq,
                                    int k_max, int ef_default, int t, float cutoff, float gp0,
                                    float gp1, BeamBuckets bb, int32_t* ws) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&ws[query_bin(bb, p, k, ef, tq, i, k_max, ef_default, t, cutoff, gp0, gp1)], 1);
}

__global__ void bucket_scatter_kernel(const float* p, const int32_t* k, const int32_t* ef,
                                      const int32_t* tq, int64_t nq, int k_max, int ef_default, int t, float cutoff,
                                      float gp0, float gp1, BeamBuckets bb, int32_t* ws,
                                      int32_t* order, int32_t* info) {
  if (blockIdx.x == 0 && threadIdx.x < bb.n) {
    const int b = threadIdx.x;
    int first = 0, cnt = 0;
    for (int j = 0; j < b * kRoutes; ++j) first += ws[j];
    for (int j = b * kRoutes; j < (b + 1) * kRoutes; ++j) cnt += ws[j];
    info[2 * b] = first;
    info[2 * b + 1] = cnt;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int bin = query_bin(bb, p, k, ef, tq, i, k_max, ef_default, t, cutoff, gp0, gp1);
    int base = 0;
    for (int j = 0; j < bin; ++j) base += ws[j];
    const int pos = atomicAdd(&ws[kBins + bin], 1);
    order[base + pos] = (int32_t)i;
  }
}

cudaError_t launch_bucketing(const QueryArgs& a, const BeamBuckets& bb, int32_t* ws,
                             int32_t* order, int32_t* info, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws, 0, 2 * kBins * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (a.nq + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  bucket_count_kernel<<<(unsigned)blocks, 256, 0, st>>>(a.p, a.k, a.ef, a.tq, a.nq, a.k_max,
                                                         a.ef_default, a.t, a.cutoff, a.gp[0],
                                                         a.gp[1], bb, ws);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bucket_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(a.p, a.k, a.ef, a.tq, a.nq, a.k_max,
                                                           a.ef_default, a.t, a.cutoff, a.gp[0],
                                                           a.gp[1], bb, ws, order, info);
  return cudaGetLastError();
}

bool pick_warp_shape(uhnsw_dtype dt, int chunks, int team_pref, bool few, WarpShape* out) {
  // The first covering shape of each list is the default.  For 128-dimension
  // FP16 rows (1M x 128, p ~ U(0.5, 2], ef 52, width 2, 10,000-query batches
  // on two streams) two rows per team and round measured 8 % faster than
  // three (1.37 vs 1.49 ms per batch) and one row 6 % slower.  A batch too
  // small to fill the GPU's warps (`few`) is bound by each query's own
  // latency: there three rows per round keep more loads in flight (serving
  // batches of 7 to 33 queries: p50 7 % and p99 up to 25 % lower than with
  // two rows).  Rows of 12 chunks (96 FP16 dimensions) take 4 lanes x 3
  // chunks, which leaves no lane on a zeroed chunk: 3.5 % faster than
  // 8 x 2 at 10M x 96, ef 512.  The shape never changes a result.
  static const WarpShape f32[] = {{8, 1, 4},  {8, 2, 2},  {16, 2, 4}, {32, 2, 2},
                                  {32, 4, 2}, {32, 8, 1}, {32, 16, 1}};
  static const WarpShape f16[] = {{8, 1, 4},  {4, 3, 2},  {8, 2, 2},  {16, 2, 2},
                                  {32, 2, 2}, {32, 4, 2}, {32, 8, 1}, {32, 16, 1}};
  static const WarpShape f16_few[] = {{8, 1, 4},  {4, 3, 2},  {8, 2, 3},  {16, 2, 2},
                                      {32, 2, 2}, {32, 4, 2}, {32, 8, 1}, {32, 16, 1}};
  const WarpShape* list = dt == UHNSW_F32 ? f32 : few ? f16_few : f16;
  const int cnt = dt == UHNSW_F32 ? (int)(sizeof(f32) / sizeof(f32[0]))
                                  : (int)(sizeof(f16) / sizeof(f16[0]));
  static_assert(sizeof(f16) == sizeof(f16_few), "the two 16-bit lists have one length");
  for (int i = 0; i < cnt; ++i)
    if (list[i].team * list[i].cpl >= chunks && (team_pref == 0 || list[i].team == team_pref)) {
      *out = list[i];
      return true;
    }
  return false;
}

cudaError_t launch_wsearch(uhnsw_dtype dt, WarpShape sh, const QueryArgs& a, int grid, size_t smem,
                           cudaStream_t st) {
  switch (dt) {
    case UHNSW_F32: return launch_wsearch_f32(sh, a, grid, smem, st);
    case UHNSW_F16: return launch_wsearch_f16(sh, a, grid, smem, st);
    case UHNSW_BF16: return launch_wsearch_bf16(sh, a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

int wsearch_occupancy(uhnsw_dtype dt, WarpShape sh, size_t smem) {
  switch (dt) {
    case UHNSW_F32: return wocc_f32(sh, smem);
    case UHNSW_F16: return wocc_f16(sh, smem);
    case UHNSW_BF16: return wocc_bf16(sh, smem);
  }
  return 0;
}

cudaError_t launch_search(uhnsw_dtype dt, TeamShape sh, const QueryArgs& a, int grid, int block,
                          size_t smem, cudaStream_t st) {
  switch (dt) {
    case UHNSW_F32: return launch_search_f32(sh, a, grid, block, smem, st);
    case UHNSW_F16: return launch_search_f16(sh, a, grid, block, smem, st);
    case UHNSW_BF16: return launch_search_bf16(sh, a, grid, block, smem, st);
  }
  return cudaErrorInvalidValue;
}

int search_occupancy(uhnsw_dtype dt, TeamShape sh, int block, size_t smem) {
  switch (dt) {
    case UHNSW_F32: return occupancy_f32(sh, block, smem);
    case UHNSW_F16: return occupancy_f16(sh, block, smem);
    case UHNSW_BF16: return occupancy_bf16(sh, block, smem);
  }
  return 0;
}

}  // namespace uhnsw_dev
