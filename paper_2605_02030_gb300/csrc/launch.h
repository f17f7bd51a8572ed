// Host-side launch interfaces of the device code (one translation unit per
// storage type keeps the build parallel).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "warp_kernels.cuh"

namespace uhnsw_dev {

// Team shape of the traversal distance: TEAM lanes per row, CPL 16-byte chunks
// per lane; the first shape whose TEAM * CPL covers the row is used.
struct TeamShape {
  int team, cpl;
};

// Returns false if no compiled shape covers rows of `chunks` 16-byte chunks.
bool pick_shape(uhnsw_dtype dt, int chunks, TeamShape* out);

// Warp-per-query kernel: TEAM lanes per row, CPL 16-byte chunks per lane,
// U rows per team loaded per round; 4 warps (queries) per block.
struct WarpShape {
  int team, cpl, u;
};
constexpr int kWarpsPerBlock = 4;
// The warp kernel's team shape for rows of `chunks` 16-byte chunks.
// team_pref 0: the narrowest compiled team that covers the row; else the
// first covering shape with exactly that many lanes.  `few`: the batch has
// fewer queries than the GPU has warp slots (WarpMinBlocks blocks of
// kWarpsPerBlock warps per SM).
bool pick_warp_shape(uhnsw_dtype dt, int chunks, int team_pref, bool few, WarpShape* out);
cudaError_t launch_wsearch(uhnsw_dtype dt, WarpShape sh, const QueryArgs& a, int grid,
                           size_t smem, cudaStream_t st);
int wsearch_occupancy(uhnsw_dtype dt, WarpShape sh, size_t smem);

// Launch the fused search kernel: one block per query (grid = nq) or, with
// a.queue_head set, `grid` persistent blocks.
cudaError_t launch_search(uhnsw_dtype dt, TeamShape sh, const QueryArgs& a, int grid, int block,
                          size_t smem, cudaStream_t st);

// Resident blocks per SM of the search kernel for this shape and smem size.
int search_occupancy(uhnsw_dtype dt, TeamShape sh, int block, size_t smem);

// Verification only, one warp per query (4 per block).
cudaError_t launch_wverify(const QueryArgs& a, cudaStream_t st);

// Beam buckets of a bucketed persistent search (ascending bounds).
struct BeamBuckets {
  int n;
  int bound[8];
};
// Query routes (graph x verification p form) and sort bins (bucket x route).
constexpr int kRoutes = 8;
constexpr int kBins = 8 * kRoutes;
// Bucket scratch: ws[2 kBins] counts and cursors, then info[16], then the order.
constexpr int kBucketInfo = 2 * kBins;
constexpr int kBucketOrder = kBucketInfo + 16;
// Groups the query indices by beam bucket, and by route inside a bucket, into
// `order` and writes {first slot, count} per bucket into info[2b], info[2b+1].
cudaError_t launch_bucketing(const QueryArgs& a, const BeamBuckets& bb, int32_t* ws,
                             int32_t* order, int32_t* info, cudaStream_t st);

cudaError_t launch_convert(const float* src, void* dst, uhnsw_dtype dt, int64_t count,
                           cudaStream_t st);
cudaError_t launch_inexact_count(const float* src, const void* dst, uhnsw_dtype dt, int64_t count,
                                 unsigned long long* bad, cudaStream_t st);

// Idealized-recall curves (idealized.cu).
cudaError_t launch_base_p(const float* p, int64_t nq, float gp0, float gp1, float cutoff,
                          float* out, cudaStream_t st);
cudaError_t launch_recall_curve(const int64_t* ids_k, const int64_t* ids_t, int64_t nq, int K,
                                int T, int32_t* counts, cudaStream_t st);
int exact_workspace_slices(int64_t n, int64_t nq, int k, int num_sms);
cudaError_t launch_exact(const float* base, int64_t n, int d, int d_pad, const float* q,
                         const float* p, int64_t nq, int k, int nslices, float* part_d,
                         int32_t* part_i, int64_t* out_ids, float* out_dist, cudaStream_t st);

// per-storage-type entry points (defined in search_<type>.cu)
cudaError_t launch_search_f32(TeamShape sh, const QueryArgs& a, int grid, int block, size_t smem,
                              cudaStream_t st);
cudaError_t launch_search_f16(TeamShape sh, const QueryArgs& a, int grid, int block, size_t smem,
                              cudaStream_t st);
cudaError_t launch_search_bf16(TeamShape sh, const QueryArgs& a, int grid, int block, size_t smem,
                               cudaStream_t st);
int occupancy_f32(TeamShape sh, int block, size_t smem);
cudaError_t launch_wsearch_f32(WarpShape sh, const QueryArgs& a, int grid, size_t smem,
                               cudaStream_t st);
cudaError_t launch_wsearch_f16(WarpShape sh, const QueryArgs& a, int grid, size_t smem,
                               cudaStream_t st);
cudaError_t launch_wsearch_bf16(WarpShape sh, const QueryArgs& a, int grid, size_t smem,
                                cudaStream_t st);
int wocc_f32(WarpShape sh, size_t smem);
int wocc_f16(WarpShape sh, size_t smem);
int wocc_bf16(WarpShape sh, size_t smem);
int occupancy_f16(TeamShape sh, int block, size_t smem);
int occupancy_bf16(TeamShape sh, int block, size_t smem);

}  // namespace uhnsw_dev
