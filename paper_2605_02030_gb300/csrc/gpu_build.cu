// HNSW construction on the GPU (the index construction behind Section 2.2's
// graphs: G1 under L1, G2 under L2, G0.5 under the L0.5 sum of U-HNSW-E, and
// the L1.5 graph of a fixed-p comparison).
//
// The published HNSW insertion, applied to batches of nodes at once:
//   - nodes are inserted in id order; node 0 is the first entry point;
//   - a batch [s, e) searches the graph of nodes [0, s): one warp per new
//     node runs the greedy descent (beam 1) above the node's level, then at
//     each level from min(top, level) down to 0 a beam search of width
//     efConstruction whose entry set is the whole result of the level above,
//     and keeps at most M links chosen by the neighbour heuristic (a
//     candidate is kept only if strictly nearer to the new node than to every
//     link already kept);
//   - the reverse links go to a per-row incoming buffer; after the batch, one
//     warp per touched row appends them, or, past the row's cap (2M at layer
//     0, M above), re-selects the row with the heuristic over its old links
//     and the incoming ones, ordered by (distance, id);
//   - the entry point moves to the first node of a new top level.
// Nodes of one batch do not link to each other directly; batches grow with
// the graph (1/16 of the nodes already inserted, at most 65,536), so that a
// node's batch is a small part of the graph it searches.  Results depend on
// the batch schedule, not on thread timing: the incoming links of a row are
// sorted before they are used, so the graph is the same on every run.
//
// Layout on the device: FP32 rows [n][d_pad]; layer 0 as [n][2M] int32 and
// the upper levels as [rows][M] int32 with the row of (v, level l) at
// up_off[v] + l - 1 (the search index's layout), -1 padded.  Every loop is
// bounded; an index or capacity problem sets an error word that the host
// reads at the end.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "uhnsw.h"
#include "uhnsw_internal.h"
#include "warp_kernels.cuh"

namespace uhnsw_dev {
namespace {

constexpr int kBuildWarps = 4;   // warps (new nodes) per block
constexpr int kInCap = 128;      // incoming links buffered per row and batch

struct BuildArgs {
  const float* X;          // [n][d_pad]
  const int32_t* lv;       // [n] levels
  const int32_t* up_off;   // [n] first upper row of the node, -1 if none
  const int32_t* up_owner; // [rows] node of each upper row
  int32_t* ell0;           // [n][M0]
  int32_t* up_adj;         // [rows][M]
  int32_t* inc_cnt;        // [n + rows] incoming links of this batch
  int32_t* inc;            // [n + rows][kInCap]
  int32_t* touched;        // rows with incoming links, then their count at touched_n
  int32_t* touched_n;
  int32_t* err;            // [0] error code, [1] dropped incoming links
  int64_t n, rows;
  int32_t d_pad, metric, M, M0, efc, hb;
  float bp;                // the p of metric 5
};

// Sum of the base-metric terms of two rows by a team of 8 lanes (each lane
// 4 elements per 32), combined over the team by a butterfly: every lane of
// the team ends with the sum.  b may point to shared memory.  Metric 5 takes
// |d_j|^bp through the fast power intrinsic.
__device__ __forceinline__ float team_dist(const float* __restrict__ a, const float* b, int d_pad,
                                           int lt, int metric, float bp) {
  float acc = 0.f;
  for (int j = lt * 4; j < d_pad; j += 32) {
    const float4 x = *reinterpret_cast<const float4*>(a + j);
    const float4 y = *reinterpret_cast<const float4*>(b + j);
    const float t[4] = {x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float v = fabsf(t[e]);
      acc += metric == UHNSW_BASE_L1    ? v
             : metric == UHNSW_BASE_L05 ? sqrtf(v)
             : metric == UHNSW_BASE_L15 ? v * sqrtf(v)
             : metric == UHNSW_BASE_LP  ? __powf(v, bp)
                                        : v * v;
    }
  }
  acc += __shfl_xor_sync(kFull, acc, 1);
  acc += __shfl_xor_sync(kFull, acc, 2);
  acc += __shfl_xor_sync(kFull, acc, 4);
  return acc;
}

// Distances from the row `x` (shared or global) to rows ids[0..m) into out.
__device__ __forceinline__ void warp_dists(const BuildArgs& a, const float* x, const uint32_t* ids,
                                           float* out, int m) {
  const int lane = threadIdx.x & 31, team = lane >> 3, lt = lane & 7;
  for (int i0 = 0; i0 < m; i0 += 4) {
    const int i = min(i0 + team, m - 1);
    const int64_t v = chk_idx((int64_t)(ids[i] & kIdMask), a.n, 20, a.err);
    const float s = team_dist(a.X + v * a.d_pad, x, a.d_pad, lt, a.metric, a.bp);
    if (lt == 0 && i0 + team < m) out[i0 + team] = s;
  }
  __syncwarp();
}

// Neighbour heuristic over the ascending candidates (cd, ci)[0..nc): a
// candidate is kept only if its distance to the base point is below its
// distance to every candidate already kept; at most m kept, into sel.
__device__ int warp_select(const BuildArgs& a, const float* cd, const uint32_t* ci, int nc, int m,
                           int32_t* sel) {
  const int lane = threadIdx.x & 31, team = lane >> 3, lt = lane & 7;
  int r = 0;
  for (int i = 0; i < nc && r < m; ++i) {
    const int64_t c = chk_idx((int64_t)(ci[i] & kIdMask), a.n, 21, a.err);
    const float dc = cd[i];
    const float* xc = a.X + c * a.d_pad;
    bool keep = true;
    for (int j0 = 0; j0 < r && keep; j0 += 4) {
      const int j = min(j0 + team, r - 1);
      const int64_t s = chk_idx((int64_t)sel[j], a.n, 22, a.err);
      const float ds = team_dist(xc, a.X + s * a.d_pad, a.d_pad, lt, a.metric, a.bp);
      const bool bad = j0 + team < r && !(dc < ds);
      keep = !__any_sync(kFull, bad);
    }
    if (keep) {
      if (lane == 0) sel[r] = (int32_t)c;
      ++r;
    }
    __syncwarp();
  }
  return r;
}

__device__ __forceinline__ const int32_t* adj_row(const BuildArgs& a, int32_t v, int l, int* deg) {
  if (l == 0) {
    *deg = a.M0;
    return a.ell0 + chk_idx(v, a.n, 23, a.err) * a.M0;
  }
  *deg = a.M;
  const int32_t r = a.up_off[chk_idx(v, a.n, 24, a.err)];
  if (r < 0) {
    *deg = 0;
    return a.up_adj;
  }
  return a.up_adj + chk_idx((int64_t)r + l - 1, a.rows, 25, a.err) * a.M;
}

// Per-warp shared memory of the insertion kernel.
struct BuildSmem {
  int qv, wd0, wi0, wd1, wi1, hash, cd, ci, sd, si, sel, total;
  __host__ __device__ BuildSmem(int d_pad, int efc, int hb, int cm, int m0) {
    int o = 0;
    qv = o; o += align16(d_pad * 4);
    wd0 = o; o += align16(efc * 4);
    wi0 = o; o += align16(efc * 4);
    wd1 = o; o += align16(efc * 4);
    wi1 = o; o += align16(efc * 4);
    hash = o; o += align16((1 << hb) * 4);
    cd = o; o += align16(cm * 4);
    ci = o; o += align16(cm * 4);
    sd = o; o += align16(cm * 4);
    si = o; o += align16(cm * 4);
    sel = o; o += align16(m0 * 4);
    total = o;
  }
};

// SEARCH-LAYER at level l with beam ef from the entry set held in (*wd, *wi)
// [0..*nw) (ascending, flags clear); on return the result set is there,
// ascending, flags clear.  The two list buffers swap roles as the merge runs.
__device__ void warp_search_layer(const BuildArgs& a, const float* qv, int l, int ef,
                                  float** wd, uint32_t** wi, float** xd, uint32_t** xi, int* nw,
                                  int32_t* tab, float* cd, uint32_t* ci, float* sd, uint32_t* si) {
  const int lane = threadIdx.x & 31;
  const int H = 1 << a.hb;
  for (int j = lane; j < H; j += 32) tab[j] = kEmpty;
  __syncwarp();
  for (int j = lane; j < *nw; j += 32) hash_insert(tab, a.hb, (int32_t)((*wi)[j] & kIdMask), a.err);
  __syncwarp();
  int hcount = *nw, bn = *nw, first = 0;
  float* bdc = *wd;
  uint32_t* bic = *wi;
  float* bdn = *xd;
  uint32_t* bin = *xi;
  const int64_t max_steps = a.n + 16;
  for (int64_t step = 0; first < bn; ++step) {
    if (step >= max_steps) {
      if (lane == 0) set_error(a.err, UHNSW_ECAPACITY);
      break;
    }
    // the first unexpanded entry of W, marked expanded
    int par = -1;
    for (int b0 = first; b0 < bn && par < 0; b0 += 32) {
      const int pos = b0 + lane;
      const unsigned ball = __ballot_sync(kFull, pos < bn && !(bic[pos] & kExpanded));
      if (ball) {
        const int src = b0 + __ffs(ball) - 1;
        par = (int)(bic[src] & kIdMask);
        __syncwarp();
        if (lane == 0) bic[src] |= kExpanded;
      }
    }
    __syncwarp();
    if (par < 0) break;
    int deg = 0;
    const int32_t* row = adj_row(a, par, l, &deg);
    int m = 0;
    for (int b0 = 0; b0 < deg; b0 += 32) {
      const int j = b0 + lane;
      const int32_t v = j < deg ? row[j] : -1;
      const bool fresh = v >= 0 && v < a.n && hash_insert(tab, a.hb, v, a.err);
      warp_append(fresh, (uint32_t)v, ci, m, deg, a.err);
    }
    __syncwarp();
    if (m > 0) warp_dists(a, qv, ci, cd, m);
    const int mk = bn == ef ? warp_reject(cd, ci, m, bdc[bn - 1], (int32_t)(bic[bn - 1] & kIdMask))
                            : m;
    int nfirst = 0;
    const int nbn = warp_merge(bdc, bic, bn, cd, ci, mk, sd, si, bdn, bin, ef, &nfirst);
    {
      float* t0 = bdc;
      bdc = bdn;
      bdn = t0;
      uint32_t* t1 = bic;
      bic = bin;
      bin = t1;
    }
    hcount += m;
    if (hcount > (H >> 1)) {
      for (int j = lane; j < H; j += 32) tab[j] = kEmpty;
      __syncwarp();
      for (int j = lane; j < nbn; j += 32) hash_insert(tab, a.hb, (int32_t)(bic[j] & kIdMask), a.err);
      __syncwarp();
      hcount = nbn;
    }
    bn = nbn;
    first = nfirst;
  }
  for (int j = lane; j < bn; j += 32) bic[j] &= kIdMask;
  __syncwarp();
  *wd = bdc;
  *wi = bic;
  *xd = bdn;
  *xi = bin;
  *nw = bn;
}

// Queues the reverse link (row r <- u) for the batch's second phase.
__device__ __forceinline__ void push_incoming(const BuildArgs& a, int64_t r, int32_t u) {
  const int pos = atomicAdd(&a.inc_cnt[r], 1);
  if (pos == 0) {
    const int t = atomicAdd(a.touched_n, 1);
    a.touched[chk_idx(t, a.n + a.rows, 26, a.err)] = (int32_t)r;
  }
  if (pos < kInCap) a.inc[r * kInCap + pos] = u;
  else atomicAdd(&a.err[1], 1);  // dropped: the row had more incoming links than the buffer
}

// Phase 1 of a batch: one warp per new node u in [s, e).
__global__ void __launch_bounds__(kBuildWarps * 32) build_insert_kernel(BuildArgs a, int64_t s, int64_t e,
                                                                       int32_t ep, int32_t top) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cm = max(a.M0, 32);
  const BuildSmem L(a.d_pad, a.efc, a.hb, cm, a.M0);
  unsigned char* ws = smem + (size_t)warp * L.total;
  float* qv = reinterpret_cast<float*>(ws + L.qv);
  int32_t* tab = reinterpret_cast<int32_t*>(ws + L.hash);
  float* cd = reinterpret_cast<float*>(ws + L.cd);
  uint32_t* ci = reinterpret_cast<uint32_t*>(ws + L.ci);
  float* sd = reinterpret_cast<float*>(ws + L.sd);
  uint32_t* si = reinterpret_cast<uint32_t*>(ws + L.si);
  int32_t* sel = reinterpret_cast<int32_t*>(ws + L.sel);
  const int64_t nwarps = (int64_t)gridDim.x * kBuildWarps;
  for (int64_t u = s + (int64_t)blockIdx.x * kBuildWarps + warp; u < e; u += nwarps) {
    const float* xu = a.X + u * a.d_pad;
    for (int j = lane; j < a.d_pad; j += 32) qv[j] = xu[j];
    __syncwarp();
    float* wd = reinterpret_cast<float*>(ws + L.wd0);
    uint32_t* wi = reinterpret_cast<uint32_t*>(ws + L.wi0);
    float* xd = reinterpret_cast<float*>(ws + L.wd1);
    uint32_t* xi = reinterpret_cast<uint32_t*>(ws + L.wi1);
    if (lane == 0) ci[0] = (uint32_t)ep;
    __syncwarp();
    warp_dists(a, qv, ci, cd, 1);
    if (lane == 0) {
      wd[0] = cd[0];
      wi[0] = (uint32_t)ep;
    }
    __syncwarp();
    int nw = 1;
    const int lu = a.lv[u];
    for (int l = top; l > lu; --l)  // greedy descent: beam 1
      warp_search_layer(a, qv, l, 1, &wd, &wi, &xd, &xi, &nw, tab, cd, ci, sd, si);
    for (int l = min(top, lu); l >= 0; --l) {
      warp_search_layer(a, qv, l, a.efc, &wd, &wi, &xd, &xi, &nw, tab, cd, ci, sd, si);
      const int r = warp_select(a, wd, wi, nw, a.M, sel);
      int deg = 0;
      int32_t* row = const_cast<int32_t*>(adj_row(a, (int32_t)u, l, &deg));
      for (int j = lane; j < deg; j += 32) row[j] = j < r ? sel[j] : -1;
      for (int j = lane; j < r; j += 32) {
        const int32_t v = sel[j];
        const int32_t off = l == 0 ? 0 : a.up_off[v];
        if (off < 0) {            // a level-l link to a node below level l
          set_error(a.err, UHNSW_EINVAL);
          continue;
        }
        const int64_t rid = l == 0 ? (int64_t)v : a.n + (int64_t)off + l - 1;
        push_incoming(a, chk_idx(rid, a.n + a.rows, 29, a.err), (int32_t)u);
      }
      __syncwarp();
    }
  }
}

// Phase 2 of a batch: one warp per row that received links.
__global__ void __launch_bounds__(kBuildWarps * 32) build_reverse_kernel(BuildArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ucap = a.M0 + kInCap;
  // per warp: owner row, union ids / distances, sorted copy, selection
  const int per = align16(a.d_pad * 4) + 4 * align16(ucap * 4) + align16(a.M0 * 4);
  unsigned char* ws = smem + (size_t)warp * per;
  float* qv = reinterpret_cast<float*>(ws);
  uint32_t* ui = reinterpret_cast<uint32_t*>(ws + align16(a.d_pad * 4));
  float* ud = reinterpret_cast<float*>(ws + align16(a.d_pad * 4) + align16(ucap * 4));
  uint32_t* oi = reinterpret_cast<uint32_t*>(ws + align16(a.d_pad * 4) + 2 * align16(ucap * 4));
  float* od = reinterpret_cast<float*>(ws + align16(a.d_pad * 4) + 3 * align16(ucap * 4));
  int32_t* sel = reinterpret_cast<int32_t*>(ws + align16(a.d_pad * 4) + 4 * align16(ucap * 4));
  const int total = *a.touched_n;
  const int nwarps = gridDim.x * kBuildWarps;
  for (int t = blockIdx.x * kBuildWarps + warp; t < total; t += nwarps) {
    const int64_t r = a.touched[chk_idx(t, a.n + a.rows, 27, a.err)];
    const bool l0 = r < a.n;
    const int64_t v = l0 ? r : a.up_owner[chk_idx(r - a.n, a.rows, 28, a.err)];
    const int cap = l0 ? a.M0 : a.M;
    int32_t* row = l0 ? a.ell0 + r * a.M0 : a.up_adj + (r - a.n) * a.M;
    const int nin = min(a.inc_cnt[r], kInCap);
    // old links (compact, -1 after the last)
    int ne = 0;
    for (int b0 = 0; b0 < cap; b0 += 32) {
      const int j = b0 + lane;
      ne += __popc(__ballot_sync(kFull, j < cap && row[j] >= 0));
    }
    for (int j = lane; j < ne; j += 32) ui[j] = (uint32_t)row[j];
    // incoming links sorted by id, so that the row does not depend on the
    // order in which the warps of phase 1 pushed them
    for (int j = lane; j < nin; j += 32) {
      const int32_t x = a.inc[r * kInCap + j];
      int rank = 0;
      for (int k = 0; k < nin; ++k) rank += a.inc[r * kInCap + k] < x;
      ui[ne + rank] = (uint32_t)x;
    }
    __syncwarp();
    const int nu = ne + nin;
    if (nu <= cap) {
      for (int j = ne + lane; j < nu; j += 32) row[j] = (int32_t)ui[j];
    } else {
      const float* xv = a.X + v * a.d_pad;
      for (int j = lane; j < a.d_pad; j += 32) qv[j] = xv[j];
      __syncwarp();
      warp_dists(a, qv, ui, ud, nu);
      // order by (distance, id)
      for (int j = lane; j < nu; j += 32) {
        const float x = ud[j];
        const int32_t xi = (int32_t)ui[j];
        int rank = 0;
        for (int k = 0; k < nu; ++k) rank += pair_lt(ud[k], (int32_t)ui[k], x, xi);
        od[rank] = x;
        oi[rank] = (uint32_t)xi;
      }
      __syncwarp();
      const int rs = warp_select(a, od, oi, nu, cap, sel);
      for (int j = lane; j < cap; j += 32) row[j] = j < rs ? sel[j] : -1;
    }
    __syncwarp();
    if (lane == 0) a.inc_cnt[r] = 0;
    __syncwarp();
  }
}

int reverse_smem(int d_pad, int M0) {
  const int ucap = M0 + kInCap;
  return kBuildWarps * (align16(d_pad * 4) + 4 * align16(ucap * 4) + align16(M0 * 4));
}

}  // namespace
}  // namespace uhnsw_dev

extern "C" int uhnsw_build_graph_gpu(const float* base, int64_t n, int32_t d, int32_t metric,
                                     int32_t M, int32_t ef_construction, const int32_t* levels,
                                     uhnsw_built** out) {
  uhnsw_internal::clear_error();
  if (!out) return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph_gpu: out is NULL");
  *out = nullptr;
  if (metric < UHNSW_BASE_L1 || metric > UHNSW_BASE_L15)
    return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph_gpu: metric must be 1, 2, 3 or 4");
  return uhnsw_internal::build_graph_gpu(base, n, d, metric, 0.f, M, ef_construction, levels, out);
}

int uhnsw_internal::build_graph_gpu(const float* base, int64_t n, int32_t d, int32_t metric,
                                    float bp, int32_t M, int32_t ef_construction,
                                    const int32_t* levels, uhnsw_built** out) {
  using namespace uhnsw_dev;
  using uhnsw_internal::fail;
  if (!base || !levels || n < 1 || n > INT32_MAX / 2 || d < 1 || d > UHNSW_MAX_DIM)
    return fail(UHNSW_EINVAL, "uhnsw_build_graph_gpu: bad base/levels/n/d");
  if (M < 2 || 2 * M > UHNSW_MAX_DEGREE || ef_construction < 1 || ef_construction > 512)
    return fail(UHNSW_EINVAL, "uhnsw_build_graph_gpu: need 2 <= M <= %d, 1 <= efc <= 512",
                UHNSW_MAX_DEGREE / 2);
  std::vector<int32_t> up_off(n, -1), up_owner;
  int32_t top = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (levels[v] < 0 || levels[v] >= UHNSW_MAX_LEVELS)
      return fail(UHNSW_EINVAL, "uhnsw_build_graph_gpu: level of node %lld is %d", (long long)v,
                  levels[v]);
    if (levels[v] > 0) {
      up_off[v] = (int32_t)up_owner.size();
      for (int l = 0; l < levels[v]; ++l) up_owner.push_back((int32_t)v);
    }
  }
  const int64_t rows = (int64_t)up_owner.size();
  const int32_t M0 = 2 * M;
  const int32_t d_pad = (d + 7) / 8 * 8;
  const int32_t efc = ef_construction;
  int hb = 11;
  while ((1 << hb) < 4 * (efc + M0)) ++hb;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(UHNSW_ECUDA, "uhnsw_build_graph_gpu: %s", cudaGetErrorString(e));
  const BuildSmem L(d_pad, efc, hb, std::max(M0, 32), M0);
  const size_t smem1 = (size_t)L.total * kBuildWarps;
  const size_t smem2 = (size_t)reverse_smem(d_pad, M0);
  if (smem1 > 227 * 1024 || smem2 > 227 * 1024)
    return fail(UHNSW_ECAPACITY, "uhnsw_build_graph_gpu: %zu / %zu bytes of shared memory per block",
                smem1, smem2);

  // device buffers
  float* X = nullptr;
  int32_t *lv = nullptr, *doff = nullptr, *downer = nullptr, *ell0 = nullptr, *up_adj = nullptr;
  int32_t *inc_cnt = nullptr, *inc = nullptr, *touched = nullptr, *scal = nullptr;
  auto release = [&]() {
    cudaFree(X); cudaFree(lv); cudaFree(doff); cudaFree(downer); cudaFree(ell0);
    cudaFree(up_adj); cudaFree(inc_cnt); cudaFree(inc); cudaFree(touched); cudaFree(scal);
  };
  const int64_t nr = n + rows;
  e = cudaMalloc(&X, (size_t)n * d_pad * 4);
  if (e == cudaSuccess) e = cudaMalloc(&lv, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&doff, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&downer, std::max<int64_t>(rows, 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ell0, (size_t)n * M0 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&up_adj, (size_t)std::max<int64_t>(rows, 1) * M * 4);
  if (e == cudaSuccess) e = cudaMalloc(&inc_cnt, nr * 4);
  if (e == cudaSuccess) e = cudaMalloc(&inc, (size_t)nr * kInCap * 4);
  if (e == cudaSuccess) e = cudaMalloc(&touched, nr * 4);
  if (e == cudaSuccess) e = cudaMalloc(&scal, 64);
  if (e != cudaSuccess) {
    release();
    return fail(UHNSW_EOOM, "uhnsw_build_graph_gpu: device memory: %s", cudaGetErrorString(e));
  }
  e = cudaMemset(X, 0, (size_t)n * d_pad * 4);
  if (e == cudaSuccess)
    e = cudaMemcpy2D(X, (size_t)d_pad * 4, base, (size_t)d * 4, (size_t)d * 4, n,
                     cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(lv, levels, n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(doff, up_off.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && rows)
    e = cudaMemcpy(downer, up_owner.data(), rows * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ell0, 0xff, (size_t)n * M0 * 4);
  if (e == cudaSuccess) e = cudaMemset(up_adj, 0xff, (size_t)std::max<int64_t>(rows, 1) * M * 4);
  if (e == cudaSuccess) e = cudaMemset(inc_cnt, 0, nr * 4);
  if (e == cudaSuccess) e = cudaMemset(scal, 0, 64);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(build_insert_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(build_reverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem2);
  int occ1 = 0, occ2 = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, build_insert_kernel,
                                                      kBuildWarps * 32, smem1);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, build_reverse_kernel,
                                                      kBuildWarps * 32, smem2);
  if (e != cudaSuccess || occ1 < 1 || occ2 < 1) {
    release();
    return fail(UHNSW_ECUDA, "uhnsw_build_graph_gpu: setup: %s",
                e != cudaSuccess ? cudaGetErrorString(e) : "kernel does not fit");
  }

  BuildArgs a;
  a.X = X;
  a.lv = lv;
  a.up_off = doff;
  a.up_owner = downer;
  a.ell0 = ell0;
  a.up_adj = up_adj;
  a.inc_cnt = inc_cnt;
  a.inc = inc;
  a.touched = touched;
  a.touched_n = scal + 8;
  a.err = scal;
  a.n = n;
  a.rows = rows;
  a.d_pad = d_pad;
  a.metric = metric;
  a.bp = bp;
  a.M = M;
  a.M0 = M0;
  a.efc = efc;
  a.hb = hb;

  int32_t ep = 0, cur_top = levels[0];
  int64_t s = 1;
  while (s < n && e == cudaSuccess) {
    const int64_t b = std::max<int64_t>(1, std::min<int64_t>(65536, s / 16));
    const int64_t end = std::min(n, s + b);
    const int64_t warps = end - s;
    const int64_t grid1 = std::min<int64_t>((warps + kBuildWarps - 1) / kBuildWarps,
                                            (int64_t)occ1 * sms);
    build_insert_kernel<<<(unsigned)grid1, kBuildWarps * 32, smem1>>>(a, s, end, ep, cur_top);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    const int64_t grid2 = std::min<int64_t>((warps * M * 2 + kBuildWarps - 1) / kBuildWarps,
                                            (int64_t)occ2 * sms);
    build_reverse_kernel<<<(unsigned)std::max<int64_t>(grid2, 1), kBuildWarps * 32, smem2>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    e = cudaMemsetAsync(a.touched_n, 0, 4);
    for (int64_t u = s; u < end; ++u)
      if (levels[u] > cur_top) {
        cur_top = levels[u];
        ep = (int32_t)u;
      }
    s = end;
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t hs[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hs, scal, 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    release();
    return fail(UHNSW_ECUDA, "uhnsw_build_graph_gpu: %s", cudaGetErrorString(e));
  }
  if (hs[0] != 0) {
    release();
    return fail(hs[0], "uhnsw_build_graph_gpu: device error %d", hs[0]);
  }
  try {
    std::vector<int32_t> h0((size_t)n * M0), hu((size_t)std::max<int64_t>(rows, 1) * M);
    e = cudaMemcpy(h0.data(), ell0, h0.size() * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hu.data(), up_adj, hu.size() * 4, cudaMemcpyDeviceToHost);
    release();
    if (e != cudaSuccess)
      return fail(UHNSW_ECUDA, "uhnsw_build_graph_gpu: download: %s", cudaGetErrorString(e));
    *out = uhnsw_internal::make_built(n, M, M0, levels, ep, cur_top, h0.data(), up_off.data(),
                                      hu.data());
    if (!*out) return fail(UHNSW_EOOM, "uhnsw_build_graph_gpu: out of host memory");
  } catch (const std::bad_alloc&) {
    release();
    return fail(UHNSW_EOOM, "uhnsw_build_graph_gpu: out of host memory");
  }
  return UHNSW_OK;
}
