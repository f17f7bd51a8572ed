// Exhaustive L_p k-NN over the FP32 master copy: for every query, the k base
// rows with the smallest (S, id), S = sum_j |x_j - q_j|^p (the exact answer
// that recall is measured against, Section 4.1.2).
//
// Pass 1 (exact_slice_kernel): block (slice, query group) scores the rows of
// its slice against QB queries.  Rows are staged in shared memory in tiles of
// TR rows x DC dimensions (row stride DC+1 floats, so the 32 rows a warp
// reads sit in 32 different banks); each thread owns one row and QPT queries
// of the group.  After every tile, scores that beat a query's running k-th
// best are appended to that query's buffer and merged into its top-k list by
// one warp.  Pass 2 (exact_merge_kernel) merges the per-slice lists.
#include <cuda_runtime.h>

#include <climits>

#include "device_common.cuh"
#include "launch.h"

namespace uhnsw_dev {

constexpr int kExQB = 16;   // queries per block
constexpr int kExTR = 64;   // rows per tile
constexpr int kExDC = 64;   // dimensions per chunk
constexpr int kExBlock = 256;
constexpr int kExQPT = kExQB / (kExBlock / kExTR);  // queries per thread = 4

struct ExactSmem {
  int tile, qsm, topd, topi, bufd, bufi, scd, sci, nwd, nwi, total;
  __host__ __device__ ExactSmem(int k) {
    int o = 0;
    tile = o; o += align16(kExTR * (kExDC + 1) * 4);
    qsm = o; o += align16(kExQB * kExDC * 4);
    topd = o; o += align16(kExQB * k * 4);
    topi = o; o += align16(kExQB * k * 4);
    bufd = o; o += align16(kExQB * kExTR * 4);
    bufi = o; o += align16(kExQB * kExTR * 4);
    scd = o; o += align16((kExBlock / 32) * kExTR * 4);
    sci = o; o += align16((kExBlock / 32) * kExTR * 4);
    nwd = o; o += align16((kExBlock / 32) * k * 4);
    nwi = o; o += align16((kExBlock / 32) * k * 4);
    total = o;
  }
  __host__ __device__ static int align16(int x) { return (x + 15) & ~15; }
};

__device__ __forceinline__ float exact_term(float a, float p, int pm) {
  if (pm == kPOne) return a;
  if (pm == kPTwo) return a * a;
  return hw_ex2(p * hw_lg2(a));
}

// Warp-level merge of c unsorted entries (bd, bi) into the ascending list
// (td, ti) of *tn entries, capped at k.  sd/si (c entries) and nd/ni (k
// entries) are this warp's scratch.
__device__ __forceinline__ void warp_merge(float* td, int32_t* ti, int* tn, int k, const float* bd,
                                           const int32_t* bi, int c, float* sd, int32_t* si,
                                           float* nd, int32_t* ni) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < c; e += 32) {
    int r = 0;
    for (int j = 0; j < c; ++j) r += pair_lt(bd[j], bi[j], bd[e], bi[e]);
    sd[r] = bd[e];
    si[r] = bi[e];
  }
  __syncwarp();
  const int n = *tn;
  for (int e = lane; e < c; e += 32) {
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (pair_lt(td[mid], ti[mid], sd[e], si[e])) lo = mid + 1;
      else hi = mid;
    }
    const int pos = lo + e;
    if (pos < k) { nd[pos] = sd[e]; ni[pos] = si[e]; }
  }
  for (int j = lane; j < n; j += 32) {
    int lo = 0, hi = c;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (pair_lt(sd[mid], si[mid], td[j], ti[j])) lo = mid + 1;
      else hi = mid;
    }
    const int pos = lo + j;
    if (pos < k) { nd[pos] = td[j]; ni[pos] = ti[j]; }
  }
  __syncwarp();
  const int nn = min(k, n + c);
  for (int j = lane; j < nn; j += 32) { td[j] = nd[j]; ti[j] = ni[j]; }
  __syncwarp();
  if (lane == 0) *tn = nn;
  __syncwarp();
}

__global__ void __launch_bounds__(kExBlock) exact_slice_kernel(
    const float* __restrict__ base, int64_t n, int d_pad, const float* __restrict__ q, int d,
    const float* __restrict__ p, int64_t nq, int k, int64_t rows_per_slice, float* part_d,
    int32_t* part_i) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ExactSmem L(k);
  float* tile = reinterpret_cast<float*>(smem + L.tile);
  float* qsm = reinterpret_cast<float*>(smem + L.qsm);
  float* topd = reinterpret_cast<float*>(smem + L.topd);
  int32_t* topi = reinterpret_cast<int32_t*>(smem + L.topi);
  float* bufd = reinterpret_cast<float*>(smem + L.bufd);
  int32_t* bufi = reinterpret_cast<int32_t*>(smem + L.bufi);
  float* scd = reinterpret_cast<float*>(smem + L.scd);
  int32_t* sci = reinterpret_cast<int32_t*>(smem + L.sci);
  float* nwd = reinterpret_cast<float*>(smem + L.nwd);
  int32_t* nwi = reinterpret_cast<int32_t*>(smem + L.nwi);
  __shared__ int tn[kExQB];
  __shared__ int bc[kExQB];
  __shared__ float thr_d[kExQB];
  __shared__ int thr_i[kExQB];

  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t q0 = (int64_t)blockIdx.y * kExQB;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_slice;
  const int64_t r1 = min(n, r0 + rows_per_slice);
  const int myrow = tid % kExTR, qg = tid / kExTR;
  const float kInf = __int_as_float(0x7f800000);

  if (tid < kExQB) {
    tn[tid] = 0;
    bc[tid] = 0;
    thr_d[tid] = kInf;
    thr_i[tid] = INT_MAX;
  }
  float pq[kExQPT];
  int pm[kExQPT];
#pragma unroll
  for (int u = 0; u < kExQPT; ++u) {
    const int64_t qq = q0 + qg * kExQPT + u;
    pq[u] = qq < nq ? p[qq] : 1.0f;
    pm[u] = pmode_of(pq[u]);
    if (pm[u] != kPOne && pm[u] != kPTwo) pm[u] = kPGeneral;
  }
  __syncthreads();

  for (int64_t rt = r0; rt < r1; rt += kExTR) {
    float acc[kExQPT];
#pragma unroll
    for (int u = 0; u < kExQPT; ++u) acc[u] = 0.f;
    for (int c0 = 0; c0 < d_pad; c0 += kExDC) {
      const int dc = min(kExDC, d_pad - c0);
      // stage the tile (rows rt.., dims c0..c0+dc) and the query chunk
      for (int e = tid; e < kExTR * kExDC; e += kExBlock) {
        const int rr = e / kExDC, jj = e % kExDC;
        const int64_t row = rt + rr;
        tile[rr * (kExDC + 1) + jj] = (row < r1 && jj < dc) ? base[row * d_pad + c0 + jj] : 0.f;
      }
      for (int e = tid; e < kExQB * kExDC; e += kExBlock) {
        const int qq = e / kExDC, jj = e % kExDC;
        const int64_t qi = q0 + qq;
        const int j = c0 + jj;
        qsm[e] = (qi < nq && jj < dc && j < d) ? q[qi * d + j] : 0.f;
      }
      __syncthreads();
      const float* trow = tile + myrow * (kExDC + 1);
      const float* qrow = qsm + qg * kExQPT * kExDC;
      for (int jj = 0; jj < dc; ++jj) {
        const float x = trow[jj];
#pragma unroll
        for (int u = 0; u < kExQPT; ++u)
          acc[u] += exact_term(fabsf(x - qrow[u * kExDC + jj]), pq[u], pm[u]);
      }
      __syncthreads();
    }
    const int64_t row = rt + myrow;
#pragma unroll
    for (int u = 0; u < kExQPT; ++u) {
      const int qq = qg * kExQPT + u;
      if (row < r1 && q0 + qq < nq && pair_lt(acc[u], (int32_t)row, thr_d[qq], thr_i[qq])) {
        const int pos = atomicAdd(&bc[qq], 1);
        bufd[qq * kExTR + pos] = acc[u];
        bufi[qq * kExTR + pos] = (int32_t)row;
      }
    }
    __syncthreads();
    for (int qq = warp; qq < kExQB; qq += kExBlock / 32) {
      const int c = bc[qq];
      if (c == 0) continue;
      warp_merge(topd + qq * k, topi + qq * k, &tn[qq], k, bufd + qq * kExTR, bufi + qq * kExTR, c,
                 scd + warp * kExTR, sci + warp * kExTR, nwd + warp * k, nwi + warp * k);
      if ((tid & 31) == 0) {
        bc[qq] = 0;
        if (tn[qq] == k) {
          thr_d[qq] = topd[qq * k + k - 1];
          thr_i[qq] = topi[qq * k + k - 1];
        }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < kExQB * k; e += kExBlock) {
    const int qq = e / k, j = e % k;
    const int64_t qi = q0 + qq;
    if (qi >= nq) continue;
    const int64_t o = ((int64_t)blockIdx.x * nq + qi) * k + j;
    part_d[o] = j < tn[qq] ? topd[e] : kInf;
    part_i[o] = j < tn[qq] ? topi[e] : INT_MAX;
  }
}

// Merge of the per-slice lists of one query: survivors are the entries not
// after the smallest per-slice k-th entry; each survivor's rank among them is
// its output position.
__global__ void exact_merge_kernel(const float* part_d, const int32_t* part_i, int nslices,
                                   int64_t nq, int k, int64_t* out_ids, float* out_dist,
                                   const float* p) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* cd = reinterpret_cast<float*>(smem);
  int32_t* ci = reinterpret_cast<int32_t*>(smem + ((nslices * k * 4 + 15) & ~15));
  __shared__ int cnt;
  __shared__ float bd;
  __shared__ int bi;
  const int64_t qi = blockIdx.x;
  if (qi >= nq) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    cnt = 0;
    bd = __int_as_float(0x7f800000);
    bi = INT_MAX;
    for (int s = 0; s < nslices; ++s) {
      const int64_t o = ((int64_t)s * nq + qi) * k + (k - 1);
      if (pair_lt(part_d[o], part_i[o], bd, bi)) { bd = part_d[o]; bi = part_i[o]; }
    }
  }
  __syncthreads();
  const float td = bd;
  const int ti = bi;
  for (int e = tid; e < nslices * k; e += blockDim.x) {
    const int s = e / k, j = e % k;
    const int64_t o = ((int64_t)s * nq + qi) * k + j;
    const float x = part_d[o];
    const int32_t xi = part_i[o];
    if (xi != INT_MAX && !pair_lt(td, ti, x, xi)) {
      const int pos = atomicAdd(&cnt, 1);
      cd[pos] = x;
      ci[pos] = xi;
    }
  }
  __syncthreads();
  const int m = cnt;
  const double inv_p = 1.0 / (double)p[qi];
  for (int e = tid; e < m; e += blockDim.x) {
    int r = 0;
    for (int j = 0; j < m; ++j) r += pair_lt(cd[j], ci[j], cd[e], ci[e]);
    if (r < k) {
      out_ids[qi * k + r] = ci[e];
      out_dist[qi * k + r] = (float)pow((double)cd[e], inv_p);
    }
  }
  for (int j = m + tid; j < k; j += blockDim.x) {
    out_ids[qi * k + j] = -1;
    out_dist[qi * k + j] = __int_as_float(0x7f800000);
  }
}

int exact_workspace_slices(int64_t n, int64_t nq, int k, int num_sms) {
  const int64_t qb = (nq + kExQB - 1) / kExQB;
  int64_t s = (4 * (int64_t)num_sms + qb - 1) / qb;
  const int64_t cap = 8192 / k;
  if (s > cap) s = cap;
  const int64_t rows_min = kExTR;
  if (s > (n + rows_min - 1) / rows_min) s = (n + rows_min - 1) / rows_min;
  return (int)(s < 1 ? 1 : s);
}

cudaError_t launch_exact(const float* base, int64_t n, int d, int d_pad, const float* q,
                         const float* p, int64_t nq, int k, int nslices, float* part_d,
                         int32_t* part_i, int64_t* out_ids, float* out_dist, cudaStream_t st) {
  const ExactSmem L(k);
  cudaError_t e = cudaFuncSetAttribute(exact_slice_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return e;
  int64_t rows = (n + nslices - 1) / nslices;
  rows = (rows + kExTR - 1) / kExTR * kExTR;
  dim3 grid(nslices, (unsigned)((nq + kExQB - 1) / kExQB));
  exact_slice_kernel<<<grid, kExBlock, L.total, st>>>(base, n, d_pad, q, d, p, nq, k, rows, part_d,
                                                      part_i);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int msm = ((nslices * k * 4 + 15) & ~15) * 2;
  if (msm > 48 * 1024) {
    e = cudaFuncSetAttribute(exact_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, msm);
    if (e != cudaSuccess) return e;
  }
  exact_merge_kernel<<<(unsigned)nq, 128, msm, st>>>(part_d, part_i, nslices, nq, k, out_ids,
                                                     out_dist, p);
  return cudaGetLastError();
}

}  // namespace uhnsw_dev
