// The U-HNSW query kernel: routing, HNSW KnnSearch and L_p verification of
// one query per thread block (Section 3.1, Algorithm 1).
//
// One block owns one query at a time (a persistent block pulls the next query
// index from a device counter).  Per query:
//   1. route: p == 1 / p == 2 search G1 / G2 for the K nearest directly;
//      otherwise p <= cutoff -> G1 (L1), else G2 (squared L2);
//   2. greedy descent from the entry point through the upper levels (beam 1);
//   3. layer-0 best-first search with beam ef' (HNSW SEARCH-LAYER);
//   4. C = the first t beam entries (ascending base distance);
//   5. verification: exact (top-K by (S, id) over C, a candidate abandoned
//      once its partial sum exceeds the running K-th S) or Algorithm 1's
//      batches of kappa with the |R_new n R| / K >= tau stop;
//   6. distances S^(1/p), ascending (distance, id), padded with -1 / +inf.
//
// Layer 0 keeps the result set W as one sorted shared-memory list of ef'
// (distance, id) entries with an "expanded" bit.  With a strict total order
// this is the same search as HNSW's two heaps: every unexpanded member of W
// sits in the candidate heap, every other heap member is worse than W's
// furthest entry, so the heap's next pop is W's best unexpanded entry, and the
// heap search stops exactly when W has none left.  Expanding one entry per step
// (search_width 1) therefore reproduces the sequential HNSW order; its
// neighbours are merged into W in one step, which equals inserting them one by
// one into a bounded W (both keep the best ef' of the union).
//
// The visited set is an open-addressing table in shared memory.  When its load
// passes one half it is cleared and refilled with the ids currently in W.  A
// node forgotten this way can be evaluated again, but it cannot re-enter W: it
// was either rejected or evicted while W was full, and W's furthest entry only
// improves afterwards.  So W, the expansion order and the result are exactly
// those of an unbounded visited set; only extra distance evaluations are paid.
#pragma once

#include <climits>
#include <type_traits>

#include "device_common.cuh"

namespace uhnsw_dev {

struct GraphDev {
  const int32_t* ell0;   // [n][deg0] layer-0 links, -1 padded
  const int32_t* up_row; // [n] first upper-level row of the node, -1 if it is only on layer 0
  const int32_t* up_adj; // [rows][deg], -1 padded; row of (v, level l) = up_row[v] + l - 1
  int32_t up_rows;
  int32_t entry;
  int32_t top_level;
  int32_t deg0;
  int32_t deg;
};

struct QueryArgs {
  const float* base32;  // FP32 master copy [n][d_pad]
  const void* trav;     // traversal copy [n][d_pad] in the kernel's element type
  int64_t n;
  int32_t d, d_pad;
  GraphDev g[2];        // graph slots: G1 (L1) and G2 (squared L2), or G0.5 and G1
  int32_t gmetric[2];   // base metric of each slot (uhnsw_base_metric)
  float gp[2];          // the p of each slot's base metric
  const float* q;       // [nq][d]
  const float* p;       // [nq]
  const int32_t* k;     // [nq] or null (k_max)
  const int32_t* ef;    // [nq] or null (ef_default)
  int64_t nq;
  int32_t k_max, ef_default, ef_cap;
  int32_t t;            // 0 => ef
  int32_t kappa;        // 0 => k
  float tau, cutoff;
  const int32_t* tq;    // [nq] per-query t, or null (t)
  const float* tauq;    // [nq] per-query tau (0 => 0.92), or null (tau)
  int32_t mode;         // uhnsw_verify_mode
  int32_t width;        // beam entries expanded per step
  int32_t hash_bits;    // visited table holds 1 << hash_bits slots
  int32_t cmax;         // capacity of the per-step candidate buffers
  int32_t vcap;         // capacity of the candidate list C (verification-only launch)
  int64_t* out_ids;     // [nq][k_max]
  float* out_dist;      // [nq][k_max]
  int32_t* stats;       // [nq][UHNSW_NSTATS] or null
  int32_t* queue_head;  // persistent launch: next query slot; null => blockIdx.x only
  const int32_t* qorder;   // bucketed launch: query of each slot, grouped by beam bucket
  const int32_t* qbucket;  // bucketed launch: {first slot, slot count} of this bucket
  int32_t* err;         // sticky device error word
  const int32_t* cand;  // verification-only launch: [nq][cand_t]
  int32_t cand_t;
  int32_t trav_exact;   // 1: the traversal copy holds every FP32 value exactly
  int32_t stage_bytes;  // warp kernel: per-warp staging buffer for cp.async row copies
  int32_t sb;           // warp kernel: traversal rows staged per batch
  int32_t sv;           // warp kernel: FP32 rows staged per verification batch (multiple of 4)
  int32_t vgroups;      // warp kernels' verification: 32-dimension groups between two drop
                        // tests (>= 1); the block kernel tests after every group
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// Routing of a query (Algorithm 1, lines 1-5): the graph slot it searches,
// whether it is answered directly (p is that graph's own base p), the slot's
// base metric and its p.  p <= cutoff selects the first slot.
struct Route {
  int slot;
  bool direct;
  int metric;
  float bp;
};
__device__ __forceinline__ Route route_query(const QueryArgs& a, float p) {
  const int slot = p == a.gp[0] ? 0 : p == a.gp[1] ? 1 : (p <= a.cutoff ? 0 : 1);
  const float bp = a.gp[slot];
  return Route{slot, p == bp, a.gmetric[slot], bp};
}

// t and tau of query qi (per-query arrays when given).
__device__ __forceinline__ int query_t(const QueryArgs& a, int64_t qi) {
  return a.tq ? a.tq[qi] : a.t;
}
__device__ __forceinline__ float query_tau(const QueryArgs& a, int64_t qi) {
  if (!a.tauq) return a.tau;
  const float v = a.tauq[qi];
  return v != 0.f ? v : 0.92f;
}

// The distance a direct query returns: the base sum's root S^(1/bp).
__device__ __forceinline__ float base_root(int metric, float bp, float s) {
  return metric == UHNSW_BASE_L1    ? s
         : metric == UHNSW_BASE_L2  ? sqrtf(s)
         : metric == UHNSW_BASE_L05 ? (float)((double)s * (double)s)
         : metric == UHNSW_BASE_L15 ? (float)pow((double)s, 1.0 / 1.5)
                                    : (float)pow((double)s, 1.0 / (double)bp);
}

// Dynamic shared-memory carve-up (byte offsets), identical on host and device.
struct SmemLayout {
  int stage, qs, bd0, bi0, bd1, bi1, hash, cd, ci, sd, si, td0, ti0, td1, ti1, cv, total;
  __host__ __device__ SmemLayout(int d_pad, int ef_cap, int hash_bits, int cmax, int k_max,
                                 int vcap, int stage_bytes = 0) {
    int o = 0;
    qs = o; o += align16(d_pad * 4);
    bd0 = o; o += align16(ef_cap * 4);
    bi0 = o; o += align16(ef_cap * 4);
    bd1 = o; o += align16(ef_cap * 4);
    bi1 = o; o += align16(ef_cap * 4);
    // The visited table lives during the search, the staged verification rows
    // after it: they share one region.
    const int hash_bytes = align16((hash_bits > 0 ? (1 << hash_bits) : 0) * 4);
    hash = o;
    stage = o;
    o += hash_bytes > align16(stage_bytes) ? hash_bytes : align16(stage_bytes);
    cd = o; o += align16(cmax * 4);
    ci = o; o += align16(cmax * 4);
    sd = o; o += align16(cmax * 4);
    si = o; o += align16(cmax * 4);
    td0 = o; o += align16(k_max * 4);
    ti0 = o; o += align16(k_max * 4);
    td1 = o; o += align16(k_max * 4);
    ti1 = o; o += align16(k_max * 4);
    cv = o; o += align16(vcap * 4);
    total = o;
  }
};

struct BlockScalars {
  int qi;
  int bn;        // beam length
  int first;     // smallest unexpanded beam position
  int m;         // new candidates this step
  int npar;
  int hcount;    // visited-table insertions since the last reset
  int tn;        // verification list length
  int wm;        // finished candidates of a verification wave
  int overlap;
  int np;        // verification: candidates started
  int terms;     // verification: |x_j - q_j|^p terms accumulated
  float thr;
  float bestd;
  int besti;
  int par[8];
  float rd[32];
  int ri[32];
};

__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t r;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

// Block-wide minimum (d, id) over [0, m); result in s.bestd / s.besti.
template <int BLOCK>
__device__ __forceinline__ void block_argmin(const float* d, const uint32_t* id, int m,
                                             BlockScalars& s) {
  float bd = __int_as_float(0x7f800000);
  int32_t bi = INT_MAX;
  for (int i = threadIdx.x; i < m; i += BLOCK) {
    float x = d[i];
    int32_t xi = (int32_t)(id[i] & kIdMask);
    if (pair_lt(x, xi, bd, bi)) { bd = x; bi = xi; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float od = __shfl_xor_sync(kFull, bd, off);
    int32_t oi = __shfl_xor_sync(kFull, bi, off);
    if (pair_lt(od, oi, bd, bi)) { bd = od; bi = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { s.rd[warp] = bd; s.ri[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < BLOCK / 32; ++w)
      if (pair_lt(s.rd[w], s.ri[w], bd, bi)) { bd = s.rd[w]; bi = s.ri[w]; }
    s.bestd = bd;
    s.besti = bi;
  }
  __syncthreads();
}

// Base-metric distances of the m rows ids[0..m) to the query (whose slice this
// lane holds in qv), written to out[0..m).  TEAM lanes share one row, each
// loading CPL 16-byte chunks; U rows per team are in flight per round.  Every
// thread of the block calls it (the round count is block-uniform).
template <typename T, int TEAM, int CPL, int BLOCK, int METRIC>
__device__ __forceinline__ void dist_batch(const T* __restrict__ rows, int d_pad,
                                           const float (&qv)[CPL][Elems16<T>::n],
                                           const uint32_t* ids, float* out, int m, int64_t n,
                                           int32_t* err, float bp) {
  constexpr int VEC = Elems16<T>::n;
  constexpr int NT = BLOCK / TEAM;
  constexpr int U = 2;
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  const int R = d_pad / VEC;
  const int rounds = (m + NT * U - 1) / (NT * U);
  for (int r = 0; r < rounds; ++r) {
    uint4 buf[U][CPL];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = r * NT * U + u * NT + team;
      const bool ok = i < m;
      const int64_t id = ok ? chk_idx((int64_t)(ids[i] & kIdMask), n, 1, err) : 0;
      const uint4* row = reinterpret_cast<const uint4*>(rows + id * d_pad);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int ch = lane + c * TEAM;
        buf[u][c] = (ok && ch < R) ? ldg16(row + ch) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float acc = 0.0f;
      if constexpr (VEC == 8 && (METRIC == UHNSW_BASE_L1 || METRIC == UHNSW_BASE_L2)) {
        // 16-bit rows, L1 / L2: paired FP32 subtracts (and squares), even and
        // odd elements accumulated apart, then added
        uint64_t acc2 = 0;  // (+0.0f, +0.0f)
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          float x[VEC];
          unpack16<T>(buf[u][c], x);
#pragma unroll
          for (int e = 0; e < VEC / 2; ++e) {
            const uint64_t df = f2_sub(f2_pack(x[2 * e], x[2 * e + 1]),
                                       f2_pack(qv[c][2 * e], qv[c][2 * e + 1]));
            if (METRIC == UHNSW_BASE_L1) {
              float lo, hi;
              asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(df));
              a0 += fabsf(lo);
              a1 += fabsf(hi);
            } else {
              acc2 = f2_fma(df, df, acc2);
            }
          }
        }
        acc = METRIC == UHNSW_BASE_L1 ? a0 + a1 : f2_hsum(acc2);
      } else {
        // (braced: a loop pragma right after a bare `else` of an
        // `if constexpr` made the front end drop the statement after it)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          float x[VEC];
          unpack16<T>(buf[u][c], x);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float df = x[e] - qv[c][e];
            if (METRIC == UHNSW_BASE_L1) acc += fabsf(df);
            else if (METRIC == UHNSW_BASE_L05) acc += hw_sqrt(fabsf(df));
            else if (METRIC == UHNSW_BASE_L15) acc += fabsf(df) * hw_sqrt(fabsf(df));
            else if (METRIC == UHNSW_BASE_LP) acc += hw_ex2(bp * hw_lg2(fabsf(df)));
            else acc = fmaf(df, df, acc);
          }
        }
      }
#pragma unroll
      for (int off = TEAM / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off, TEAM);
      const int i = r * NT * U + u * NT + team;
      if (lane == 0 && i < m) out[i] = acc;
    }
  }
}

template <typename T, int TEAM, int CPL, int BLOCK>
__device__ __forceinline__ void dist_batch_metric(int metric, float bp, const T* rows, int d_pad,
                                                  const float (&qv)[CPL][Elems16<T>::n],
                                                  const uint32_t* ids, float* out, int m,
                                                  int64_t n, int32_t* err) {
  if (metric == UHNSW_BASE_L1) dist_batch<T, TEAM, CPL, BLOCK, 1>(rows, d_pad, qv, ids, out, m, n, err, bp);
  else if (metric == UHNSW_BASE_L2) dist_batch<T, TEAM, CPL, BLOCK, 2>(rows, d_pad, qv, ids, out, m, n, err, bp);
  else if (metric == UHNSW_BASE_L05) dist_batch<T, TEAM, CPL, BLOCK, 3>(rows, d_pad, qv, ids, out, m, n, err, bp);
  else if (metric == UHNSW_BASE_L15) dist_batch<T, TEAM, CPL, BLOCK, 4>(rows, d_pad, qv, ids, out, m, n, err, bp);
  else dist_batch<T, TEAM, CPL, BLOCK, 5>(rows, d_pad, qv, ids, out, m, n, err, bp);
}

// ---------------------------------------------------------------- verification
struct VerifyBufs {
  float* td[2];
  uint32_t* ti[2];
  float* wd;   // wave results
  uint32_t* wi;
  float* sd;   // merge scratch
  uint32_t* si;
};

// L_p sum of base row `id` against the query in shared memory, by a team of 8
// lanes (4 consecutive dimensions per lane, 32 per group).  After every group
// the team's partial sum is compared with thr: once it is larger the
// candidate is dropped (returns false).  Partial sums of non-negative FP32
// terms never decrease (the butterfly sum is monotone in every argument), so a
// dropped candidate cannot belong to the K smallest.
template <int PM>
__device__ __forceinline__ bool lp_sum_team(const float* __restrict__ base32, int d, int d_pad,
                                            const float* qs, float p, int32_t id, float thr,
                                            unsigned tmask, int lane8, float& S, int& groups) {
  const float* row = base32 + (int64_t)id * d_pad;
  float acc = 0.0f;
  const int G = (d + 31) >> 5;
  groups = 0;
  for (int g = 0; g < G; ++g) {
    const int j = g * 32 + lane8 * 4;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f), qq = x;
    if (j < d_pad) {
      x = __ldg(reinterpret_cast<const float4*>(row + j));
      qq = *reinterpret_cast<const float4*>(qs + j);
    }
    acc += pow_term<PM>(fabsf(x.x - qq.x), p);
    acc += pow_term<PM>(fabsf(x.y - qq.y), p);
    acc += pow_term<PM>(fabsf(x.z - qq.z), p);
    acc += pow_term<PM>(fabsf(x.w - qq.w), p);
    float tot = acc;
    tot += __shfl_xor_sync(tmask, tot, 1);
    tot += __shfl_xor_sync(tmask, tot, 2);
    tot += __shfl_xor_sync(tmask, tot, 4);
    groups = g + 1;
    if (tot > thr) return false;
    S = tot;
  }
  return true;
}

// One wave of verification: candidate C[w0 + team] per team of 8 lanes,
// finished ones appended to (wd, wi), dropped ones only counted.
template <int BLOCK, int PM>
__device__ __forceinline__ void verify_wave(const QueryArgs& a, const float* qs, float p,
                                            const uint32_t* C, int w0, int wend, float thr,
                                            const VerifyBufs& vb, BlockScalars& s) {
  const int team = threadIdx.x >> 3, lane8 = threadIdx.x & 7;
  const unsigned tmask = 0xffu << ((threadIdx.x & 31) & ~7);
  const int i = w0 + team;
  if (i < wend) {
    const int32_t id = (int32_t)chk_idx((int64_t)(C[i] & kIdMask), a.n, 2, a.err);
    float S = 0.f;
    int groups = 0;
    const bool done = lp_sum_team<PM>(a.base32, a.d, a.d_pad, qs, p, id, thr, tmask, lane8, S,
                                      groups);
    if (lane8 == 0) {
      atomicAdd(&s.np, 1);
      atomicAdd(&s.terms, min(groups * 32, a.d));
      if (done) {
        const int pos = (int)chk_idx(atomicAdd(&s.wm, 1), BLOCK / 8, 9, a.err);
        vb.wd[pos] = S;
        vb.wi[pos] = (uint32_t)id;
      }
    }
  }
  __syncthreads();
}

// Merge the wave's finished candidates into the running top-k list and
// refresh the drop threshold (the k-th smallest S, +inf while fewer).
template <int BLOCK>
__device__ __forceinline__ void verify_fold(int k, const VerifyBufs& vb, BlockScalars& s,
                                            int& cur) {
  const int tn = block_merge(vb.td[cur], vb.ti[cur], s.tn, vb.wd, vb.wi, s.wm, vb.sd, vb.si,
                             vb.td[cur ^ 1], vb.ti[cur ^ 1], k, nullptr);
  cur ^= 1;
  if (threadIdx.x == 0) {
    s.tn = tn;
    s.thr = tn == k ? vb.td[cur][k - 1] : __int_as_float(0x7f800000);
    s.wm = 0;
  }
  __syncthreads();
}

// Verification of the candidate list C[0..t) (ids, flag bit ignored) for one
// query whose vector is in shared memory.  Exact mode: top-k by (S, id) over
// all of C with the partial-sum drop.  Paper mode (Algorithm 1 lines 6-10):
// R = the first k of C; then batches of kappa; after each batch R_new = top-k
// of R u R', stop once (float)|R_new n R| / (float)k >= tau.  The result is
// left in (vb.td[cur], vb.ti[cur]) with s.tn entries.
template <int BLOCK, int PM>
__device__ void verify_run(const QueryArgs& a, const float* qs, float p, const uint32_t* C, int t,
                           int k, int kappa, float tau, bool exact, const VerifyBufs& vb,
                           BlockScalars& s, int& cur) {
  constexpr int NVT = BLOCK / 8;
  const float kInf = __int_as_float(0x7f800000);
  if (threadIdx.x == 0) {
    s.tn = 0;
    s.thr = kInf;
    s.wm = 0;
    s.np = 0;
    s.terms = 0;
  }
  __syncthreads();
  if (exact || a.mode != UHNSW_VERIFY_PAPER) {
    for (int w0 = 0; w0 < t; w0 += NVT) {
      verify_wave<BLOCK, PM>(a, qs, p, C, w0, min(w0 + NVT, t), s.thr, vb, s);
      verify_fold<BLOCK>(k, vb, s, cur);
    }
    return;
  }
  const int n0 = min(k, t);
  for (int w0 = 0; w0 < n0; w0 += NVT) {
    verify_wave<BLOCK, PM>(a, qs, p, C, w0, min(w0 + NVT, n0), kInf, vb, s);
    verify_fold<BLOCK>(k, vb, s, cur);
  }
  int i = n0;
  while (i < t) {
    const int bend = min(i + kappa, t);
    for (int j = threadIdx.x; j < s.tn; j += BLOCK) vb.ti[cur][j] |= kExpanded;  // mark R
    __syncthreads();
    for (int w0 = i; w0 < bend; w0 += NVT) {
      verify_wave<BLOCK, PM>(a, qs, p, C, w0, min(w0 + NVT, bend), s.thr, vb, s);
      verify_fold<BLOCK>(k, vb, s, cur);
    }
    i = bend;
    if (threadIdx.x == 0) {
      int ov = 0;
      for (int j = 0; j < s.tn; ++j) ov += (int)(vb.ti[cur][j] >> 31);
      s.overlap = ov;
    }
    __syncthreads();
    const int ov = s.overlap;
    for (int j = threadIdx.x; j < s.tn; j += BLOCK) vb.ti[cur][j] &= kIdMask;
    __syncthreads();
    if ((float)ov / (float)k >= tau) break;
  }
}

template <int BLOCK>
__device__ __forceinline__ void verify_dispatch(const QueryArgs& a, const float* qs, float p,
                                                const uint32_t* C, int t, int k, int kappa,
                                                float tau, bool exact, const VerifyBufs& vb,
                                                BlockScalars& s, int& cur) {
  switch (pmode_of(p)) {
    case kPOne: verify_run<BLOCK, kPOne>(a, qs, p, C, t, k, kappa, tau, exact, vb, s, cur); break;
    case kPTwo: verify_run<BLOCK, kPTwo>(a, qs, p, C, t, k, kappa, tau, exact, vb, s, cur); break;
    case kPHalf: verify_run<BLOCK, kPHalf>(a, qs, p, C, t, k, kappa, tau, exact, vb, s, cur); break;
    case kPThreeHalves:
      verify_run<BLOCK, kPThreeHalves>(a, qs, p, C, t, k, kappa, tau, exact, vb, s, cur);
      break;
    default: verify_run<BLOCK, kPGeneral>(a, qs, p, C, t, k, kappa, tau, exact, vb, s, cur); break;
  }
}

// Writes the verified list as (id, S^(1/p)) rows padded to k_max.
template <int BLOCK>
__device__ __forceinline__ void write_verified(const QueryArgs& a, int64_t qi, float p, int k,
                                               const VerifyBufs& vb, const BlockScalars& s,
                                               int cur) {
  int64_t* oid = a.out_ids + qi * a.k_max;
  float* od = a.out_dist + qi * a.k_max;
  const double inv_p = 1.0 / (double)p;
  for (int j = threadIdx.x; j < a.k_max; j += BLOCK) {
    if (j < k && j < s.tn) {
      oid[j] = (int64_t)(vb.ti[cur][j] & kIdMask);
      od[j] = (float)pow((double)vb.td[cur][j], inv_p);
    } else {
      oid[j] = -1;
      od[j] = __int_as_float(0x7f800000);
    }
  }
}

// Per-query counters; the caller lets exactly one thread of the query call it.
__device__ __forceinline__ void put_stats(const QueryArgs& a, int64_t qi, int nb, int np,
                                          int terms, int nexp, int nres, int status, int graph,
                                          int nadj) {
  if (!a.stats) return;
  int32_t* st = a.stats + qi * UHNSW_NSTATS;
  st[UHNSW_STAT_NB] = nb;
  st[UHNSW_STAT_NP] = np;
  st[UHNSW_STAT_TERMS] = terms;
  st[UHNSW_STAT_EXPANSIONS] = nexp;
  st[UHNSW_STAT_RESETS] = nres;
  st[UHNSW_STAT_STATUS] = status;
  st[UHNSW_STAT_GRAPH] = graph;
  st[UHNSW_STAT_ADJ] = nadj;
}

__device__ __forceinline__ void write_stats(const QueryArgs& a, int64_t qi, int nb, int np,
                                            int terms, int nexp, int nres, int status, int graph,
                                            int nadj) {
  if (threadIdx.x == 0) put_stats(a, qi, nb, np, terms, nexp, nres, status, graph, nadj);
}

__device__ __forceinline__ void write_invalid(const QueryArgs& a, int64_t qi, int BLOCKN) {
  for (int j = threadIdx.x; j < a.k_max; j += BLOCKN) {
    a.out_ids[qi * a.k_max + j] = -1;
    a.out_dist[qi * a.k_max + j] = __int_as_float(0x7f800000);
  }
  write_stats(a, qi, 0, 0, 0, 0, 0, UHNSW_EINVAL, 0, 0);
}

// Ballot compaction of `keep` lanes' values into out[s.m ...] (order within a
// warp kept, across warps arbitrary).
__device__ __forceinline__ void compact_append(bool keep, uint32_t v, uint32_t* out, int* counter,
                                               int cap, int32_t* err) {
  const unsigned ball = __ballot_sync(kFull, keep);
  int base = 0;
  if ((threadIdx.x & 31) == 0 && ball) base = atomicAdd(counter, __popc(ball));
  base = __shfl_sync(kFull, base, 0);
  if (keep) out[chk_idx(base + __popc(ball & lanemask_lt()), cap, 6, err)] = v;
}

// ---------------------------------------------------------------- one query
template <typename T, int TEAM, int CPL, int BLOCK>
__device__ void run_query(const QueryArgs& a, int64_t qi, unsigned char* smem, const SmemLayout& L,
                          BlockScalars& s) {
  constexpr int VEC = Elems16<T>::n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* qs = reinterpret_cast<float*>(smem + L.qs);
  float* bd[2] = {reinterpret_cast<float*>(smem + L.bd0), reinterpret_cast<float*>(smem + L.bd1)};
  uint32_t* bi[2] = {reinterpret_cast<uint32_t*>(smem + L.bi0),
                     reinterpret_cast<uint32_t*>(smem + L.bi1)};
  int32_t* tab = reinterpret_cast<int32_t*>(smem + L.hash);
  float* cd = reinterpret_cast<float*>(smem + L.cd);
  uint32_t* ci = reinterpret_cast<uint32_t*>(smem + L.ci);
  float* sd = reinterpret_cast<float*>(smem + L.sd);
  uint32_t* si = reinterpret_cast<uint32_t*>(smem + L.si);

  // 1. routing and per-query parameters (Algorithm 1 lines 1-5)
  const float p = a.p[qi];
  const int k = a.k ? a.k[qi] : a.k_max;
  const int ef = a.ef ? a.ef[qi] : a.ef_default;
  const Route rt = route_query(a, p);
  const bool direct = rt.direct;
  const int metric = rt.metric;
  const int tq = query_t(a, qi);
  int tt = direct ? k : (tq > 0 ? tq : ef);
  if (tt < k) tt = k;
  const int efp = max(ef, tt);
  const GraphDev& g = a.g[rt.slot];
  const bool ok = (p > 0.f) && (p <= 2.f) && k >= 1 && k <= a.k_max && ef >= 1 && tq >= 0 &&
                  efp <= a.ef_cap && g.ell0 != nullptr && a.width * g.deg0 <= a.cmax &&
                  g.deg <= a.cmax;
  if (!ok) {
    write_invalid(a, qi, BLOCK);
    return;
  }
  for (int j = tid; j < a.d_pad; j += BLOCK) qs[j] = j < a.d ? a.q[qi * a.d + j] : 0.f;
  __syncthreads();
  float qv[CPL][VEC];
  {
    const int lt = tid % TEAM;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int idx = (lt + c * TEAM) * VEC + e;
        qv[c][e] = idx < a.d_pad ? qs[idx] : 0.f;
      }
    }
  }
  const T* trav = reinterpret_cast<const T*>(a.trav);
  int nb = 0, nadj = 0, nexp = 0, nres = 0;

  // 2. greedy descent through the upper levels (HNSW search with beam 1)
  if (tid == 0) ci[0] = (uint32_t)g.entry;
  __syncthreads();
  dist_batch_metric<T, TEAM, CPL, BLOCK>(metric, rt.bp, trav, a.d_pad, qv, ci, cd, 1, a.n, a.err);
  __syncthreads();
  int cur = g.entry;
  float cur_d = cd[0];
  nb = 1;
  __syncthreads();
  for (int l = g.top_level; l >= 1; --l) {
    for (int guard = 0; guard <= (int)min(a.n, (int64_t)INT_MAX - 1); ++guard) {
      if (tid == 0) s.m = 0;
      __syncthreads();
      const int32_t row = g.up_row[chk_idx(cur, a.n, 3, a.err)];
      if (row < 0) {
        set_error(a.err, UHNSW_EINVAL);
        break;
      }
      const int32_t* adj = g.up_adj + chk_idx((int64_t)row + l - 1, g.up_rows, 4, a.err) * g.deg;
      for (int b0 = 0; b0 < g.deg; b0 += BLOCK) {
        const int j = b0 + tid;
        const int32_t v = j < g.deg ? adj[j] : -1;
        compact_append(v >= 0, (uint32_t)v, ci, &s.m, a.cmax, a.err);
      }
      __syncthreads();
      const int m = s.m;
      nadj += 1;
      nb += m;
      dist_batch_metric<T, TEAM, CPL, BLOCK>(metric, rt.bp, trav, a.d_pad, qv, ci, cd, m, a.n, a.err);
      __syncthreads();
      block_argmin<BLOCK>(cd, ci, m, s);
      if (m > 0 && pair_lt(s.bestd, s.besti, cur_d, cur)) {
        cur = s.besti;
        cur_d = s.bestd;
      } else {
        break;
      }
    }
  }

  // 3. layer-0 search with beam ef' (one sorted list W with expanded bits)
  const int hb = a.hash_bits;
  const int H = 1 << hb;
  for (int j = tid; j < H; j += BLOCK) tab[j] = kEmpty;
  __syncthreads();
  if (tid == 0) {
    hash_insert(tab, hb, cur, a.err);
    bd[0][0] = cur_d;
    bi[0][0] = (uint32_t)cur;
    s.bn = 1;
    s.first = 0;
    s.hcount = 1;
  }
  __syncthreads();
  int cb = 0;
  const int deg0 = g.deg0;
  const int width = a.width;
  const int64_t max_steps = a.n + 16;
  for (int64_t step = 0;; ++step) {
    // Block-shared state is read into registers here, before the step's first
    // barrier; thread 0 rewrites s.bn / s.hcount only after the step's last
    // merge barrier, so no thread can observe the next step's values early.
    const int bn = s.bn, first = s.first, hcount = s.hcount;
    if (first >= bn) break;
    if (step >= max_steps) {
      set_error(a.err, UHNSW_ECAPACITY);
      break;
    }
    if (warp == 0) {
      int npar = 0;
      for (int b0 = first; b0 < bn && npar < width; b0 += 32) {
        const int pos = b0 + lane;
        const bool un = pos < bn && !(bi[cb][pos] & kExpanded);
        const unsigned ball = __ballot_sync(kFull, un);
        const int need = width - npar;
        const int r = __popc(ball & lanemask_lt());
        if (un && r < need) {
          s.par[chk_idx(npar + r, 8, 7, a.err)] = (int)bi[cb][pos];
          bi[cb][pos] |= kExpanded;
        }
        npar += min(__popc(ball), need);
      }
      if (lane == 0) {
        s.npar = npar;
        s.m = 0;
      }
    }
    __syncthreads();
    const int npar = s.npar;
    const int total = npar * deg0;
    for (int b0 = 0; b0 < total; b0 += BLOCK) {
      const int j = b0 + tid;
      int32_t v = -1;
      if (j < total) v = g.ell0[chk_idx(s.par[j / deg0], a.n, 5, a.err) * deg0 + (j % deg0)];
      const bool fresh = v >= 0 && hash_insert(tab, hb, v, a.err);
      compact_append(fresh, (uint32_t)v, ci, &s.m, a.cmax, a.err);
    }
    __syncthreads();
    const int m = s.m;
    nexp += npar;
    nadj += npar;
    nb += m;
    dist_batch_metric<T, TEAM, CPL, BLOCK>(metric, rt.bp, trav, a.d_pad, qv, ci, cd, m, a.n, a.err);
    if (tid == 0) s.first = INT_MAX;
    __syncthreads();
    const int nbn = block_merge(bd[cb], bi[cb], bn, cd, ci, m, sd, si, bd[cb ^ 1], bi[cb ^ 1], efp,
                                &s.first);
    cb ^= 1;
    int hc = hcount + m;
    if (hc > (H >> 1)) {
      for (int j = tid; j < H; j += BLOCK) tab[j] = kEmpty;
      __syncthreads();
      for (int j = tid; j < nbn; j += BLOCK) hash_insert(tab, hb, (int32_t)(bi[cb][j] & kIdMask), a.err);
      hc = nbn;
      ++nres;
    }
    if (tid == 0) {
      s.bn = nbn;
      s.hcount = hc;
    }
    __syncthreads();
  }

  // 4-6. candidate set, verification and output
  const int bn = s.bn;
  // p in {1, 2}: the beam's first k directly on FP32 rows (or on an exact
  // FP16/BF16 copy); on an inexact copy the whole beam is re-ranked by its
  // FP32 base distance.
  const bool reduced = !std::is_same<T, float>::value && !a.trav_exact;
  const int nc = (direct && reduced) ? bn : min(tt, bn);
  int64_t* oid = a.out_ids + qi * a.k_max;
  float* odist = a.out_dist + qi * a.k_max;
  if (direct && !reduced) {
    for (int j = tid; j < a.k_max; j += BLOCK) {
      if (j < k && j < bn) {
        oid[j] = (int64_t)(bi[cb][j] & kIdMask);
        const float dd = bd[cb][j];
        odist[j] = base_root(metric, rt.bp, dd);
      } else {
        oid[j] = -1;
        odist[j] = __int_as_float(0x7f800000);
      }
    }
    write_stats(a, qi, nb, 0, 0, nexp, nres, 0, rt.slot + 1, nadj);
    return;
  }
  VerifyBufs vb;
  vb.td[0] = reinterpret_cast<float*>(smem + L.td0);
  vb.td[1] = reinterpret_cast<float*>(smem + L.td1);
  vb.ti[0] = reinterpret_cast<uint32_t*>(smem + L.ti0);
  vb.ti[1] = reinterpret_cast<uint32_t*>(smem + L.ti1);
  vb.wd = cd;
  vb.wi = ci;
  vb.sd = sd;
  vb.si = si;
  int vc = 0;
  const int kappa = a.kappa > 0 ? a.kappa : k;
  verify_dispatch<BLOCK>(a, qs, p, bi[cb], nc, k, kappa, query_tau(a, qi), direct, vb, s, vc);
  write_verified<BLOCK>(a, qi, p, k, vb, s, vc);
  write_stats(a, qi, nb, s.np, s.terms, nexp, nres, 0, rt.slot + 1, nadj);
}

template <typename T, int TEAM, int CPL, int BLOCK>
__global__ void __launch_bounds__(BLOCK) uhnsw_search_kernel(const QueryArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BlockScalars s;
  const SmemLayout L(a.d_pad, a.ef_cap, a.hash_bits, a.cmax, a.k_max, a.vcap);
  if ((uint32_t)L.total > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) set_error(a.err, UHNSW_ECAPACITY);
    return;
  }
  int64_t qi = blockIdx.x;
  for (;;) {
    if (a.queue_head) {
      if (threadIdx.x == 0) {
        const int slot = atomicAdd(a.queue_head, 1);
        s.qi = !a.qbucket ? slot : (slot < a.qbucket[1] ? a.qorder[a.qbucket[0] + slot] : (int)a.nq);
      }
      __syncthreads();
      qi = s.qi;
    }
    if (qi >= a.nq) break;
    run_query<T, TEAM, CPL, BLOCK>(a, qi, smem, L, s);
    __syncthreads();
    if (!a.queue_head) break;
  }
}

}  // namespace uhnsw_dev
