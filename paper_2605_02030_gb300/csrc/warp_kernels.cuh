// Warp-per-query form of the query kernel (same algorithm and result as
// uhnsw_search_kernel in query_kernels.cuh, Section 3.1 / Algorithm 1).
//
// Each warp owns one query at a time and a private slice of the block's
// shared memory (query vector, the two ping-pong lists of W, the visited
// table, candidate and verification buffers).  All coordination is warp
// level (ballots, shuffles, __syncwarp), so a block is just WARPS independent
// searches and an SM keeps as many queries in flight as its registers and
// shared memory allow: the layer-0 search is a chain of dependent global loads
// (adjacency row, then the candidates' rows) whose latency is hidden by the
// number of queries in flight, not by the width of one query.
//
// Candidate rows of the search are loaded into registers, U rows per team of
// lanes per round; the FP32 rows of the verification are copied into a
// per-warp staging area with cp.async, a.sv rows at a time, and summed from
// shared memory.
//
// The search order is HNSW's (one expansion per step when width == 1), the
// merge keeps the best ef' of W and the new candidates by (distance, id), and
// the verification uses the same 8-lane teams and 32-dimension groups as the
// block kernel, so both kernels return identical ids and distances.
#pragma once

#include "query_kernels.cuh"

namespace uhnsw_dev {

__device__ __forceinline__ int warp_min_int(int v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

// Warp version of block_merge: m unsorted new entries (nd, ni) into the
// ascending (ld, li) of n entries, first `cap` of the union into (od, oi).
// Returns the new length; *first receives the smallest output position of an
// entry without the flag bit (INT_MAX if none), identical in every lane.
__device__ __forceinline__ int warp_merge(const float* ld, const uint32_t* li, int n,
                                          const float* nd, const uint32_t* ni, int m, float* sd,
                                          uint32_t* si, float* od, uint32_t* oi, int cap,
                                          int* first) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < m; i += 32) {
    const float x = nd[i];
    const int32_t xi = (int32_t)(ni[i] & kIdMask);
    int r = 0;
    for (int j = 0; j < m; ++j) r += pair_lt(nd[j], (int32_t)(ni[j] & kIdMask), x, xi);
    r = (int)chk_idx(r, m, 8, nullptr);
    sd[r] = x;
    si[r] = ni[i];
  }
  __syncwarp();
  int f = INT_MAX;
  for (int i = lane; i < m; i += 32) {
    const int pos = lower_bound_pair(ld, li, n, sd[i], (int32_t)(si[i] & kIdMask)) + i;
    if (pos < cap) {
      od[pos] = sd[i];
      oi[pos] = si[i];
      if (!(si[i] & kExpanded)) f = min(f, pos);
    }
  }
  for (int j = lane; j < n; j += 32) {
    const int pos = lower_bound_pair(sd, si, m, ld[j], (int32_t)(li[j] & kIdMask)) + j;
    if (pos < cap) {
      od[pos] = ld[j];
      oi[pos] = li[j];
      if (!(li[j] & kExpanded)) f = min(f, pos);
    }
  }
  if (first) *first = warp_min_int(f);
  __syncwarp();
  const int total = n + m;
  return total < cap ? total : cap;
}

__device__ __forceinline__ void cp_async16(uint32_t smem_addr, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gsrc)
               : "memory");
}

// Waits for this lane's outstanding cp.async copies; the caller follows with
// __syncwarp() so that every lane's copies are visible to the warp.
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void prefetch_l2(const void* g) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(g));
}

// Elementwise |x - q| (metric 1), (x - q)^2 (metric 2), |x - q|^(1/2)
// (metric 3), |x - q|^(3/2) (metric 4) or |x - q|^bp (metric 5) summed over
// one 16-byte chunk of a row, as even / odd element pairs accumulated into acc.
// q holds the chunk's query values as FP32 pairs (little-endian: element 2e in
// the low half).
template <typename T, int METRIC>
__device__ __forceinline__ void chunk_partial(const uint4& v, const uint64_t (&q)[Elems16<T>::n / 2],
                                              uint64_t& acc, float bp) {
  constexpr int VEC = Elems16<T>::n;
  float x[VEC];
  unpack16<T>(v, x);
#pragma unroll
  for (int e = 0; e < VEC / 2; ++e) {
    const uint64_t df = f2_sub(f2_pack(x[2 * e], x[2 * e + 1]), q[e]);
    if (METRIC == UHNSW_BASE_L1) {
      acc = f2_add(acc, df & 0x7fffffff7fffffffull);
    } else if (METRIC == UHNSW_BASE_L05) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(df));
      acc = f2_add(acc, f2_pack(hw_sqrt(fabsf(lo)), hw_sqrt(fabsf(hi))));
    } else if (METRIC == UHNSW_BASE_L15) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(df));
      lo = fabsf(lo);
      hi = fabsf(hi);
      acc = f2_add(acc, f2_pack(lo * hw_sqrt(lo), hi * hw_sqrt(hi)));
    } else if (METRIC == UHNSW_BASE_LP) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(df));
      acc = f2_add(acc, f2_pack(hw_ex2(bp * hw_lg2(fabsf(lo))), hw_ex2(bp * hw_lg2(fabsf(hi)))));
    } else {
      acc = f2_fma(df, df, acc);
    }
  }
}

// Copies rows ids[0..nb) (row_chunks 16-byte chunks each, stride `stride`
// elements of T) into `stage` (row-major) and waits for them.  When a row is
// a divisor or a multiple of 32 chunks the lane -> (row, chunk) map needs no
// division.
template <typename T>
__device__ __forceinline__ void warp_stage_rows(const T* __restrict__ rows, int stride,
                                                int row_chunks, const uint32_t* ids, int nb,
                                                unsigned char* stage, int64_t n, int32_t* err) {
  constexpr int VEC = 16 / (int)sizeof(T);
  const int lane = threadIdx.x & 31;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage);
  if (row_chunks <= 32 && (32 % row_chunks) == 0) {
    const int per = 32 / row_chunks;
    const int sub = lane / row_chunks, ch = lane - sub * row_chunks;
    for (int r0 = 0; r0 < nb; r0 += per) {
      const int r = r0 + sub;
      if (r < nb) {
        const int64_t id = chk_idx((int64_t)(ids[r] & kIdMask), n, 1, err);
        cp_async16(sbase + (uint32_t)(r * row_chunks + ch) * 16u, rows + id * stride + ch * VEC);
      }
    }
  } else if ((row_chunks & 31) == 0) {
    for (int r = 0; r < nb; ++r) {
      const int64_t id = chk_idx((int64_t)(ids[r] & kIdMask), n, 1, err);
      for (int c0 = 0; c0 < row_chunks; c0 += 32)
        cp_async16(sbase + (uint32_t)(r * row_chunks + c0 + lane) * 16u,
                   rows + id * stride + (c0 + lane) * VEC);
    }
  } else {
    const int tot = nb * row_chunks;
    for (int c = lane; c < tot; c += 32) {
      const int r = c / row_chunks, ch = c - r * row_chunks;
      const int64_t id = chk_idx((int64_t)(ids[r] & kIdMask), n, 1, err);
      cp_async16(sbase + (uint32_t)c * 16u, rows + id * stride + ch * VEC);
    }
  }
  cp_async_wait_all();
  __syncwarp();
}

// Base distances of ids[0..m) by one warp.  TEAM lanes per row, CPL 16-byte
// chunks per lane, U rows per team loaded into registers per round; the query
// chunk is read from shared memory once per round and applied to the U rows.
// Each row accumulates its chunks in order c = 0 .. CPL-1, elements in order,
// then the team's lanes are summed by a butterfly.  (Staging the rows in
// shared memory with cp.async measured slower here: it cost more in occupancy
// than it gained in loads in flight.)
template <typename T, int TEAM, int CPL, int U, int METRIC>
__device__ __forceinline__ void warp_dist(const T* __restrict__ rows, int d_pad, const float* qs,
                                          const uint32_t* ids, float* out, int m, int64_t n,
                                          int32_t* err, float bp) {
  constexpr int VEC = Elems16<T>::n;
  constexpr int NT = 32 / TEAM;
  const int lane = threadIdx.x & 31;
  const int team = lane / TEAM, lt = lane % TEAM;
  const int R = d_pad / VEC;
  const int rounds = (m + NT * U - 1) / (NT * U);
  // A row of exactly TEAM * CPL chunks needs no chunk bounds; otherwise the
  // chunks past the row read the row's last chunk and are zeroed (no branch
  // around the loads).  Rows past m repeat the last candidate's row (already
  // in flight, so no extra DRAM traffic) and their sums are not written.
  const bool cover = TEAM * CPL == R;
  for (int r = 0; r < rounds; ++r) {
    uint4 buf[U][CPL];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = min(r * NT * U + u * NT + team, m - 1);
      const int64_t id = chk_idx((int64_t)(ids[i] & kIdMask), n, 1, err);
      const uint4* row = reinterpret_cast<const uint4*>(rows + id * d_pad);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int ch = lt + c * TEAM;
        buf[u][c] = __ldg(row + (cover ? ch : min(ch, R - 1)));
        if (!cover && ch >= R) buf[u][c] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    uint64_t acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0;  // (+0.0f, +0.0f)
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = lt + c * TEAM;
      uint64_t q[VEC / 2];
      const ulonglong2* qp = reinterpret_cast<const ulonglong2*>(qs + (cover ? ch : min(ch, R - 1)) * VEC);
#pragma unroll
      for (int e = 0; e < VEC / 4; ++e) {
        const ulonglong2 v = qp[e];
        q[2 * e] = v.x;
        q[2 * e + 1] = v.y;
      }
      if (!cover && ch >= R) {
#pragma unroll
        for (int e = 0; e < VEC / 2; ++e) q[e] = 0ull;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) chunk_partial<T, METRIC>(buf[u][c], q, acc[u], bp);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float s = f2_hsum(acc[u]);
#pragma unroll
      for (int off = TEAM / 2; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off, TEAM);
      const int i = r * NT * U + u * NT + team;
      if (lt == 0 && i < m) out[i] = s;
    }
  }
  __syncwarp();
}

template <typename T, int TEAM, int CPL, int U>
__device__ __forceinline__ void warp_dist_metric(int metric, float bp, const T* rows, int d_pad,
                                                 const float* qs, const uint32_t* ids, float* out,
                                                 int m, int64_t n, int32_t* err) {
  if (metric == UHNSW_BASE_L1) warp_dist<T, TEAM, CPL, U, 1>(rows, d_pad, qs, ids, out, m, n, err, bp);
  else if (metric == UHNSW_BASE_L2) warp_dist<T, TEAM, CPL, U, 2>(rows, d_pad, qs, ids, out, m, n, err, bp);
  else if (metric == UHNSW_BASE_L05) warp_dist<T, TEAM, CPL, U, 3>(rows, d_pad, qs, ids, out, m, n, err, bp);
  else if (metric == UHNSW_BASE_L15) warp_dist<T, TEAM, CPL, U, 4>(rows, d_pad, qs, ids, out, m, n, err, bp);
  else warp_dist<T, TEAM, CPL, U, 5>(rows, d_pad, qs, ids, out, m, n, err, bp);
}

// Drops the candidates that cannot enter a full W (those not before its last
// entry), compacting (cd, ci)[0..m) in place; returns the number kept.
__device__ __forceinline__ int warp_reject(float* cd, uint32_t* ci, int m, float wd, int32_t wi) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int b0 = 0; b0 < m; b0 += 32) {
    const int i = b0 + lane;
    float x = 0.f;
    uint32_t xi = 0;
    bool keep = false;
    if (i < m) {
      x = cd[i];
      xi = ci[i];
      keep = pair_lt(x, (int32_t)(xi & kIdMask), wd, wi);
    }
    const unsigned ball = __ballot_sync(kFull, keep);
    __syncwarp();
    if (keep) {
      const int pos = cnt + __popc(ball & lanemask_lt());
      cd[pos] = x;
      ci[pos] = xi;
    }
    cnt += __popc(ball);
    __syncwarp();
  }
  return cnt;
}

// Appends lanes with keep set to out[*cnt ...] in lane order; *cnt is a
// warp-uniform register.
__device__ __forceinline__ void warp_append(bool keep, uint32_t v, uint32_t* out, int& cnt, int cap,
                                            int32_t* err) {
  const unsigned ball = __ballot_sync(kFull, keep);
  if (keep) out[chk_idx(cnt + __popc(ball & lanemask_lt()), cap, 6, err)] = v;
  cnt += __popc(ball);
}

// ---------------------------------------------------------------- verification (warp)
struct WarpVerify {
  float* td[2];     // indexed only through cur_d() / nxt_d() (selects, no local memory)
  uint32_t* ti[2];
  float* wd;
  uint32_t* wi;
  float* sd;
  uint32_t* si;
  int cur = 0;
  int tn = 0;
  float thr;
  int np = 0;
  int terms = 0;
  __device__ __forceinline__ float* cd_() const { return cur ? td[1] : td[0]; }
  __device__ __forceinline__ uint32_t* ci_() const { return cur ? ti[1] : ti[0]; }
  __device__ __forceinline__ float* nd_() const { return cur ? td[0] : td[1]; }
  __device__ __forceinline__ uint32_t* ni_() const { return cur ? ti[0] : ti[1]; }
};

// acc + |x - q|^p over the four elements of a group, in element order.
template <int PM>
__device__ __forceinline__ float add_terms4(float acc, const float4& x, const float4& q, float p) {
  acc += pow_term<PM>(fabsf(x.x - q.x), p);
  acc += pow_term<PM>(fabsf(x.y - q.y), p);
  acc += pow_term<PM>(fabsf(x.z - q.z), p);
  acc += pow_term<PM>(fabsf(x.w - q.w), p);
  return acc;
}
// L_p sum of a staged FP32 row (shared memory) by a team of 8 lanes, with the
// same grouping and drop test as lp_sum_team.  The p form `pm` selects the
// term code per 32-dimension group (a uniform branch), so that the
// verification exists once in the kernel and not once per p form.
__device__ __forceinline__ bool lp_sum_team_staged(const float* srow, int d, int d_pad,
                                                   const float* qs, float p, int pm, float thr,
                                                   unsigned tmask, int lane8, float& S,
                                                   int& groups, int vgroups) {
  float acc = 0.0f;
  const int G = (d + 31) >> 5;
  groups = 0;
  int until_test = vgroups;
  for (int g = 0; g < G; ++g) {
    const int j = g * 32 + lane8 * 4;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f), qq = x;
    if (j < d_pad) {
      x = *reinterpret_cast<const float4*>(srow + j);
      qq = *reinterpret_cast<const float4*>(qs + j);
    }
    switch (pm) {
      case kPOne: acc = add_terms4<kPOne>(acc, x, qq, p); break;
      case kPTwo: acc = add_terms4<kPTwo>(acc, x, qq, p); break;
      case kPHalf: acc = add_terms4<kPHalf>(acc, x, qq, p); break;
      case kPThreeHalves: acc = add_terms4<kPThreeHalves>(acc, x, qq, p); break;
      default: acc = add_terms4<kPGeneral>(acc, x, qq, p); break;
    }
    groups = g + 1;
    if (--until_test > 0 && groups != G) continue;  // no drop test after this group
    until_test = vgroups;
    float tot = acc;
    tot += __shfl_xor_sync(tmask, tot, 1);
    tot += __shfl_xor_sync(tmask, tot, 2);
    tot += __shfl_xor_sync(tmask, tot, 4);
    if (tot > thr) return false;
    S = tot;
  }
  return true;
}

// Verifies C[i0 .. i1): rows are staged a.sv at a time; each wave takes 4
// staged candidates (8 lanes each) against the running threshold and folds
// the finished ones into the top-k list.  With fixed_thr set, nothing is
// dropped (the first K of Algorithm 1).
__device__ __forceinline__ void warp_verify_range(const QueryArgs& a, const float* qs, float p,
                                                  int pm, const uint32_t* C, int i0, int i1, int k,
                                                  bool no_drop, unsigned char* stage,
                                                  WarpVerify& v) {
  const int lane = threadIdx.x & 31;
  const int team = lane >> 3, lane8 = lane & 7;
  const unsigned tmask = 0xffu << (team * 8);
  const int vchunks = a.d_pad / 4;
  const float kInf = __int_as_float(0x7f800000);
  for (int s0 = i0; s0 < i1; s0 += a.sv) {
    const int nb = min(a.sv, i1 - s0);
    warp_stage_rows<float>(a.base32, a.d_pad, vchunks, C + s0, nb, stage, a.n, a.err);
    for (int w0 = 0; w0 < nb; w0 += 4) {
      const int r = w0 + team;
      bool done = false;
      float S = 0.f;
      int groups = 0;
      if (r < nb) {
        const float* srow = reinterpret_cast<const float*>(stage) + (size_t)r * a.d_pad;
        done = lp_sum_team_staged(srow, a.d, a.d_pad, qs, p, pm, no_drop ? kInf : v.thr, tmask,
                                  lane8, S, groups, a.vgroups);
      }
      const unsigned leaders = __ballot_sync(kFull, lane8 == 0 && r < nb);
      const unsigned fin = __ballot_sync(kFull, lane8 == 0 && done);
      v.np += __popc(leaders);
      int tg = (lane8 == 0 && r < nb) ? min(groups * 32, a.d) : 0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) tg += __shfl_xor_sync(kFull, tg, off);
      v.terms += tg;
      if (lane8 == 0 && done) {
        const int pos = __popc(fin & lanemask_lt());
        v.wd[pos] = S;
        v.wi[pos] = C[s0 + r] & kIdMask;
      }
      __syncwarp();
      v.tn = warp_merge(v.cd_(), v.ci_(), v.tn, v.wd, v.wi, __popc(fin), v.sd, v.si, v.nd_(),
                        v.ni_(), k, nullptr);
      v.cur ^= 1;
      v.thr = v.tn == k ? v.cd_()[k - 1] : kInf;
    }
    __syncwarp();
  }
}

// acc + |x - q|^p over one group's four elements, the p form chosen at run
// time: with SQ false p = 1, p = 2 or general p, with SQ true p = 0.5 or 1.5.
template <bool SQ>
__device__ __forceinline__ float add_group(float acc, const float4& x, const float4& q, float p,
                                           int pm) {
  if (SQ) return pm == kPHalf ? add_terms4<kPHalf>(acc, x, q, p)
                              : add_terms4<kPThreeHalves>(acc, x, q, p);
  switch (pm) {
    case kPOne: return add_terms4<kPOne>(acc, x, q, p);
    case kPTwo: return add_terms4<kPTwo>(acc, x, q, p);
    default: return add_terms4<kPGeneral>(acc, x, q, p);
  }
}

// L_p sums of two candidates (ids ida, idb; -1 = none) by one team of 8
// lanes.  A candidate is tested against thr after every vgroups groups and
// after its last; *done = finished below thr (S = its sum), *groups = groups
// accumulated.  Dropped or absent candidates take no further SFU work.
template <bool SQ>
__device__ __forceinline__ void lp_sum_pair(const float* __restrict__ base32, int d, int d_pad,
                                            const float* qs, float p, int pm, int32_t ida, int32_t idb,
                                            float thr, unsigned tmask, int lane8, int vgroups,
                                            bool& doneA, float& SA, int& gA, bool& doneB,
                                            float& SB, int& gB) {
  const int G = (d + 31) >> 5;
  bool liveA = ida >= 0, liveB = idb >= 0;
  float accA = 0.f, accB = 0.f;
  int until_test = vgroups;
  gA = gB = 0;
  SA = SB = 0.f;
  const float* ra = base32 + (int64_t)(ida >= 0 ? ida : 0) * d_pad;
  const float* rb = base32 + (int64_t)(idb >= 0 ? idb : 0) * d_pad;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int g0 = 0; g0 < G && (liveA || liveB); g0 += 4) {
    float4 xa[4], xb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = (g0 + u) * 32 + lane8 * 4;
      const bool in = g0 + u < G && j < d_pad;
      xa[u] = (liveA && in) ? __ldg(reinterpret_cast<const float4*>(ra + j)) : z;
      xb[u] = (liveB && in) ? __ldg(reinterpret_cast<const float4*>(rb + j)) : z;
    }
    // (fully unrolled: no break, so that xa / xb stay in registers)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int g = g0 + u;
      if (g < G) {
        const int j = g * 32 + lane8 * 4;
        const float4 qq = j < d_pad ? *reinterpret_cast<const float4*>(qs + j) : z;
        if (liveA) {
          accA = add_group<SQ>(accA, xa[u], qq, p, pm);
          gA = g + 1;
        }
        if (liveB) {
          accB = add_group<SQ>(accB, xb[u], qq, p, pm);
          gB = g + 1;
        }
        if (--until_test == 0 || g + 1 == G) {
          until_test = vgroups;
          float ta = accA, tb = accB;
          ta += __shfl_xor_sync(tmask, ta, 1);
          tb += __shfl_xor_sync(tmask, tb, 1);
          ta += __shfl_xor_sync(tmask, ta, 2);
          tb += __shfl_xor_sync(tmask, tb, 2);
          ta += __shfl_xor_sync(tmask, ta, 4);
          tb += __shfl_xor_sync(tmask, tb, 4);
          if (liveA) {
            if (ta > thr) liveA = false;
            else SA = ta;
          }
          if (liveB) {
            if (tb > thr) liveB = false;
            else SB = tb;
          }
        }
      }
    }
  }
  doneA = liveA;
  doneB = liveB;
}

// Verifies C[i0 .. i1) in waves of 8 candidates (two per team) against the
// running threshold (none with no_drop) and folds the finished ones into the
// top-k list.
template <bool SQ>
__device__ __forceinline__ void wverify_range(const QueryArgs& a, const float* qs, float p, int pm,
                                              const uint32_t* C, int i0, int i1, int k,
                                              bool no_drop, WarpVerify& v) {
  const int lane = threadIdx.x & 31;
  const int team = lane >> 3, lane8 = lane & 7;
  const unsigned tmask = 0xffu << (team * 8);
  const float kInf = __int_as_float(0x7f800000);
  for (int s0 = i0; s0 < i1; s0 += 8) {
    const int ia = s0 + team, ib = s0 + 4 + team;
    const int32_t ida = ia < i1 ? (int32_t)chk_idx((int64_t)(C[ia] & kIdMask), a.n, 2, a.err) : -1;
    const int32_t idb = ib < i1 ? (int32_t)chk_idx((int64_t)(C[ib] & kIdMask), a.n, 2, a.err) : -1;
    bool dA, dB;
    float SA, SB;
    int gA, gB;
    lp_sum_pair<SQ>(a.base32, a.d, a.d_pad, qs, p, pm, ida, idb, no_drop ? kInf : v.thr, tmask,
                    lane8, a.vgroups, dA, SA, gA, dB, SB, gB);
    const bool lead = lane8 == 0;
    v.np += __popc(__ballot_sync(kFull, lead && ida >= 0)) +
            __popc(__ballot_sync(kFull, lead && idb >= 0));
    int tg = lead ? (ida >= 0 ? min(gA * 32, a.d) : 0) + (idb >= 0 ? min(gB * 32, a.d) : 0) : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tg += __shfl_xor_sync(kFull, tg, off);
    v.terms += tg;
    const unsigned finA = __ballot_sync(kFull, lead && dA);
    const unsigned finB = __ballot_sync(kFull, lead && dB);
    if (lead && dA) {
      const int pos = __popc(finA & lanemask_lt());
      v.wd[pos] = SA;
      v.wi[pos] = (uint32_t)ida;
    }
    if (lead && dB) {
      const int pos = __popc(finA) + __popc(finB & lanemask_lt());
      v.wd[pos] = SB;
      v.wi[pos] = (uint32_t)idb;
    }
    __syncwarp();
    v.tn = warp_merge(v.cd_(), v.ci_(), v.tn, v.wd, v.wi, __popc(finA) + __popc(finB), v.sd, v.si,
                      v.nd_(), v.ni_(), k, nullptr);
    v.cur ^= 1;
    v.thr = v.tn == k ? v.cd_()[k - 1] : kInf;
  }
}

// Exact mode verifies all of C as one range.  Algorithm 1 takes the first K
// without a drop test, then batches of kappa until the overlap test passes.
// One call site of warp_verify_range for every p form keeps the kernel's code
// small.
__device__ __forceinline__ void warp_verify_run(const QueryArgs& a, const float* qs, float p,
                                                const uint32_t* C, int t, int k, int kappa,
                                                float tau, bool exact, unsigned char* stage,
                                                WarpVerify& v) {
  const int lane = threadIdx.x & 31;
  const int pm = pmode_of(p);
  v.tn = 0;
  v.thr = __int_as_float(0x7f800000);
  const bool paper = !exact && a.mode == UHNSW_VERIFY_PAPER;
  const int n0 = paper ? min(k, t) : t;
  for (int i = 0; i < t;) {
    const int bend = i == 0 ? n0 : min(i + kappa, t);
    if (i > 0) {
      for (int j = lane; j < v.tn; j += 32) v.ci_()[j] |= kExpanded;  // mark R
      __syncwarp();
    }
    warp_verify_range(a, qs, p, pm, C, i, bend, k, paper && i == 0, stage, v);
    const bool batch = i > 0;
    i = bend;
    if (batch) {
      int ov = 0;
      for (int j = lane; j < v.tn; j += 32) ov += (int)(v.ci_()[j] >> 31);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ov += __shfl_xor_sync(kFull, ov, off);
      for (int j = lane; j < v.tn; j += 32) v.ci_()[j] &= kIdMask;
      __syncwarp();
      if ((float)ov / (float)k >= tau) break;
    }
  }
}

// ---------------------------------------------------------------- one query (warp)
template <typename T, int TEAM, int CPL, int U>
__device__ void warp_query(const QueryArgs& a, int64_t qi, unsigned char* ws, const SmemLayout& L) {
  const int lane = threadIdx.x & 31;
  const float kInf = __int_as_float(0x7f800000);
  unsigned char* stage = ws + L.stage;
  float* qs = reinterpret_cast<float*>(ws + L.qs);
  float* const bd0 = reinterpret_cast<float*>(ws + L.bd0);
  float* const bd1 = reinterpret_cast<float*>(ws + L.bd1);
  uint32_t* const bi0 = reinterpret_cast<uint32_t*>(ws + L.bi0);
  uint32_t* const bi1 = reinterpret_cast<uint32_t*>(ws + L.bi1);
  int32_t* tab = reinterpret_cast<int32_t*>(ws + L.hash);
  float* cd = reinterpret_cast<float*>(ws + L.cd);
  uint32_t* ci = reinterpret_cast<uint32_t*>(ws + L.ci);
  float* sd = reinterpret_cast<float*>(ws + L.sd);
  uint32_t* si = reinterpret_cast<uint32_t*>(ws + L.si);
  int64_t* oid = a.out_ids + qi * a.k_max;
  float* odist = a.out_dist + qi * a.k_max;

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
  const GraphDev g = rt.slot == 0 ? a.g[0] : a.g[1];
  const bool ok = (p > 0.f) && (p <= 2.f) && k >= 1 && k <= a.k_max && ef >= 1 && tq >= 0 &&
                  efp <= a.ef_cap && g.ell0 != nullptr && a.width * g.deg0 <= a.cmax &&
                  g.deg <= a.cmax;
  if (!ok) {
    for (int j = lane; j < a.k_max; j += 32) {
      oid[j] = -1;
      odist[j] = kInf;
    }
    if (lane == 0) put_stats(a, qi, 0, 0, 0, 0, 0, UHNSW_EINVAL, 0, 0);
    return;
  }
  for (int j = lane; j < a.d_pad; j += 32) qs[j] = j < a.d ? a.q[qi * a.d + j] : 0.f;
  __syncwarp();
  const T* trav = reinterpret_cast<const T*>(a.trav);
  int nb = 1, nadj = 0, nexp = 0, nres = 0;

  // One loop, one distance call site: the greedy descent through the upper
  // levels (level >= 1), then the layer-0 search with beam ef'.  Each pass
  // computes the base distances of the list (ci, m) gathered by the pass
  // before: first the entry point alone, then the neighbours of the current
  // node at `level`, then the unvisited neighbours of the expanded parents.
  const int hb = a.hash_bits;
  const int H = 1 << hb;
  const int deg0 = g.deg0;
  const int width = a.width;
  int level = g.top_level;
  bool descending = true, at_entry = true;
  int cur = g.entry;
  float cur_d = kInf;
  int bn = 0, first = 0, hcount = 0, m = 1;
  float* bdc = bd0;      // current W (distances / ids); the other buffer receives the merge
  uint32_t* bic = bi0;
  float* bdn = bd1;
  uint32_t* bin = bi1;
  if (lane == 0) ci[0] = (uint32_t)g.entry;
  __syncwarp();
  const int64_t max_steps = ((int64_t)g.top_level + 1) * (a.n + 1) + 16;
  for (int64_t step = 0;; ++step) {
    if (step >= max_steps) {
      if (lane == 0) set_error(a.err, UHNSW_ECAPACITY);
      break;
    }
    warp_dist_metric<T, TEAM, CPL, U>(metric, rt.bp, trav, a.d_pad, qs, ci, cd, m, a.n, a.err);
    if (descending) {
      if (at_entry) {
        cur_d = cd[0];
        at_entry = false;
      } else {
        float bdd = kInf;
        int32_t bii = INT_MAX;
        for (int i = lane; i < m; i += 32)
          if (pair_lt(cd[i], (int32_t)ci[i], bdd, bii)) { bdd = cd[i]; bii = (int32_t)ci[i]; }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float od = __shfl_xor_sync(kFull, bdd, off);
          const int32_t oi = __shfl_xor_sync(kFull, bii, off);
          if (pair_lt(od, oi, bdd, bii)) { bdd = od; bii = oi; }
        }
        __syncwarp();
        if (m > 0 && pair_lt(bdd, bii, cur_d, cur)) {
          cur = bii;
          cur_d = bdd;
        } else {
          --level;
        }
      }
      if (level >= 1) {
        // the neighbours of cur at `level`
        const int32_t row = g.up_row[chk_idx(cur, a.n, 3, a.err)];
        if (row >= 0) {
          const int32_t* adj =
              g.up_adj + chk_idx((int64_t)row + level - 1, g.up_rows, 4, a.err) * g.deg;
          m = 0;
          for (int b0 = 0; b0 < g.deg; b0 += 32) {
            const int j = b0 + lane;
            const int32_t v = j < g.deg ? adj[j] : -1;
            warp_append(v >= 0, (uint32_t)v, ci, m, a.cmax, a.err);
          }
          __syncwarp();
          nadj += 1;
          nb += m;
          continue;
        }
        if (lane == 0) set_error(a.err, UHNSW_EINVAL);  // a node above its own level
      }
      // layer 0 starts from W = {cur}
      descending = false;
      for (int j = lane; j < H; j += 32) tab[j] = kEmpty;
      __syncwarp();
      if (lane == 0) {
        hash_insert(tab, hb, cur, a.err);
        bd0[0] = cur_d;
        bi0[0] = (uint32_t)cur;
      }
      __syncwarp();
      bn = 1;
      first = 0;
      hcount = 1;
    } else {
      // candidates behind a full W's last entry cannot enter it: drop them before sorting
      const int mk = bn == efp
                         ? warp_reject(cd, ci, m, bdc[bn - 1], (int32_t)(bic[bn - 1] & kIdMask))
                         : m;
      int nfirst;
      const int nbn = warp_merge(bdc, bic, bn, cd, ci, mk, sd, si, bdn, bin, efp, &nfirst);
      {
        float* t0 = bdc;
        bdc = bdn;
        bdn = t0;
        uint32_t* t1 = bic;
        bic = bin;
        bin = t1;
      }
      int hc = hcount + m;
      if (hc > (H >> 1)) {
        for (int j = lane; j < H; j += 32) tab[j] = kEmpty;
        __syncwarp();
        for (int j = lane; j < nbn; j += 32) hash_insert(tab, hb, (int32_t)(bic[j] & kIdMask), a.err);
        __syncwarp();
        hc = nbn;
        ++nres;
      }
      bn = nbn;
      first = nfirst;
      hcount = hc;
    }
    if (first >= bn) break;
    // Parents: the first `width` unexpanded entries of W, marked expanded.
    // The unexpanded entry after them is most likely the next step's parent:
    // its adjacency row is pulled toward L2 while this step runs.
    int npar = 0, nxt = -1;
    uint32_t par_mine = 0;  // lane j < npar holds parent j
    for (int b0 = first; b0 < bn && nxt < 0; b0 += 32) {
      const int pos = b0 + lane;
      unsigned ball = __ballot_sync(kFull, pos < bn && !(bic[pos] & kExpanded));
      while (ball && npar < width) {
        const int src = __ffs(ball) - 1;
        const uint32_t v = bic[b0 + src];
        __syncwarp();
        if (lane == npar) par_mine = v;
        if (lane == src) bic[pos] = v | kExpanded;
        ball &= ball - 1;
        ++npar;
      }
      if (ball) nxt = (int)bic[b0 + __ffs(ball) - 1];
    }
    if (nxt >= 0 && lane < (deg0 * 4 + 127) / 128)
      prefetch_l2(g.ell0 + chk_idx(nxt, a.n, 5, a.err) * deg0 + lane * 32);
    __syncwarp();
    // the unvisited neighbours of the parents, in parent order
    m = 0;
    for (int s = 0; s < npar; ++s) {
      const uint32_t parent = __shfl_sync(kFull, par_mine, s);
      const int32_t* adj = g.ell0 + chk_idx(parent, a.n, 5, a.err) * deg0;
      for (int b0 = 0; b0 < deg0; b0 += 32) {
        const int j = b0 + lane;
        const int32_t v = j < deg0 ? adj[j] : -1;
        const bool fresh = v >= 0 && hash_insert(tab, hb, v, a.err);
        warp_append(fresh, (uint32_t)v, ci, m, a.cmax, a.err);
      }
    }
    __syncwarp();
    nexp += npar;
    nadj += npar;
    nb += m;
  }

  // p in {1, 2} returns the beam's first k directly when the beam ran on the
  // FP32 rows or on an FP16/BF16 copy that holds every value exactly; on an
  // inexact copy the whole beam is re-ranked by its FP32 base distance, so
  // that returned distances are FP32 ones.
  const bool reduced = !std::is_same<T, float>::value && !a.trav_exact;
  const int nc = (direct && reduced) ? bn : min(tt, bn);
  if (direct && !reduced) {
    for (int j = lane; j < a.k_max; j += 32) {
      if (j < k && j < bn) {
        oid[j] = (int64_t)(bic[j] & kIdMask);
        const float dd = bdc[j];
        odist[j] = base_root(metric, rt.bp, dd);
      } else {
        oid[j] = -1;
        odist[j] = kInf;
      }
    }
    if (lane == 0) put_stats(a, qi, nb, 0, 0, nexp, nres, 0, rt.slot + 1, nadj);
    return;
  }
  WarpVerify v;
  v.td[0] = reinterpret_cast<float*>(ws + L.td0);
  v.td[1] = reinterpret_cast<float*>(ws + L.td1);
  v.ti[0] = reinterpret_cast<uint32_t*>(ws + L.ti0);
  v.ti[1] = reinterpret_cast<uint32_t*>(ws + L.ti1);
  v.wd = cd;
  v.wi = ci;
  v.sd = sd;
  v.si = si;
  const int kappa = a.kappa > 0 ? a.kappa : k;
  warp_verify_run(a, qs, p, bic, nc, k, kappa, query_tau(a, qi), direct, stage, v);
  const double inv_p = 1.0 / (double)p;
  for (int j = lane; j < a.k_max; j += 32) {
    if (j < k && j < v.tn) {
      oid[j] = (int64_t)(v.ci_()[j] & kIdMask);
      odist[j] = (float)pow((double)v.cd_()[j], inv_p);
    } else {
      oid[j] = -1;
      odist[j] = kInf;
    }
  }
  if (lane == 0) put_stats(a, qi, nb, v.np, v.terms, nexp, nres, 0, rt.slot + 1, nadj);
}

// ---------------------------------------------------------------- verification only (warp)
// The verification-only launch (uhnsw_verify, Algorithm 1 lines 6-10 on given
// candidate lists): one warp per query, no block-wide barrier.  Each 8-lane
// team takes two candidates at once and reads their FP32 rows four
// 32-dimension groups at a time into registers, all loads of a block issued
// before any arithmetic, so that the SFU work of one candidate overlaps the
// other's reductions and the next block's loads.  Every lane sums the same
// elements in the same order as lp_sum_team (element j = 32 g + 4 lane + e),
// so the sums are bit-identical to the block kernel's.

// Shared-memory carve-up of one warp of the verification-only kernel.
struct WVerifyLayout {
  int qs, td0, ti0, td1, ti1, wd, wi, sd, si, cv, total;
  __host__ __device__ WVerifyLayout(int d_pad, int k_max, int vcap) {
    int o = 0;
    qs = o; o += align16(d_pad * 4);
    td0 = o; o += align16(k_max * 4);
    ti0 = o; o += align16(k_max * 4);
    td1 = o; o += align16(k_max * 4);
    ti1 = o; o += align16(k_max * 4);
    wd = o; o += align16(8 * 4);
    wi = o; o += align16(8 * 4);
    sd = o; o += align16(8 * 4);
    si = o; o += align16(8 * 4);
    cv = o; o += align16(vcap * 4);
    total = o;
  }
};

// Exact mode over all of C, or Algorithm 1's first K then batches of kappa.
template <bool SQ>
__device__ __forceinline__ void wverify_run(const QueryArgs& a, const float* qs, float p, int pm,
                                            const uint32_t* C, int t, int k, WarpVerify& v) {
  const int lane = threadIdx.x & 31;
  v.tn = 0;
  v.thr = __int_as_float(0x7f800000);
  if (a.mode != UHNSW_VERIFY_PAPER) {
    wverify_range<SQ>(a, qs, p, pm, C, 0, t, k, false, v);
    return;
  }
  const int kappa = a.kappa > 0 ? a.kappa : k;
  const int n0 = min(k, t);
  wverify_range<SQ>(a, qs, p, pm, C, 0, n0, k, true, v);
  for (int i = n0; i < t;) {
    const int bend = min(i + kappa, t);
    for (int j = lane; j < v.tn; j += 32) v.ci_()[j] |= kExpanded;  // mark R
    __syncwarp();
    wverify_range<SQ>(a, qs, p, pm, C, i, bend, k, false, v);
    i = bend;
    int ov = 0;
    for (int j = lane; j < v.tn; j += 32) ov += (int)(v.ci_()[j] >> 31);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ov += __shfl_xor_sync(kFull, ov, off);
    for (int j = lane; j < v.tn; j += 32) v.ci_()[j] &= kIdMask;
    __syncwarp();
    if ((float)ov / (float)k >= a.tau) break;
  }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) uhnsw_wverify_kernel(const QueryArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WVerifyLayout L(a.d_pad, a.k_max, a.vcap);
  constexpr int warps = WARPS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((uint32_t)(L.total * warps) > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) set_error(a.err, UHNSW_ECAPACITY);
    return;
  }
  const int64_t qi = (int64_t)blockIdx.x * warps + warp;
  if (qi >= a.nq) return;
  unsigned char* ws = smem + (size_t)warp * L.total;
  const float p = a.p[qi];
  const int k = a.k_max;
  int64_t* oid = a.out_ids + qi * a.k_max;
  float* od = a.out_dist + qi * a.k_max;
  const float kInf = __int_as_float(0x7f800000);
  if (!(p > 0.f) || !(p <= 2.f)) {
    for (int j = lane; j < k; j += 32) {
      oid[j] = -1;
      od[j] = kInf;
    }
    if (lane == 0) put_stats(a, qi, 0, 0, 0, 0, 0, UHNSW_EINVAL, 0, 0);
    return;
  }
  float* qs = reinterpret_cast<float*>(ws + L.qs);
  uint32_t* cv = reinterpret_cast<uint32_t*>(ws + L.cv);
  for (int j = lane; j < a.d_pad; j += 32) qs[j] = j < a.d ? a.q[qi * a.d + j] : 0.f;
  // the valid candidate slots, in order
  int tv = 0;
  const int32_t* row = a.cand + qi * a.cand_t;
  for (int b0 = 0; b0 < a.cand_t; b0 += 32) {
    const int j = b0 + lane;
    const int32_t c = j < a.cand_t ? row[j] : -1;
    warp_append(c >= 0 && c < a.n, (uint32_t)c, cv, tv, a.vcap, a.err);
  }
  __syncwarp();
  WarpVerify v;
  v.td[0] = reinterpret_cast<float*>(ws + L.td0);
  v.td[1] = reinterpret_cast<float*>(ws + L.td1);
  v.ti[0] = reinterpret_cast<uint32_t*>(ws + L.ti0);
  v.ti[1] = reinterpret_cast<uint32_t*>(ws + L.ti1);
  v.wd = reinterpret_cast<float*>(ws + L.wd);
  v.wi = reinterpret_cast<uint32_t*>(ws + L.wi);
  v.sd = reinterpret_cast<float*>(ws + L.sd);
  v.si = reinterpret_cast<uint32_t*>(ws + L.si);
  const int pm = pmode_of(p);
  if (pm == kPHalf || pm == kPThreeHalves) wverify_run<true>(a, qs, p, pm, cv, tv, k, v);
  else wverify_run<false>(a, qs, p, pm, cv, tv, k, v);
  const double inv_p = 1.0 / (double)p;
  for (int j = lane; j < k; j += 32) {
    if (j < v.tn) {
      oid[j] = (int64_t)(v.ci_()[j] & kIdMask);
      od[j] = (float)pow((double)v.cd_()[j], inv_p);  // inline: a call here costs spills
    } else {
      oid[j] = -1;
      od[j] = kInf;
    }
  }
  if (lane == 0) put_stats(a, qi, 0, v.np, v.terms, 0, 0, 0, 0, 0);
}

// WARPS independent queries per block; a.queue_head set = persistent (each
// warp pulls the next query index), else query = blockIdx.x * WARPS + warp.
//
// Blocks per SM asked of the register allocator: 6 (80 registers, 24 queries
// per SM).  It measured faster than 8 blocks at 64 registers, whose spill
// traffic reached DRAM (1.83 vs 1.99 ms and 2.31 vs 2.74 ms per 10,000
// queries on 1M x 128), and than 7 blocks at 72 registers.  The smaller
// shared-memory carve-out also leaves a larger L1 for the rows.
#ifdef UHNSW_WARP_MINB
template <typename T>
struct WarpMinBlocks {
  static constexpr int value = UHNSW_WARP_MINB;
};
#else
template <typename T>
struct WarpMinBlocks {
  static constexpr int value = 6;
};
#endif
template <typename T, int TEAM, int CPL, int U, int WARPS, int MINB = WarpMinBlocks<T>::value>
__global__ void __launch_bounds__(WARPS * 32, MINB) uhnsw_wsearch_kernel(const QueryArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L(a.d_pad, a.ef_cap, a.hash_bits, a.cmax, a.k_max, 0, a.stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((uint32_t)(L.total * WARPS) > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) set_error(a.err, UHNSW_ECAPACITY);
    return;
  }
  unsigned char* ws = smem + (size_t)warp * L.total;
  int64_t qi = (int64_t)blockIdx.x * WARPS + warp;
  for (;;) {
    if (a.queue_head) {
      int v = 0;
      if (lane == 0) {
        const int slot = atomicAdd(a.queue_head, 1);
        v = !a.qbucket ? slot : (slot < a.qbucket[1] ? a.qorder[a.qbucket[0] + slot] : (int)a.nq);
      }
      qi = __shfl_sync(kFull, v, 0);
    }
    if (qi >= a.nq) break;
    warp_query<T, TEAM, CPL, U>(a, qi, ws, L);
    __syncwarp();
    if (!a.queue_head) break;
  }
}

}  // namespace uhnsw_dev
