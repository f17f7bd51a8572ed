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

// Base distances of ids[0..m) by one warp: TEAM lanes per row, CPL 16-byte
// chunks per lane, U rows per team in flight per round.
template <typename T, int TEAM, int CPL, int U, int METRIC>
__device__ __forceinline__ void warp_dist(const T* __restrict__ rows, int d_pad,
                                          const float (&qv)[CPL][Elems16<T>::n],
                                          const uint32_t* ids, float* out, int m, int64_t n,
                                          int32_t* err) {
  constexpr int VEC = Elems16<T>::n;
  constexpr int NT = 32 / TEAM;
  const int lane = threadIdx.x & 31;
  const int team = lane / TEAM, lt = lane % TEAM;
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
        const int ch = lt + c * TEAM;
        buf[u][c] = (ok && ch < R) ? ldg16(row + ch) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        float x[VEC];
        unpack16<T>(buf[u][c], x);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const float df = x[e] - qv[c][e];
          if (METRIC == 1) acc += fabsf(df);
          else acc = fmaf(df, df, acc);
        }
      }
#pragma unroll
      for (int off = TEAM / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off, TEAM);
      const int i = r * NT * U + u * NT + team;
      if (lt == 0 && i < m) out[i] = acc;
    }
  }
  __syncwarp();
}

template <typename T, int TEAM, int CPL, int U>
__device__ __forceinline__ void warp_dist_metric(int metric, const T* rows, int d_pad,
                                                 const float (&qv)[CPL][Elems16<T>::n],
                                                 const uint32_t* ids, float* out, int m,
                                                 int64_t n, int32_t* err) {
  if (metric == 1) warp_dist<T, TEAM, CPL, U, 1>(rows, d_pad, qv, ids, out, m, n, err);
  else warp_dist<T, TEAM, CPL, U, 2>(rows, d_pad, qv, ids, out, m, n, err);
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

// One wave: 4 candidates C[w0 .. wend) per warp (8 lanes each); finished sums
// are folded into the running top-k list.
template <int PM>
__device__ __forceinline__ void warp_verify_wave(const QueryArgs& a, const float* qs, float p,
                                                 const uint32_t* C, int w0, int wend, int k,
                                                 WarpVerify& v) {
  const int lane = threadIdx.x & 31;
  const int team = lane >> 3, lane8 = lane & 7;
  const unsigned tmask = 0xffu << (team * 8);
  const int i = w0 + team;
  bool done = false;
  float S = 0.f;
  int groups = 0;
  int32_t id = 0;
  if (i < wend) {
    id = (int32_t)chk_idx((int64_t)(C[i] & kIdMask), a.n, 2, a.err);
    done = lp_sum_team<PM>(a.base32, a.d, a.d_pad, qs, p, id, v.thr, tmask, lane8, S, groups);
  }
  const unsigned leaders = __ballot_sync(kFull, lane8 == 0 && i < wend);
  const unsigned fin = __ballot_sync(kFull, lane8 == 0 && done);
  // counters (lane-uniform): candidates started and terms accumulated
  v.np += __popc(leaders);
  int tg = (lane8 == 0 && i < wend) ? min(groups * 32, a.d) : 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) tg += __shfl_xor_sync(kFull, tg, off);
  v.terms += tg;
  if (lane8 == 0 && done) {
    const int pos = __popc(fin & lanemask_lt());
    v.wd[pos] = S;
    v.wi[pos] = (uint32_t)id;
  }
  __syncwarp();
  const int wm = __popc(fin);
  v.tn = warp_merge(v.cd_(), v.ci_(), v.tn, v.wd, v.wi, wm, v.sd, v.si, v.nd_(), v.ni_(), k,
                    nullptr);
  v.cur ^= 1;
  v.thr = v.tn == k ? v.cd_()[k - 1] : __int_as_float(0x7f800000);
}

template <int PM>
__device__ void warp_verify_run(const QueryArgs& a, const float* qs, float p, const uint32_t* C,
                                int t, int k, int kappa, WarpVerify& v) {
  const float kInf = __int_as_float(0x7f800000);
  const int lane = threadIdx.x & 31;
  v.tn = 0;
  v.thr = kInf;
  if (a.mode != UHNSW_VERIFY_PAPER) {
    for (int w0 = 0; w0 < t; w0 += 4) warp_verify_wave<PM>(a, qs, p, C, w0, min(w0 + 4, t), k, v);
    return;
  }
  const int n0 = min(k, t);
  for (int w0 = 0; w0 < n0; w0 += 4) {
    v.thr = kInf;
    warp_verify_wave<PM>(a, qs, p, C, w0, min(w0 + 4, n0), k, v);
  }
  v.thr = v.tn == k ? v.cd_()[k - 1] : kInf;
  int i = n0;
  while (i < t) {
    const int bend = min(i + kappa, t);
    for (int j = lane; j < v.tn; j += 32) v.ci_()[j] |= kExpanded;  // mark R
    __syncwarp();
    for (int w0 = i; w0 < bend; w0 += 4) warp_verify_wave<PM>(a, qs, p, C, w0, min(w0 + 4, bend), k, v);
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

__device__ __forceinline__ void warp_verify_dispatch(const QueryArgs& a, const float* qs, float p,
                                                     const uint32_t* C, int t, int k, int kappa,
                                                     WarpVerify& v) {
  switch (pmode_of(p)) {
    case kPOne: warp_verify_run<kPOne>(a, qs, p, C, t, k, kappa, v); break;
    case kPTwo: warp_verify_run<kPTwo>(a, qs, p, C, t, k, kappa, v); break;
    case kPHalf: warp_verify_run<kPHalf>(a, qs, p, C, t, k, kappa, v); break;
    case kPThreeHalves: warp_verify_run<kPThreeHalves>(a, qs, p, C, t, k, kappa, v); break;
    default: warp_verify_run<kPGeneral>(a, qs, p, C, t, k, kappa, v); break;
  }
}

// ---------------------------------------------------------------- one query (warp)
template <typename T, int TEAM, int CPL, int U>
__device__ void warp_query(const QueryArgs& a, int64_t qi, unsigned char* ws, const SmemLayout& L) {
  constexpr int VEC = Elems16<T>::n;
  const int lane = threadIdx.x & 31;
  const float kInf = __int_as_float(0x7f800000);
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
  const bool direct = (p == 1.0f) || (p == 2.0f);
  const int metric = direct ? (p == 1.0f ? 1 : 2) : (p <= a.cutoff ? 1 : 2);
  int tt = direct ? k : (a.t > 0 ? a.t : ef);
  if (tt < k) tt = k;
  const int efp = max(ef, tt);
  const GraphDev g = metric == 1 ? a.g[0] : a.g[1];
  const bool ok = (p > 0.f) && (p <= 2.f) && k >= 1 && k <= a.k_max && ef >= 1 &&
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
  float qv[CPL][VEC];
  {
    const int lt = lane % TEAM;
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int idx = (lt + c * TEAM) * VEC + e;
        qv[c][e] = idx < a.d_pad ? qs[idx] : 0.f;
      }
  }
  const T* trav = reinterpret_cast<const T*>(a.trav);
  int nb = 1, nadj = 0, nexp = 0, nres = 0;

  // greedy descent through the upper levels
  if (lane == 0) ci[0] = (uint32_t)g.entry;
  __syncwarp();
  warp_dist_metric<T, TEAM, CPL, U>(metric, trav, a.d_pad, qv, ci, cd, 1, a.n, a.err);
  int cur = g.entry;
  float cur_d = cd[0];
  __syncwarp();
  for (int l = g.top_level; l >= 1; --l) {
    for (int guard = 0; guard <= (int)min(a.n, (int64_t)INT_MAX - 1); ++guard) {
      const int32_t row = g.up_row[chk_idx(cur, a.n, 3, a.err)];
      if (row < 0) {
        if (lane == 0) set_error(a.err, UHNSW_EINVAL);
        break;
      }
      const int32_t* adj = g.up_adj + chk_idx((int64_t)row + l - 1, g.up_rows, 4, a.err) * g.deg;
      int m = 0;
      for (int b0 = 0; b0 < g.deg; b0 += 32) {
        const int j = b0 + lane;
        const int32_t v = j < g.deg ? adj[j] : -1;
        warp_append(v >= 0, (uint32_t)v, ci, m, a.cmax, a.err);
      }
      __syncwarp();
      nadj += 1;
      nb += m;
      warp_dist_metric<T, TEAM, CPL, U>(metric, trav, a.d_pad, qv, ci, cd, m, a.n, a.err);
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
        break;
      }
    }
  }

  // layer-0 search with beam ef'
  const int hb = a.hash_bits;
  const int H = 1 << hb;
  for (int j = lane; j < H; j += 32) tab[j] = kEmpty;
  __syncwarp();
  if (lane == 0) {
    hash_insert(tab, hb, cur, a.err);
    bd0[0] = cur_d;
    bi0[0] = (uint32_t)cur;
  }
  __syncwarp();
  int bn = 1, first = 0, hcount = 1;
  float* bdc = bd0;      // current W (distances / ids); the other buffer receives the merge
  uint32_t* bic = bi0;
  float* bdn = bd1;
  uint32_t* bin = bi1;
  const int deg0 = g.deg0;
  const int width = a.width;
  const int64_t max_steps = a.n + 16;
  for (int64_t step = 0; first < bn; ++step) {
    if (step >= max_steps) {
      if (lane == 0) set_error(a.err, UHNSW_ECAPACITY);
      break;
    }
    // parents: the first `width` unexpanded entries of W
    int npar = 0;
    uint32_t par_mine = 0;  // lane j < npar holds parent j
    for (int b0 = first; b0 < bn && npar < width; b0 += 32) {
      const int pos = b0 + lane;
      const bool un = pos < bn && !(bic[pos] & kExpanded);
      const unsigned ball = __ballot_sync(kFull, un);
      const int need = width - npar;
      const int r = __popc(ball & lanemask_lt());
      uint32_t pid = 0;
      const bool take = un && r < need;
      if (take) {
        pid = bic[pos];
        bic[pos] = pid | kExpanded;
      }
      // move each taken id to lane npar + r
      const unsigned takers = __ballot_sync(kFull, take);
      for (int s = 0; s < min(__popc(ball), need); ++s) {
        const int src = __fns(takers, 0, s + 1);
        const uint32_t v = __shfl_sync(kFull, pid, src);
        if (lane == npar + s) par_mine = v;
      }
      npar += min(__popc(ball), need);
    }
    __syncwarp();
    const int total = npar * deg0;
    int m = 0;
    for (int b0 = 0; b0 < total; b0 += 32) {
      const int j = b0 + lane;
      const int pj = j / deg0;
      const uint32_t parent = __shfl_sync(kFull, par_mine, pj < 32 ? pj : 0);
      int32_t v = -1;
      if (j < total) v = g.ell0[chk_idx(parent, a.n, 5, a.err) * deg0 + (j % deg0)];
      const bool fresh = v >= 0 && hash_insert(tab, hb, v, a.err);
      warp_append(fresh, (uint32_t)v, ci, m, a.cmax, a.err);
    }
    __syncwarp();
    nexp += npar;
    nadj += npar;
    nb += m;
    warp_dist_metric<T, TEAM, CPL, U>(metric, trav, a.d_pad, qv, ci, cd, m, a.n, a.err);
    int nfirst;
    const int nbn = warp_merge(bdc, bic, bn, cd, ci, m, sd, si, bdn, bin, efp, &nfirst);
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

  const int nc = min(tt, bn);
  if (direct) {
    for (int j = lane; j < a.k_max; j += 32) {
      if (j < k && j < bn) {
        oid[j] = (int64_t)(bic[j] & kIdMask);
        const float dd = bdc[j];
        odist[j] = metric == 1 ? dd : sqrtf(dd);
      } else {
        oid[j] = -1;
        odist[j] = kInf;
      }
    }
    if (lane == 0) put_stats(a, qi, nb, 0, 0, nexp, nres, 0, metric, nadj);
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
  warp_verify_dispatch(a, qs, p, bic, nc, k, kappa, v);
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
  if (lane == 0) put_stats(a, qi, nb, v.np, v.terms, nexp, nres, 0, metric, nadj);
}

// WARPS independent queries per block; a.queue_head set = persistent (each
// warp pulls the next query index), else query = blockIdx.x * WARPS + warp.
#ifndef UHNSW_WARP_MINB
#define UHNSW_WARP_MINB 8
#endif
template <typename T, int TEAM, int CPL, int U, int WARPS, int MINB = UHNSW_WARP_MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) uhnsw_wsearch_kernel(const QueryArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L(a.d_pad, a.ef_cap, a.hash_bits, a.cmax, a.k_max, 0);
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
      if (lane == 0) v = atomicAdd(a.queue_head, 1);
      qi = __shfl_sync(kFull, v, 0);
    }
    if (qi >= a.nq) break;
    warp_query<T, TEAM, CPL, U>(a, qi, ws, L);
    __syncwarp();
    if (!a.queue_head) break;
  }
}

}  // namespace uhnsw_dev
