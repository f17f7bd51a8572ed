// Host side of the C ABI declared in uhnsw.h: argument validation, index
// upload (FP32 master rows, FP16/BF16 traversal rows, padded layer-0 link
// tables, upper-level link rows), kernel dispatch, CUDA-graph replay of
// repeated call shapes, the host-buffer search and the error channel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "launch.h"
#include "uhnsw.h"
#include "uhnsw_internal.h"

namespace uhnsw_internal {

static thread_local char g_err[512] = {0};

void clear_error() { g_err[0] = 0; }

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

}  // namespace uhnsw_internal

using uhnsw_internal::clear_error;
using uhnsw_internal::fail;
using namespace uhnsw_dev;

namespace {

struct DevGraph {
  bool present = false;
  int32_t* ell0 = nullptr;
  int32_t* up_row = nullptr;
  int32_t* up_adj = nullptr;
  int32_t up_rows = 0;
  int32_t entry = 0, top_level = 0, deg0 = 0, deg = 0;
  int64_t bytes = 0;
};

struct GraphKey {
  const void* ptr[7];
  int64_t nq;
  int32_t k_max, ef_default;
  uhnsw_search_opts opts;
  void* stream;
  bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
};

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? UHNSW_EOOM : UHNSW_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}
int cuda_fail(cudaError_t e, const char* fn, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? UHNSW_EOOM : UHNSW_ECUDA, "%s: %s: %s", fn, what,
              cudaGetErrorString(e));
}

int next_pow2_bits(int64_t x) {
  int b = 0;
  while ((1ll << b) < x) ++b;
  return b;
}

}  // namespace

struct uhnsw_index {
  int device = 0;
  int num_sms = 0;
  int64_t n = 0;
  int32_t d = 0, d_pad = 0;
  uhnsw_dtype tdtype = UHNSW_F32;
  bool trav_exact = true;  // the traversal copy reproduces every FP32 value
  int32_t gmetric[2] = {UHNSW_BASE_L1, UHNSW_BASE_L2};  // base metric of each graph slot
  float gp[2] = {1.f, 2.f};       // the p of each slot's base metric
  float* base32 = nullptr;
  void* trav = nullptr;
  DevGraph g[2];
  int32_t* err = nullptr;         // sticky device error word
  int64_t bytes = 0;
  cudaStream_t capture_stream = nullptr;
  std::mutex mu;
  std::vector<GraphEntry> graphs;
  // exact-search workspace
  void* exact_ws = nullptr;
  size_t exact_ws_bytes = 0;
  // State of each stream that searched this index, so that searches on
  // different streams may overlap on the GPU.  The persistent-search queue:
  // work counters (one per beam bucket) and the ordering workspace (bin
  // counters and cursors, bucket slots, the order array); a workspace that
  // grows keeps its old buffer alive until the index is freed, since CUDA
  // graphs captured on that stream still point at it.  The host-buffer
  // searches' device staging.  A lock that keeps one call's work together
  // on the stream (queue reset, ordering, search; the copies of a
  // host-buffer search), so that calls from several host threads on one
  // stream do not interleave.
  struct StreamState {
    void* stream = nullptr;
    int32_t* head = nullptr;
    int32_t* ws = nullptr;
    int64_t cap = 0;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    std::mutex mu;
  };
  std::vector<std::unique_ptr<StreamState>> streams;
  std::vector<void*> retired;
  std::mutex streams_mu;
  // autotuned launch configurations: key (ef bucket, k bucket) -> options
  std::vector<std::pair<int64_t, uhnsw_search_opts>> tuned;
  std::mutex tuned_mu;

  ~uhnsw_index() {
    for (auto& e : graphs) cudaGraphExecDestroy(e.exec);
    for (auto& gg : g) {
      cudaFree(gg.ell0);
      cudaFree(gg.up_row);
      cudaFree(gg.up_adj);
    }
    if (trav && trav != base32) cudaFree(trav);
    cudaFree(base32);
    cudaFree(err);
    for (auto& ss : streams) {
      cudaFree(ss->head);
      cudaFree(ss->ws);
      cudaFree(ss->stage);
    }
    for (void* r : retired) cudaFree(r);
    cudaFree(exact_ws);
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

namespace {

// Checks the CSR of one graph and builds its device tables on the host.
int check_and_pack(const uhnsw_graph* g, int64_t n, const char* name, std::vector<int32_t>& ell0,
                   std::vector<int32_t>& up_row, std::vector<int32_t>& up_adj) {
  if (g->num_levels < 1 || g->num_levels > UHNSW_MAX_LEVELS)
    return fail(UHNSW_EINVAL, "%s: num_levels %d not in [1, %d]", name, g->num_levels,
                UHNSW_MAX_LEVELS);
  if (!g->level_count) return fail(UHNSW_EINVAL, "%s: level_count is NULL", name);
  const int32_t deg0 = g->max_degree0, deg = g->max_degree;
  if (deg0 < 1 || deg0 > UHNSW_MAX_DEGREE || deg < 1 || deg > UHNSW_MAX_DEGREE)
    return fail(UHNSW_EINVAL, "%s: degrees (%d, %d) not in [1, %d]", name, deg0, deg,
                UHNSW_MAX_DEGREE);
  if (g->level_count[0] != n)
    return fail(UHNSW_EINVAL, "%s: level 0 has %d nodes, base has %lld", name, g->level_count[0],
                (long long)n);
  std::vector<int8_t> top(n, 0);  // highest level of each node
  for (int32_t l = 0; l < g->num_levels; ++l) {
    const int64_t cnt = g->level_count[l];
    const int32_t* nodes = g->level_nodes[l];
    const int64_t* off = g->level_offsets[l];
    const int32_t* nb = g->level_nbrs[l];
    if (cnt < 1 || cnt > n) return fail(UHNSW_EINVAL, "%s: level %d has %lld nodes", name, l, (long long)cnt);
    if (!off || (!nb && off[cnt] > 0)) return fail(UHNSW_EINVAL, "%s: level %d arrays missing", name, l);
    if (l > 0 && !nodes) return fail(UHNSW_EINVAL, "%s: level %d nodes is NULL", name, l);
    if (off[0] != 0) return fail(UHNSW_EINVAL, "%s: level %d offsets[0] != 0", name, l);
    const int32_t cap = l == 0 ? deg0 : deg;
    for (int64_t i = 0; i < cnt; ++i) {
      const int32_t v = nodes ? nodes[i] : (int32_t)i;
      if (v < 0 || v >= n) return fail(UHNSW_EINVAL, "%s: level %d node %d out of range", name, l, v);
      if (nodes && i > 0 && nodes[i - 1] >= v)
        return fail(UHNSW_EINVAL, "%s: level %d nodes not strictly ascending", name, l);
      if (l > 0 && top[v] != l - 1)
        return fail(UHNSW_EINVAL, "%s: node %d on level %d but not on level %d", name, v, l, l - 1);
      const int64_t a = off[i], b = off[i + 1];
      if (b < a || b - a > cap)
        return fail(UHNSW_EINVAL, "%s: level %d node %d has degree %lld (cap %d)", name, l, v,
                    (long long)(b - a), cap);
      for (int64_t e = a; e < b; ++e)
        if (nb[e] < 0 || nb[e] >= n)
          return fail(UHNSW_EINVAL, "%s: level %d link %d out of range", name, l, nb[e]);
      if (l > 0) top[v] = (int8_t)l;
    }
  }
  // every neighbour at level l must itself be on level l
  for (int32_t l = 1; l < g->num_levels; ++l) {
    const int64_t cnt = g->level_count[l];
    for (int64_t e = 0; e < g->level_offsets[l][cnt]; ++e)
      if (top[g->level_nbrs[l][e]] < l)
        return fail(UHNSW_EINVAL, "%s: level %d links to node %d, which is not on it", name, l,
                    g->level_nbrs[l][e]);
  }
  if (g->entry_point < 0 || g->entry_point >= n || top[g->entry_point] != g->num_levels - 1)
    return fail(UHNSW_EINVAL, "%s: entry point %d is not on the top level", name, g->entry_point);

  ell0.assign(n * (int64_t)deg0, -1);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t a = g->level_offsets[0][i], b = g->level_offsets[0][i + 1];
    const int32_t v = g->level_nodes[0] ? g->level_nodes[0][i] : (int32_t)i;
    std::copy(g->level_nbrs[0] + a, g->level_nbrs[0] + b, ell0.begin() + (int64_t)v * deg0);
  }
  up_row.assign(n, -1);
  int64_t rows = 0;
  for (int64_t v = 0; v < n; ++v)
    if (top[v] > 0) {
      up_row[v] = (int32_t)rows;
      rows += top[v];
    }
  if (rows > INT32_MAX) return fail(UHNSW_ECAPACITY, "%s: too many upper-level rows", name);
  up_adj.assign(std::max<int64_t>(rows, 1) * deg, -1);
  for (int32_t l = 1; l < g->num_levels; ++l)
    for (int64_t i = 0; i < g->level_count[l]; ++i) {
      const int32_t v = g->level_nodes[l][i];
      const int64_t a = g->level_offsets[l][i], b = g->level_offsets[l][i + 1];
      std::copy(g->level_nbrs[l] + a, g->level_nbrs[l] + b,
                up_adj.begin() + ((int64_t)up_row[v] + l - 1) * deg);
    }
  return UHNSW_OK;
}

template <typename T>
int upload(const std::vector<T>& h, T** d, int64_t* bytes) {
  const size_t sz = h.size() * sizeof(T);
  cudaError_t e = cudaMalloc(d, sz);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  *bytes += sz;
  e = cudaMemcpy(*d, h.data(), sz, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return UHNSW_OK;
}

GraphDev to_dev(const DevGraph& g) {
  GraphDev r;
  r.ell0 = g.present ? g.ell0 : nullptr;
  r.up_row = g.up_row;
  r.up_adj = g.up_adj;
  r.up_rows = g.up_rows;
  r.entry = g.entry;
  r.top_level = g.top_level;
  r.deg0 = g.deg0;
  r.deg = g.deg;
  return r;
}

constexpr int kBlock = 128;

// The p of a base metric code 1-4 (uhnsw_base_metric).
float base_metric_p(int32_t m) {
  return m == UHNSW_BASE_L1 ? 1.f : m == UHNSW_BASE_L2 ? 2.f : m == UHNSW_BASE_L05 ? 0.5f : 1.5f;
}

}  // namespace

extern "C" const char* uhnsw_last_error(void) { return uhnsw_internal::g_err; }

extern "C" int uhnsw_load(const float* base, int64_t n, int32_t d, const uhnsw_graph* g1,
                          const uhnsw_graph* g2, const uhnsw_load_opts* opts, uhnsw_index** out) {
  clear_error();
  if (!out) return fail(UHNSW_EINVAL, "uhnsw_load: out is NULL");
  *out = nullptr;
  if (!base) return fail(UHNSW_EINVAL, "uhnsw_load: base is NULL");
  if (n < 1 || n > INT32_MAX) return fail(UHNSW_EINVAL, "uhnsw_load: n=%lld out of range", (long long)n);
  if (d < 1 || d > UHNSW_MAX_DIM) return fail(UHNSW_EINVAL, "uhnsw_load: d=%d out of range", d);
  if (!g1 && !g2) return fail(UHNSW_EINVAL, "uhnsw_load: no graph given");
  const uhnsw_dtype dt = opts ? opts->traverse_dtype : UHNSW_F32;
  if (dt != UHNSW_F32 && dt != UHNSW_F16 && dt != UHNSW_BF16)
    return fail(UHNSW_EINVAL, "uhnsw_load: unknown traverse dtype %d", (int)dt);
  int32_t gm[2] = {UHNSW_BASE_L1, UHNSW_BASE_L2};
  float gp[2] = {1.f, 2.f};
  for (int i = 0; i < 2; ++i) {
    const int32_t m = opts ? opts->base_metric[i] : 0;
    if (m == 0) continue;
    if (m < UHNSW_BASE_L1 || m > UHNSW_BASE_LP)
      return fail(UHNSW_EINVAL, "uhnsw_load: base_metric[%d]=%d is not a uhnsw_base_metric", i, m);
    if (m == UHNSW_BASE_LP) {
      const float bp = opts->base_p[i];
      if (!(bp > 0.f && bp <= 2.f))
        return fail(UHNSW_EINVAL, "uhnsw_load: base_p[%d]=%g outside (0, 2]", i, (double)bp);
      gm[i] = uhnsw_internal::base_metric_of_p(bp);
      gp[i] = bp;
    } else {
      gm[i] = m;
      gp[i] = base_metric_p(m);
    }
  }
  if (!(gp[0] < gp[1]))
    return fail(UHNSW_EINVAL, "uhnsw_load: the first graph's base p must be below the second's");

  std::vector<int32_t> ell[2], upr[2], upa[2];
  try {
    const uhnsw_graph* gs[2] = {g1, g2};
    for (int i = 0; i < 2; ++i) {
      if (!gs[i]) continue;
      int rc = check_and_pack(gs[i], n, i == 0 ? "G1" : "G2", ell[i], upr[i], upa[i]);
      if (rc != UHNSW_OK) return rc;
    }
  } catch (const std::bad_alloc&) {
    return fail(UHNSW_EOOM, "uhnsw_load: out of host memory");
  }

  uhnsw_index* idx = new (std::nothrow) uhnsw_index();
  if (!idx) return fail(UHNSW_EOOM, "uhnsw_load: out of host memory");
  cudaError_t e = cudaGetDevice(&idx->device);
  if (e != cudaSuccess) {
    delete idx;
    return cuda_fail(e, "uhnsw_load: cudaGetDevice");
  }
  e = cudaDeviceGetAttribute(&idx->num_sms, cudaDevAttrMultiProcessorCount, idx->device);
  if (e != cudaSuccess) {
    delete idx;
    return cuda_fail(e, "uhnsw_load: cudaDeviceGetAttribute");
  }
  idx->n = n;
  idx->d = d;
  idx->d_pad = (d + 7) / 8 * 8;
  idx->tdtype = dt;
  for (int i = 0; i < 2; ++i) {
    idx->gmetric[i] = gm[i];
    idx->gp[i] = gp[i];
  }
  int rc = UHNSW_OK;
  const size_t row32 = (size_t)idx->d_pad * 4;
  do {
    e = cudaMalloc(&idx->base32, row32 * n);
    if (e != cudaSuccess) { rc = cuda_fail(e, "uhnsw_load: base"); break; }
    idx->bytes += row32 * n;
    e = cudaMemset(idx->base32, 0, row32 * n);
    if (e == cudaSuccess)
      e = cudaMemcpy2D(idx->base32, row32, base, (size_t)d * 4, (size_t)d * 4, n,
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { rc = cuda_fail(e, "uhnsw_load: base upload"); break; }
    if (dt == UHNSW_F32) {
      idx->trav = idx->base32;
    } else {
      e = cudaMalloc(&idx->trav, row32 / 2 * n);
      if (e != cudaSuccess) { rc = cuda_fail(e, "uhnsw_load: traversal copy"); break; }
      idx->bytes += row32 / 2 * n;
      e = launch_convert(idx->base32, idx->trav, dt, (int64_t)idx->d_pad * n, 0);
      unsigned long long* bad = nullptr;
      if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(unsigned long long));
      if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(unsigned long long));
      if (e == cudaSuccess)
        e = launch_inexact_count(idx->base32, idx->trav, dt, (int64_t)idx->d_pad * n, bad, 0);
      unsigned long long nbad = 1;
      if (e == cudaSuccess) e = cudaMemcpy(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost);
      cudaFree(bad);
      if (e != cudaSuccess) { rc = cuda_fail(e, "uhnsw_load: convert"); break; }
      idx->trav_exact = nbad == 0;
    }
    const uhnsw_graph* gs[2] = {g1, g2};
    for (int i = 0; i < 2 && rc == UHNSW_OK; ++i) {
      if (!gs[i]) continue;
      DevGraph& G = idx->g[i];
      G.present = true;
      G.entry = gs[i]->entry_point;
      G.top_level = gs[i]->num_levels - 1;
      G.deg0 = gs[i]->max_degree0;
      G.deg = gs[i]->max_degree;
      G.up_rows = (int32_t)(upa[i].size() / G.deg);
      rc = upload(ell[i], &G.ell0, &idx->bytes);
      if (rc == UHNSW_OK) rc = upload(upr[i], &G.up_row, &idx->bytes);
      if (rc == UHNSW_OK) rc = upload(upa[i], &G.up_adj, &idx->bytes);
    }
    if (rc != UHNSW_OK) break;
    e = cudaMalloc(&idx->err, 16);
    if (e == cudaSuccess) e = cudaMemset(idx->err, 0, 16);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&idx->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { rc = cuda_fail(e, "uhnsw_load: state"); break; }
  } while (0);
  if (rc != UHNSW_OK) {
    delete idx;
    return rc;
  }
  *out = idx;
  return UHNSW_OK;
}

namespace {

struct Launch {
  QueryArgs a;
  bool warp;     // warp-per-query kernel, else block-per-query
  size_t smem;
  int grid;
};

struct Prepared {
  QueryArgs a;
  TeamShape shape;    // block-per-query kernel
  WarpShape wshape;   // warp-per-query kernel
  bool persistent;
  // persistent search: the queue is ordered by (beam bucket, route); with
  // per-query ef, one launch per beam bucket, largest first, each sized for
  // its own bucket's beam
  bool bucketed = false;
  BeamBuckets bb;
  cudaEvent_t events[2] = {nullptr, nullptr};  // opts.kernel_events, if given
  int32_t* qhead = nullptr;  // the stream's queue (persistent search)
  int32_t* qws = nullptr;
  uhnsw_index::StreamState* qstate = nullptr;
  std::vector<Launch> launches;
};

// Visited-table size (log2 slots) of a launch whose beam is at most `bound`:
// the caller's choice (already checked against its minimum, and kept inside
// the minimum of this bound's table too), else 4 (bound + width * M0) rounded
// up to a power of two, at least 2^9.
int visited_bits(int asked, int bound, int width, int deg0) {
  const int def = std::max(9, next_pow2_bits(4ll * (bound + width * deg0)));
  if (asked <= 0) return def;
  return std::max(asked, next_pow2_bits(2ll * (bound + width * deg0)));
}

// The state of `stream` (created on the stream's first search that needs it).
int stream_state(uhnsw_index* idx, void* stream, uhnsw_index::StreamState** out) {
  std::lock_guard<std::mutex> lock(idx->streams_mu);
  for (auto& x : idx->streams)
    if (x->stream == stream) {
      *out = x.get();
      return UHNSW_OK;
    }
  std::unique_ptr<uhnsw_index::StreamState> fresh(new (std::nothrow) uhnsw_index::StreamState);
  if (!fresh) return fail(UHNSW_EOOM, "uhnsw_search: stream state");
  fresh->stream = stream;
  *out = fresh.get();
  idx->streams.push_back(std::move(fresh));
  return UHNSW_OK;
}

// The persistent-search queue of `stream` with an ordering workspace of at
// least `need` words.
int queue_for(uhnsw_index* idx, void* stream, int64_t need, uhnsw_index::StreamState** out) {
  uhnsw_index::StreamState* qu = nullptr;
  int rc = stream_state(idx, stream, &qu);
  if (rc != UHNSW_OK) return rc;
  std::lock_guard<std::mutex> lock(idx->streams_mu);
  if (!qu->head) {
    cudaError_t e = cudaMalloc(&qu->head, 16 * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: queue counters");
  }
  if (need > qu->cap) {
    const int64_t cap = std::max(need, 2 * qu->cap);
    int32_t* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, cap * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: queue workspace");
    if (qu->ws) idx->retired.push_back(qu->ws);
    qu->ws = ws;
    qu->cap = cap;
  }
  *out = qu;
  return UHNSW_OK;
}

// Validates host-side search arguments and fills the launch description for
// a search queued on `stream`.
int prepare_search(uhnsw_index* idx, const float* q, const float* p, const int32_t* k,
                   const int32_t* ef, int64_t nq, int32_t k_max, int32_t ef_default,
                   const uhnsw_search_opts* o, int64_t* out_ids, float* out_dist, void* stream,
                   Prepared* P) {
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_search: index is NULL");
  if (nq < 0 || nq > INT32_MAX) return fail(UHNSW_EINVAL, "uhnsw_search: nq=%lld", (long long)nq);
  if (nq > 0 && (!q || !p || !out_ids || !out_dist))
    return fail(UHNSW_EINVAL, "uhnsw_search: NULL q/p/out pointer");
  if (k_max < 1 || k_max > UHNSW_MAX_EF)
    return fail(UHNSW_EINVAL, "uhnsw_search: k_max=%d not in [1, %d]", k_max, UHNSW_MAX_EF);
  if (ef_default < 1 || ef_default > UHNSW_MAX_EF)
    return fail(UHNSW_EINVAL, "uhnsw_search: ef_default=%d not in [1, %d]", ef_default, UHNSW_MAX_EF);
  uhnsw_search_opts opts;
  std::memset(&opts, 0, sizeof(opts));
  if (o) opts = *o;
  if (opts.t < 0 || opts.t > UHNSW_MAX_EF) return fail(UHNSW_EINVAL, "uhnsw_search: t=%d", opts.t);
  if (opts.kappa < 0) return fail(UHNSW_EINVAL, "uhnsw_search: kappa=%d", opts.kappa);
  if (!std::isfinite(opts.tau)) return fail(UHNSW_EINVAL, "uhnsw_search: tau");
  if (!(opts.cutoff >= 0.f) || !std::isfinite(opts.cutoff))
    return fail(UHNSW_EINVAL, "uhnsw_search: cutoff");
  if (opts.verify_mode != UHNSW_VERIFY_EXACT && opts.verify_mode != UHNSW_VERIFY_PAPER)
    return fail(UHNSW_EINVAL, "uhnsw_search: verify_mode=%d", opts.verify_mode);
  if (opts.search_width < 0 || opts.search_width > 8)
    return fail(UHNSW_EINVAL, "uhnsw_search: search_width=%d not in [0, 8]", opts.search_width);
  if (opts.query_threads != 0 && opts.query_threads != 32 && opts.query_threads != kBlock)
    return fail(UHNSW_EINVAL, "uhnsw_search: query_threads=%d not 0, 32 or %d", opts.query_threads,
                kBlock);
  if (opts.ef_max < 0 || opts.ef_max > UHNSW_MAX_EF)
    return fail(UHNSW_EINVAL, "uhnsw_search: ef_max=%d", opts.ef_max);
  if (opts.team_lanes != 0 && opts.team_lanes != 4 && opts.team_lanes != 8 &&
      opts.team_lanes != 16 && opts.team_lanes != 32)
    return fail(UHNSW_EINVAL, "uhnsw_search: team_lanes=%d not 0, 4, 8, 16 or 32",
                opts.team_lanes);
  if (opts.stage_bytes < 0 || opts.stage_bytes > 64 * 1024)
    return fail(UHNSW_EINVAL, "uhnsw_search: stage_bytes=%d not in [0, 65536]", opts.stage_bytes);
  if (opts.hash_bits < 0 || opts.hash_bits > 15)
    return fail(UHNSW_EINVAL, "uhnsw_search: hash_bits=%d not in [0, 15]", opts.hash_bits);
  if (opts.verify_groups < 0 || opts.verify_groups > 16)
    return fail(UHNSW_EINVAL, "uhnsw_search: verify_groups=%d not in [0, 16]", opts.verify_groups);

  int ef_cap;
  const bool per_query_beam = ef != nullptr || opts.t_per_query != nullptr;
  if (per_query_beam) ef_cap = opts.ef_max > 0 ? opts.ef_max : UHNSW_MAX_EF;
  else ef_cap = std::max({ef_default, opts.t, k_max});
  if (ef_cap > UHNSW_MAX_EF)
    return fail(UHNSW_EINVAL, "uhnsw_search: beam %d exceeds %d", ef_cap, UHNSW_MAX_EF);
  // query_threads given by the caller is binding; otherwise (0, or the
  // autotuned choice) a beam bucket whose warp-kernel layout does not fit in
  // shared memory runs the block kernel instead
  const bool forced = opts.query_threads != 0;
  if (opts.query_threads == 0) {
    // the autotuned configuration of this bucket, if any
    const int64_t key = ((int64_t)(1 << next_pow2_bits(ef_cap)) << 16) | (1 << next_pow2_bits(k_max));
    std::lock_guard<std::mutex> lock(idx->tuned_mu);
    for (const auto& tv : idx->tuned)
      if (tv.first == key) {
        opts.query_threads = tv.second.query_threads;
        opts.team_lanes = tv.second.team_lanes;
        opts.stage_bytes = tv.second.stage_bytes;
        if (opts.hash_bits == 0) opts.hash_bits = tv.second.hash_bits;
        if (opts.verify_groups == 0) opts.verify_groups = tv.second.verify_groups;
        break;
      }
  }
  const int width = std::max(1, opts.search_width);
  int deg0 = 0, deg = 0;
  for (auto& G : idx->g)
    if (G.present) {
      deg0 = std::max(deg0, G.deg0);
      deg = std::max(deg, G.deg);
    }
  const bool want_warp = opts.query_threads != kBlock;
  if (next_pow2_bits(4ll * (ef_cap + width * deg0)) > 15)
    return fail(UHNSW_ECAPACITY, "uhnsw_search: visited table too large");
  if (opts.hash_bits != 0 && opts.hash_bits < next_pow2_bits(2ll * (ef_cap + width * deg0)))
    return fail(UHNSW_EINVAL, "uhnsw_search: hash_bits=%d below the minimum %d for beam %d",
                opts.hash_bits, next_pow2_bits(2ll * (ef_cap + width * deg0)), ef_cap);
  const int chunks = idx->d_pad / (idx->tdtype == UHNSW_F32 ? 4 : 8);
  TeamShape sh{0, 0};
  WarpShape wsh{0, 0, 0};
  const bool have_block = pick_shape(idx->tdtype, chunks, &sh);
  const bool few = nq < (int64_t)idx->num_sms * WarpMinBlocks<float>::value * kWarpsPerBlock;
  const bool have_warp = pick_warp_shape(idx->tdtype, chunks, opts.team_lanes, few, &wsh);
  if (want_warp ? !have_warp : !have_block)
    return fail(UHNSW_ECAPACITY, "uhnsw_search: no kernel shape for d=%d", idx->d);
  // warp kernel: the FP32 rows being verified are staged sv at a time (a
  // multiple of the 4 teams of a warp); by default as many as fit in the
  // launch's visited table (the two share one region), 4 to 16
  const int vrow = idx->d_pad * 4;
  const int sv_asked = opts.stage_bytes > 0 ? std::max(4, (opts.stage_bytes / vrow) & ~3) : 0;
  constexpr size_t kSmemMax = 227 * 1024;

  QueryArgs& a = P->a;
  std::memset(&a, 0, sizeof(a));
  a.base32 = idx->base32;
  a.trav = idx->trav;
  a.n = idx->n;
  a.d = idx->d;
  a.d_pad = idx->d_pad;
  a.g[0] = to_dev(idx->g[0]);
  a.g[1] = to_dev(idx->g[1]);
  for (int i = 0; i < 2; ++i) {
    a.gmetric[i] = idx->gmetric[i];
    a.gp[i] = idx->gp[i];
  }
  a.q = q;
  a.p = p;
  a.k = k;
  a.ef = ef;
  a.nq = nq;
  a.k_max = k_max;
  a.ef_default = ef_default;
  a.ef_cap = ef_cap;
  a.t = opts.t;
  a.kappa = opts.kappa;
  a.tau = opts.tau != 0.f ? opts.tau : 0.92f;
  a.tq = opts.t_per_query;
  a.tauq = opts.tau_per_query;
  a.cutoff = opts.cutoff > 0.f ? opts.cutoff : 1.4f;
  a.mode = opts.verify_mode;
  a.width = width;
  // a drop test every 2 groups by default (measured 1 % faster than every
  // group at 1M x 128, ef 52)
  a.vgroups = opts.verify_groups > 0 ? opts.verify_groups : 2;
  a.vcap = 0;
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.stats = opts.stats;
  a.err = idx->err;
  a.trav_exact = idx->trav_exact ? 1 : 0;
  a.queue_head = nullptr;  // set below for a persistent search
  a.sb = 0;
  P->shape = sh;
  P->wshape = wsh;
  P->persistent = opts.persistent != 0;
  if (opts.kernel_events) {
    const cudaEvent_t* ev = static_cast<const cudaEvent_t*>(opts.kernel_events);
    if (!ev[0] || !ev[1]) return fail(UHNSW_EINVAL, "uhnsw_search: kernel_events holds a NULL event");
    P->events[0] = ev[0];
    P->events[1] = ev[1];
  }

  // One launch description for a beam bound: kernel kind, layout, grid.
  auto describe = [&](int bound, Launch* Lo) -> int {
    Lo->a = a;
    Lo->a.ef_cap = bound;
    Lo->a.hash_bits = visited_bits(opts.hash_bits, bound, width, deg0);
    bool w = want_warp;
    for (int attempt = 0; attempt < 2; ++attempt) {
      const int cmax = std::max({width * deg0, deg, w ? 4 : kBlock / 8});
      const int sv = sv_asked > 0 ? sv_asked
                                  : std::min(16, std::max(4, (((1 << Lo->a.hash_bits) * 4) / vrow) & ~3));
      const int stage = w ? sv * vrow : 0;
      const SmemLayout Lw(idx->d_pad, bound, Lo->a.hash_bits, cmax, k_max, 0, stage);
      const size_t smem = w ? (size_t)Lw.total * kWarpsPerBlock : (size_t)Lw.total;
      if (smem <= kSmemMax) {
        Lo->warp = w;
        Lo->smem = smem;
        Lo->a.cmax = cmax;
        Lo->a.stage_bytes = stage;
        Lo->a.sv = w ? sv : 0;
        const int64_t per_block = w ? kWarpsPerBlock : 1;
        Lo->grid = (int)((nq + per_block - 1) / per_block);
        if (P->persistent) {
          const int occ = w ? wsearch_occupancy(idx->tdtype, wsh, smem)
                            : search_occupancy(idx->tdtype, sh, kBlock, smem);
          if (occ < 1) return fail(UHNSW_ECUDA, "uhnsw_search: kernel does not fit (smem %zu)", smem);
          Lo->grid = (int)std::min<int64_t>(Lo->grid, (int64_t)occ * idx->num_sms);
        }
        return UHNSW_OK;
      }
      if (!w || forced || !have_block)
        return fail(UHNSW_ECAPACITY, "uhnsw_search: %zu bytes of shared memory per block", smem);
      w = false;  // the block kernel holds one query per block
    }
    return fail(UHNSW_ECAPACITY, "uhnsw_search: no launch fits");
  };

  P->launches.clear();
  P->bucketed = P->persistent && nq > 0;
  if (P->bucketed) {
    // beam buckets <= 64, 128, 256, 512, capped at ef_cap (one bucket when
    // every query has the same ef)
    P->bb.n = 0;
    if (per_query_beam)
      for (int bound : {64, 128, 256, 512})
        if (bound < ef_cap) P->bb.bound[P->bb.n++] = bound;
    P->bb.bound[P->bb.n++] = ef_cap;
    uhnsw_index::StreamState* qu = nullptr;
    const int rq = queue_for(idx, stream, kBucketOrder + nq, &qu);
    if (rq != UHNSW_OK) return rq;
    P->qhead = qu->head;
    P->qws = qu->ws;
    P->qstate = qu;
    for (int b = P->bb.n - 1; b >= 0; --b) {
      Launch Lb;
      const int rc = describe(P->bb.bound[b], &Lb);
      if (rc != UHNSW_OK) return rc;
      Lb.a.queue_head = qu->head + b;
      Lb.a.qorder = qu->ws + kBucketOrder;
      Lb.a.qbucket = qu->ws + kBucketInfo + 2 * b;
      P->launches.push_back(Lb);
    }
  } else {
    Launch L1;
    const int rc = describe(ef_cap, &L1);
    if (rc != UHNSW_OK) return rc;
    P->launches.push_back(L1);
  }
  P->a = P->launches.front().a;
  return UHNSW_OK;
}

int enqueue_search(uhnsw_index* idx, const Prepared& P, cudaStream_t st) {
  if (P.a.nq == 0) return UHNSW_OK;
  cudaError_t e;
  if (P.bucketed) {
    e = cudaMemsetAsync(P.qhead, 0, 16 * sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: queue reset");
    e = launch_bucketing(P.a, P.bb, P.qws, P.qws + kBucketOrder, P.qws + kBucketInfo, st);
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: bucketing");
  }
  if (P.events[0]) {
    e = cudaEventRecord(P.events[0], st);
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: kernel_events[0]");
  }
  for (const Launch& L : P.launches) {
    e = L.warp ? launch_wsearch(idx->tdtype, P.wshape, L.a, L.grid, L.smem, st)
               : launch_search(idx->tdtype, P.shape, L.a, L.grid, kBlock, L.smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: launch");
  }
  if (P.events[1]) {
    e = cudaEventRecord(P.events[1], st);
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: kernel_events[1]");
  }
  return UHNSW_OK;
}

}  // namespace

extern "C" int uhnsw_search(uhnsw_index* idx, const float* q, const float* p, const int32_t* k,
                            const int32_t* ef, int64_t nq, int32_t k_max, int32_t ef_default,
                            const uhnsw_search_opts* opts, int64_t* out_ids, float* out_dist,
                            void* stream) {
  clear_error();
  Prepared P;
  int rc = prepare_search(idx, q, p, k, ef, nq, k_max, ef_default, opts, out_ids, out_dist, stream,
                          &P);
  if (rc != UHNSW_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // a persistent search's queue reset, ordering and launch stay together on
  // the stream when several host threads search on it
  std::unique_lock<std::mutex> qlock;
  if (P.qstate) qlock = std::unique_lock<std::mutex>(P.qstate->mu);
  // A plain cudaEventRecord inside a stream capture only marks a dependency
  // (it records nothing when the graph runs), so timed calls skip the graph.
  if (!opts || !opts->use_graph || opts->kernel_events || nq == 0)
    return enqueue_search(idx, P, st);

  // CUDA-graph path: capture the launch sequence once per call shape, replay.
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.ptr[0] = q;
  key.ptr[1] = p;
  key.ptr[2] = k;
  key.ptr[3] = ef;
  key.ptr[4] = out_ids;
  key.ptr[5] = out_dist;
  key.ptr[6] = opts->stats;
  key.nq = nq;
  key.k_max = k_max;
  key.ef_default = ef_default;
  key.opts = *opts;
  key.stream = stream;
  std::lock_guard<std::mutex> lock(idx->mu);
  for (auto& ge : idx->graphs)
    if (ge.key == key) {
      cudaError_t e = cudaGraphLaunch(ge.exec, st);
      return e == cudaSuccess ? UHNSW_OK : cuda_fail(e, "uhnsw_search: cudaGraphLaunch");
    }
  cudaStream_t cs = idx->capture_stream;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: begin capture");
  rc = enqueue_search(idx, P, cs);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (rc != UHNSW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_search: instantiate");
  if (idx->graphs.size() >= 16) {
    cudaGraphExecDestroy(idx->graphs.front().exec);
    idx->graphs.erase(idx->graphs.begin());
  }
  idx->graphs.push_back(GraphEntry{key, exec});
  e = cudaGraphLaunch(exec, st);
  return e == cudaSuccess ? UHNSW_OK : cuda_fail(e, "uhnsw_search: cudaGraphLaunch");
}

namespace {

// uhnsw_search_host and uhnsw_search_host_async: the inputs copied into the
// stream's staging, the search, the results copied back, all queued on
// `stream`; `wait` then synchronises the stream.
int search_host_impl(const char* fn, uhnsw_index* idx, const float* q, const float* p,
                     const int32_t* k, const int32_t* ef, int64_t nq, int32_t k_max,
                     int32_t ef_default, const uhnsw_search_opts* opts, int64_t* out_ids,
                     float* out_dist, void* stream, bool wait) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "%s: index is NULL", fn);
  if (nq < 0 || nq > INT32_MAX) return fail(UHNSW_EINVAL, "%s: nq", fn);
  if (nq == 0) return UHNSW_OK;
  if (!q || !p || !out_ids || !out_dist) return fail(UHNSW_EINVAL, "%s: NULL pointer", fn);
  if (k_max < 1 || k_max > UHNSW_MAX_EF) return fail(UHNSW_EINVAL, "%s: k_max", fn);
  const int32_t* ht = opts ? opts->t_per_query : nullptr;    // host arrays here
  const float* htau = opts ? opts->tau_per_query : nullptr;
  const size_t bq = (size_t)nq * idx->d * 4, bp = (size_t)nq * 4, bk = k ? (size_t)nq * 4 : 0,
               be = ef ? (size_t)nq * 4 : 0, bi = (size_t)nq * k_max * 8,
               bd = (size_t)nq * k_max * 4, bt = ht ? (size_t)nq * 4 : 0,
               bta = htau ? (size_t)nq * 4 : 0;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t need = al(bq) + al(bp) + al(bk) + al(be) + al(bi) + al(bd) + al(bt) + al(bta);
  uhnsw_index::StreamState* ss = nullptr;
  int rc = stream_state(idx, stream, &ss);
  if (rc != UHNSW_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(ss->mu);
  if (need > ss->stage_bytes) {
    // the stream's earlier searches may still read the old staging
    cudaError_t e = ss->stage ? cudaStreamSynchronize(st) : cudaSuccess;
    if (e == cudaSuccess) e = cudaFree(ss->stage);
    ss->stage = nullptr;
    ss->stage_bytes = 0;
    if (e == cudaSuccess) e = cudaMalloc(&ss->stage, need);
    if (e != cudaSuccess) return cuda_fail(e, fn, "staging");
    ss->stage_bytes = need;
  }
  char* s = (char*)ss->stage;
  float* dq = (float*)s; s += al(bq);
  float* dp = (float*)s; s += al(bp);
  int32_t* dk = k ? (int32_t*)s : nullptr; s += al(bk);
  int32_t* de = ef ? (int32_t*)s : nullptr; s += al(be);
  int64_t* di = (int64_t*)s; s += al(bi);
  float* dd = (float*)s; s += al(bd);
  int32_t* dt = ht ? (int32_t*)s : nullptr; s += al(bt);
  float* dta = htau ? (float*)s : nullptr;
  Prepared P;
  uhnsw_search_opts o2;
  std::memset(&o2, 0, sizeof(o2));
  if (opts) o2 = *opts;
  o2.use_graph = 0;
  o2.t_per_query = dt;
  o2.tau_per_query = dta;
  rc = prepare_search(idx, dq, dp, dk, de, nq, k_max, ef_default, &o2, di, dd, stream, &P);
  if (rc != UHNSW_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(dq, q, bq, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dp, p, bp, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && k) e = cudaMemcpyAsync(dk, k, bk, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ef) e = cudaMemcpyAsync(de, ef, be, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ht) e = cudaMemcpyAsync(dt, ht, bt, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && htau) e = cudaMemcpyAsync(dta, htau, bta, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, fn, "upload");
  rc = enqueue_search(idx, P, st);
  if (rc != UHNSW_OK) return rc;
  e = cudaMemcpyAsync(out_ids, di, bi, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_dist, dd, bd, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && wait) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, fn, "download");
  return UHNSW_OK;
}

}  // namespace

extern "C" int uhnsw_search_host(uhnsw_index* idx, const float* q, const float* p, const int32_t* k,
                                 const int32_t* ef, int64_t nq, int32_t k_max, int32_t ef_default,
                                 const uhnsw_search_opts* opts, int64_t* out_ids, float* out_dist,
                                 void* stream) {
  return search_host_impl("uhnsw_search_host", idx, q, p, k, ef, nq, k_max, ef_default, opts,
                          out_ids, out_dist, stream, true);
}

extern "C" int uhnsw_search_host_async(uhnsw_index* idx, const float* q, const float* p,
                                       const int32_t* k, const int32_t* ef, int64_t nq,
                                       int32_t k_max, int32_t ef_default,
                                       const uhnsw_search_opts* opts, int64_t* out_ids,
                                       float* out_dist, void* stream) {
  return search_host_impl("uhnsw_search_host_async", idx, q, p, k, ef, nq, k_max, ef_default,
                          opts, out_ids, out_dist, stream, false);
}

extern "C" int uhnsw_verify(uhnsw_index* idx, const float* q, const float* p, const int32_t* cand,
                            int32_t t, int32_t k, int64_t nq, const uhnsw_search_opts* o,
                            int64_t* out_ids, float* out_dist, void* stream) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_verify: index is NULL");
  if (nq < 0 || nq > INT32_MAX) return fail(UHNSW_EINVAL, "uhnsw_verify: nq");
  if (k < 1 || k > UHNSW_MAX_EF) return fail(UHNSW_EINVAL, "uhnsw_verify: k=%d", k);
  if (t < 0 || t > 4096) return fail(UHNSW_EINVAL, "uhnsw_verify: t=%d not in [0, 4096]", t);
  if (nq > 0 && (!q || !p || !out_ids || !out_dist || (t > 0 && !cand)))
    return fail(UHNSW_EINVAL, "uhnsw_verify: NULL pointer");
  uhnsw_search_opts opts;
  std::memset(&opts, 0, sizeof(opts));
  if (o) opts = *o;
  if (opts.verify_mode != UHNSW_VERIFY_EXACT && opts.verify_mode != UHNSW_VERIFY_PAPER)
    return fail(UHNSW_EINVAL, "uhnsw_verify: verify_mode");
  if (opts.kappa < 0 || !std::isfinite(opts.tau)) return fail(UHNSW_EINVAL, "uhnsw_verify: kappa/tau");
  if (opts.verify_groups < 0 || opts.verify_groups > 16)
    return fail(UHNSW_EINVAL, "uhnsw_verify: verify_groups=%d not in [0, 16]", opts.verify_groups);
  if (nq == 0) return UHNSW_OK;
  QueryArgs a;
  std::memset(&a, 0, sizeof(a));
  a.base32 = idx->base32;
  a.n = idx->n;
  a.d = idx->d;
  a.d_pad = idx->d_pad;
  a.q = q;
  a.p = p;
  a.nq = nq;
  a.k_max = k;
  a.kappa = opts.kappa;
  a.tau = opts.tau != 0.f ? opts.tau : 0.92f;
  a.mode = opts.verify_mode;
  a.vgroups = opts.verify_groups > 0 ? opts.verify_groups : 1;
  a.cmax = kBlock / 8;
  a.vcap = std::max(t, 1);
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.stats = opts.stats;
  a.err = idx->err;
  a.cand = cand;
  a.cand_t = t;
  cudaError_t e = launch_wverify(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_verify: launch");
  return UHNSW_OK;
}

extern "C" int uhnsw_exact(uhnsw_index* idx, const float* q, const float* p, int64_t nq, int32_t k,
                           int64_t* out_ids, float* out_dist, void* stream) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_exact: index is NULL");
  if (nq < 0 || nq > INT32_MAX / 2) return fail(UHNSW_EINVAL, "uhnsw_exact: nq");
  if (k < 1 || k > 256) return fail(UHNSW_EINVAL, "uhnsw_exact: k=%d not in [1, 256]", k);
  if (nq > 0 && (!q || !p || !out_ids || !out_dist)) return fail(UHNSW_EINVAL, "uhnsw_exact: NULL pointer");
  if (nq == 0) return UHNSW_OK;
  const int ns = exact_workspace_slices(idx->n, nq, k, idx->num_sms);
  const size_t need = (size_t)ns * nq * k * 8;
  std::lock_guard<std::mutex> lock(idx->mu);
  if (need > idx->exact_ws_bytes) {
    cudaFree(idx->exact_ws);
    idx->exact_ws = nullptr;
    idx->exact_ws_bytes = 0;
    cudaError_t e = cudaMalloc(&idx->exact_ws, need);
    if (e != cudaSuccess) return cuda_fail(e, "uhnsw_exact: workspace");
    idx->exact_ws_bytes = need;
  }
  float* pd = (float*)idx->exact_ws;
  int32_t* pi = (int32_t*)((char*)idx->exact_ws + (size_t)ns * nq * k * 4);
  cudaError_t e = launch_exact(idx->base32, idx->n, idx->d, idx->d_pad, q, p, nq, k, ns, pd, pi,
                               out_ids, out_dist, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_exact: launch");
  return UHNSW_OK;
}

extern "C" int uhnsw_idealized_recall(uhnsw_index* idx, const float* q, const float* p,
                                      int64_t nq, int32_t K, int32_t t_max, float cutoff,
                                      int32_t* counts, void* stream) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_idealized_recall: index is NULL");
  if (nq < 0 || nq > INT32_MAX / 2) return fail(UHNSW_EINVAL, "uhnsw_idealized_recall: nq");
  if (K < 1 || t_max < K || t_max > 256)
    return fail(UHNSW_EINVAL, "uhnsw_idealized_recall: need 1 <= K <= t_max <= 256 (K=%d, t_max=%d)",
                K, t_max);
  if (!(cutoff >= 0.f) || !std::isfinite(cutoff))
    return fail(UHNSW_EINVAL, "uhnsw_idealized_recall: cutoff");
  if (nq > 0 && (!q || !p || !counts)) return fail(UHNSW_EINVAL, "uhnsw_idealized_recall: NULL pointer");
  if (nq == 0) return UHNSW_OK;
  const float cut = cutoff > 0.f ? cutoff : 1.4f;
  const int ns = std::max(exact_workspace_slices(idx->n, nq, K, idx->num_sms),
                          exact_workspace_slices(idx->n, nq, t_max, idx->num_sms));
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t b_ik = (size_t)nq * K * 8, b_dk = (size_t)nq * K * 4;
  const size_t b_it = (size_t)nq * t_max * 8, b_dt = (size_t)nq * t_max * 4;
  const size_t b_pb = (size_t)nq * 4, b_ws = (size_t)ns * nq * t_max * 8;
  const size_t need = al(b_ik) + al(b_dk) + al(b_it) + al(b_dt) + al(b_pb) + al(b_ws);
  char* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, need);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_idealized_recall: scratch");
  char* s = buf;
  int64_t* ik = (int64_t*)s; s += al(b_ik);
  float* dk = (float*)s; s += al(b_dk);
  int64_t* it = (int64_t*)s; s += al(b_it);
  float* dt = (float*)s; s += al(b_dt);
  float* pb = (float*)s; s += al(b_pb);
  float* pd = (float*)s;
  cudaStream_t st = (cudaStream_t)stream;
  const float gp0 = idx->gp[0], gp1 = idx->gp[1];
  // exact L_p top-K, exact base-metric top-t_max, then the curves
  e = launch_exact(idx->base32, idx->n, idx->d, idx->d_pad, q, p, nq, K, ns, pd,
                   (int32_t*)((char*)pd + (size_t)ns * nq * K * 4), ik, dk, st);
  if (e == cudaSuccess) e = launch_base_p(p, nq, gp0, gp1, cut, pb, st);
  if (e == cudaSuccess)
    e = launch_exact(idx->base32, idx->n, idx->d, idx->d_pad, q, pb, nq, t_max, ns, pd,
                     (int32_t*)((char*)pd + (size_t)ns * nq * t_max * 4), it, dt, st);
  if (e == cudaSuccess) e = launch_recall_curve(ik, it, nq, K, t_max, counts, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_idealized_recall: run");
  return UHNSW_OK;
}

extern "C" int uhnsw_plan_t(const int32_t* counts, const float* p, int64_t n, int32_t K,
                            int32_t t_max, float target, float p_lo, float bin_width,
                            int32_t nbins, int32_t* out_t) {
  clear_error();
  if (n < 0 || K < 1 || t_max < K || nbins < 1 || !(bin_width > 0.f) || !(target > 0.f) ||
      !(target <= 1.f) || (n > 0 && (!counts || !p)) || !out_t)
    return fail(UHNSW_EINVAL, "uhnsw_plan_t: bad argument");
  std::vector<double> sum((size_t)nbins * t_max, 0.0);
  std::vector<int64_t> cnt(nbins, 0);
  for (int64_t i = 0; i < n; ++i) {
    // bin b holds p in (p_lo + b w, p_lo + (b + 1) w]; values outside go to the end
    // bins.  A p within 1e-4 bin widths of an upper edge counts as on it, so
    // that FP32 values of grid points (0.6f is above 0.6) fall in their bin.
    int b = (int)std::ceil((double)(p[i] - p_lo) / bin_width - 1e-4) - 1;
    b = std::min(std::max(b, 0), nbins - 1);
    ++cnt[b];
    for (int t = 0; t < t_max; ++t) sum[(size_t)b * t_max + t] += counts[i * t_max + t];
  }
  for (int b = 0; b < nbins; ++b) {
    out_t[b] = 0;
    if (!cnt[b]) continue;
    out_t[b] = t_max;
    for (int t = 0; t < t_max; ++t)
      if (sum[(size_t)b * t_max + t] / ((double)cnt[b] * K) >= (double)target) {
        out_t[b] = t + 1;
        break;
      }
  }
  return UHNSW_OK;
}

// Scratch of uhnsw_exact_static: the per-slice partial top-k lists (distances
// then ids) of one call.  Host code must not take this name's address (it is a
// host-side stand-in); it uses the device address looked up per device below.
static __device__ __align__(256) unsigned char g_exact_static_scratch[UHNSW_EXACT_STATIC_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int uhnsw_exact_static(uhnsw_index* idx, const float* q, const float* p, int64_t nq,
                                  int32_t k, int64_t* out_ids, float* out_dist, void* stream) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_exact_static: index is NULL");
  if (nq < 0 || nq > INT32_MAX / 2) return fail(UHNSW_EINVAL, "uhnsw_exact_static: nq");
  if (k < 1 || k > 256) return fail(UHNSW_EINVAL, "uhnsw_exact_static: k=%d not in [1, 256]", k);
  if (nq > 0 && (!q || !p || !out_ids || !out_dist))
    return fail(UHNSW_EINVAL, "uhnsw_exact_static: NULL pointer");
  const int64_t per_slice = nq * (int64_t)k * 8;
  if (per_slice > (int64_t)UHNSW_EXACT_STATIC_BYTES)
    return fail(UHNSW_ECAPACITY, "uhnsw_exact_static: nq*k*8 = %lld bytes exceeds %d",
                (long long)per_slice, UHNSW_EXACT_STATIC_BYTES);
  if (nq == 0) return UHNSW_OK;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_exact_static: cudaGetDevice");
  if (dev != idx->device)
    return fail(UHNSW_EINVAL, "uhnsw_exact_static: current device %d is not the index's %d", dev,
                idx->device);
  if (dev < 0 || dev >= kMaxDevices)
    return fail(UHNSW_ECAPACITY, "uhnsw_exact_static: device ordinal %d", dev);
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_exact_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "uhnsw_exact_static: cudaGetSymbolAddress");
      g_static_addr[dev] = addr;
    }
    base = g_static_addr[dev];
  }
  int ns = exact_workspace_slices(idx->n, nq, k, idx->num_sms);
  const int64_t fit = (int64_t)UHNSW_EXACT_STATIC_BYTES / per_slice;
  if (ns > fit) ns = (int)fit;
  float* pd = (float*)base;
  int32_t* pi = (int32_t*)((char*)base + (size_t)ns * nq * k * 4);
  e = launch_exact(idx->base32, idx->n, idx->d, idx->d_pad, q, p, nq, k, ns, pd, pi, out_ids,
                   out_dist, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_exact_static: launch");
  return UHNSW_OK;
}

int64_t uhnsw_internal::query_state_bytes(const uhnsw_index* idx, int32_t ef, int32_t k,
                                          const uhnsw_search_opts* o) {
  if (!idx || ef < 1 || k < 1) return fail(UHNSW_EINVAL, "query_state_bytes: bad argument");
  uhnsw_search_opts opts;
  std::memset(&opts, 0, sizeof(opts));
  if (o) opts = *o;
  const bool warp = opts.query_threads != kBlock;
  const int width = std::max(1, opts.search_width);
  int deg0 = 0, deg = 0;
  for (auto& G : idx->g)
    if (G.present) {
      deg0 = std::max(deg0, G.deg0);
      deg = std::max(deg, G.deg);
    }
  const int efp = std::max(ef, k);
  const int cmax = std::max({width * deg0, deg, warp ? 4 : kBlock / 8});
  const int hb = visited_bits(opts.hash_bits, efp, width, deg0);
  int stage = 0;
  if (warp) {
    const int vrow = idx->d_pad * 4;
    stage = std::max(4, (opts.stage_bytes > 0 ? opts.stage_bytes / vrow : 4) & ~3) * vrow;
  }
  return SmemLayout(idx->d_pad, efp, hb, cmax, k, 0, stage).total;
}

extern "C" int uhnsw_autotune(uhnsw_index* idx, const float* q, const float* p, int64_t nq,
                              int32_t k, int32_t ef, const uhnsw_search_opts* base, void* stream,
                              uhnsw_search_opts* best, float* best_ms) {
  clear_error();
  if (!idx || !q || !p || nq < 1 || k < 1 || ef < 1)
    return fail(UHNSW_EINVAL, "uhnsw_autotune: bad argument");
  uhnsw_search_opts b;
  std::memset(&b, 0, sizeof(b));
  if (base) b = *base;
  b.stats = nullptr;
  b.use_graph = 0;
  const int efp = std::max({ef, k, b.t});
  if (efp > UHNSW_MAX_EF) return fail(UHNSW_EINVAL, "uhnsw_autotune: beam %d", efp);
  const int chunks = idx->d_pad / (idx->tdtype == UHNSW_F32 ? 4 : 8);
  std::vector<uhnsw_search_opts> cands;
  int deg0 = 0;
  for (auto& G : idx->g)
    if (G.present) deg0 = std::max(deg0, G.deg0);
  const int width = std::max(1, b.search_width);
  const int hb_def = visited_bits(0, efp, width, deg0);
  // the caller's table size and drop-test interval are kept; otherwise the
  // default table and one twice as large, and a drop test every 1, 2 or 4
  // groups (none of them changes a result)
  std::vector<int> hbs, vgs;
  if (b.hash_bits > 0) hbs = {b.hash_bits};
  else if (hb_def < 15) hbs = {0, hb_def + 1};
  else hbs = {0};
  if (b.verify_groups > 0) vgs = {b.verify_groups};
  else vgs = {1, 2, 4};
  for (int team : {4, 8, 16, 32}) {
    WarpShape ws;
    if (!pick_warp_shape(idx->tdtype, chunks, team, false, &ws)) continue;
    for (int rows : {4, 8, 16})
      for (int hb : hbs)
        for (int vg : vgs) {
          uhnsw_search_opts c = b;
          c.query_threads = 32;
          c.team_lanes = team;
          c.stage_bytes = rows * idx->d_pad * 4;
          c.hash_bits = hb;
          c.verify_groups = vg;
          cands.push_back(c);
        }
  }
  for (int hb : hbs) {  // (the block kernel tests after every group: no interval to try)
    uhnsw_search_opts c = b;
    c.query_threads = kBlock;
    c.team_lanes = 0;
    c.stage_bytes = 0;
    c.hash_bits = hb;
    cands.push_back(c);
  }
  int64_t* ids = nullptr;
  float* dist = nullptr;
  cudaError_t e = cudaMalloc(&ids, nq * k * 8);
  if (e == cudaSuccess) e = cudaMalloc(&dist, nq * k * 4);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaFree(ids);
    cudaFree(dist);
    return cuda_fail(e, "uhnsw_autotune: setup");
  }
  cudaStream_t st = (cudaStream_t)stream;
  float best_t = 1e30f;
  int best_i = -1;
  int rc = UHNSW_OK;
  for (size_t i = 0; i < cands.size() && rc == UHNSW_OK; ++i) {
    float ts[3];
    for (int r = 0; r < 4 && rc == UHNSW_OK; ++r) {
      cudaEventRecord(e0, st);
      rc = uhnsw_search(idx, q, p, nullptr, nullptr, nq, k, efp, &cands[i], ids, dist, stream);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      if (rc == UHNSW_OK && e != cudaSuccess) rc = cuda_fail(e, "uhnsw_autotune: run");
      if (rc == UHNSW_OK && r > 0) cudaEventElapsedTime(&ts[r - 1], e0, e1);
    }
    if (rc == UHNSW_ECAPACITY) {  // this configuration does not fit: skip it
      clear_error();
      rc = UHNSW_OK;
      continue;
    }
    if (rc != UHNSW_OK) break;
    std::sort(ts, ts + 3);
    if (ts[1] < best_t) {
      best_t = ts[1];
      best_i = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(ids);
  cudaFree(dist);
  if (rc != UHNSW_OK) return rc;
  if (best_i < 0) return fail(UHNSW_ECAPACITY, "uhnsw_autotune: no configuration fits");
  const int64_t key = ((int64_t)(1 << next_pow2_bits(efp)) << 16) | (1 << next_pow2_bits(k));
  {
    std::lock_guard<std::mutex> lock(idx->tuned_mu);
    bool found = false;
    for (auto& tv : idx->tuned)
      if (tv.first == key) {
        tv.second = cands[best_i];
        found = true;
      }
    if (!found) idx->tuned.emplace_back(key, cands[best_i]);
  }
  if (best) *best = cands[best_i];
  if (best_ms) *best_ms = best_t;
  return UHNSW_OK;
}

extern "C" int uhnsw_autotune_save(const uhnsw_index* idx, const char* path) {
  clear_error();
  if (!idx || !path) return fail(UHNSW_EINVAL, "uhnsw_autotune_save: NULL argument");
  FILE* f = fopen(path, "w");
  if (!f) return fail(UHNSW_EINVAL, "uhnsw_autotune_save: cannot open %s", path);
  std::lock_guard<std::mutex> lock(const_cast<uhnsw_index*>(idx)->tuned_mu);
  for (const auto& tv : idx->tuned)
    fprintf(f, "%d %d %lld %lld %d %d %d %d %d\n", (int)idx->tdtype, idx->d,
            (long long)(tv.first >> 16), (long long)(tv.first & 0xffff), tv.second.query_threads,
            tv.second.team_lanes, tv.second.stage_bytes, tv.second.hash_bits,
            tv.second.verify_groups);
  fclose(f);
  return UHNSW_OK;
}

extern "C" int uhnsw_autotune_load(uhnsw_index* idx, const char* path) {
  clear_error();
  if (!idx || !path) return fail(UHNSW_EINVAL, "uhnsw_autotune_load: NULL argument");
  FILE* f = fopen(path, "r");
  if (!f) return fail(UHNSW_EINVAL, "uhnsw_autotune_load: cannot open %s", path);
  int dt, d, qt, team, stage;
  long long efb, kb;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    int hb = 0, vg = 0;
    const int got = sscanf(line, "%d %d %lld %lld %d %d %d %d %d", &dt, &d, &efb, &kb, &qt, &team,
                           &stage, &hb, &vg);
    if (got != 7 && got != 9) continue;
    if (dt != (int)idx->tdtype || d != idx->d) continue;
    if ((qt != 32 && qt != kBlock) || (team != 0 && team != 8 && team != 16 && team != 32) ||
        stage < 0 || stage > 64 * 1024 || efb < 1 || kb < 1 || hb < 0 || hb > 15 || vg < 0 ||
        vg > 16)
      continue;
    uhnsw_search_opts o;
    std::memset(&o, 0, sizeof(o));
    o.query_threads = qt;
    o.team_lanes = team;
    o.stage_bytes = stage;
    o.hash_bits = hb;
    o.verify_groups = vg;
    const int64_t key = (efb << 16) | kb;
    std::lock_guard<std::mutex> lock(idx->tuned_mu);
    bool found = false;
    for (auto& tv : idx->tuned)
      if (tv.first == key) {
        tv.second = o;
        found = true;
      }
    if (!found) idx->tuned.emplace_back(key, o);
  }
  fclose(f);
  return UHNSW_OK;
}

extern "C" int uhnsw_index_info(const uhnsw_index* idx, int64_t* n, int32_t* d, int32_t* d_pad,
                                int64_t* device_bytes, int32_t* max_degree0) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_index_info: index is NULL");
  if (n) *n = idx->n;
  if (d) *d = idx->d;
  if (d_pad) *d_pad = idx->d_pad;
  if (device_bytes) *device_bytes = idx->bytes;
  if (max_degree0) *max_degree0 = std::max(idx->g[0].deg0, idx->g[1].deg0);
  return UHNSW_OK;
}

extern "C" int uhnsw_device_status(uhnsw_index* idx) {
  clear_error();
  if (!idx) return fail(UHNSW_EINVAL, "uhnsw_device_status: index is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_device_status: synchronize");
  int32_t v[4] = {0, 0, 0, 0};
  e = cudaMemcpy(v, idx->err, 16, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(idx->err, 0, 16);
  if (e != cudaSuccess) return cuda_fail(e, "uhnsw_device_status: read");
  if (v[0] != 0)
    return fail(v[0], "uhnsw_device_status: device recorded error %d (site %d, value %d, limit %d)",
                v[0], v[1], v[2], v[3]);
  return UHNSW_OK;
}

extern "C" void uhnsw_free(uhnsw_index* idx) { delete idx; }
