// Host-side HNSW construction (Section 2.2: G1 is built under L1, G2 under
// L2, by incremental insertion with M links per node and an
// efConstruction-wide insertion beam).  It follows the published HNSW
// insertion: greedy descent (beam 1) above the node's level, then at each
// level a beam search of width efConstruction, the neighbour-selection
// heuristic (a candidate is kept only if it is strictly nearer to the new node
// than to every neighbour already kept), bidirectional links, and heuristic
// re-selection of a neighbour's list when it exceeds its cap (2M at layer 0,
// M above).  The beam of the next level starts from the whole result of the
// level above.
//
// Order everywhere: (distance, id) lexicographic.  Distances are FP32; on
// integer-valued data (and data on a coarse binary grid) L1 and squared-L2
// sums are exact in FP32, so a single-threaded build is reproducible bit for
// bit.  With several threads, nodes are inserted concurrently under per-node
// spin locks, as usual for parallel HNSW builds; the graph then depends on
// thread timing but keeps every structural invariant.
//
// This file is not on the query path: it produces the CSR graphs that
// uhnsw_load consumes.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <queue>
#include <thread>
#include <vector>

#include "uhnsw.h"
#include "uhnsw_internal.h"

namespace {

struct DI {
  float d;
  int32_t id;
};
inline bool di_less(const DI& a, const DI& b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }
struct DIWorstOnTop {  // max-heap by (d, id)
  bool operator()(const DI& a, const DI& b) const { return di_less(a, b); }
};
struct DIBestOnTop {  // min-heap by (d, id)
  bool operator()(const DI& a, const DI& b) const { return di_less(b, a); }
};

typedef float v4f __attribute__((vector_size(16)));

inline v4f load4(const float* p) {
  v4f v;
  std::memcpy(&v, p, sizeof(v));
  return v;
}

// Base metric in FP32: metric 1 -> sum |d_j|, metric 2 -> sum d_j^2,
// metric 3 -> sum |d_j|^(1/2) (the L0.5 graph of U-HNSW-E, Section 4.5),
// metric 4 -> sum |d_j|^(3/2) (an L1.5 graph, Section 4.3's fixed-p HNSW),
// metric 5 -> sum |d_j|^bp (the fixed-p HNSW at any other p).
// Four independent 4-wide partial sums, then a fixed combination order; the
// same for every call, so the build is reproducible on one machine.
float base_distance(const float* a, const float* b, int32_t d, int32_t metric, float bp) {
  v4f s0 = {0, 0, 0, 0}, s1 = s0, s2 = s0, s3 = s0;
  int32_t j = 0;
  if (metric == 1) {
    for (; j + 16 <= d; j += 16) {
      v4f x0 = load4(a + j) - load4(b + j), x1 = load4(a + j + 4) - load4(b + j + 4);
      v4f x2 = load4(a + j + 8) - load4(b + j + 8), x3 = load4(a + j + 12) - load4(b + j + 12);
      for (int u = 0; u < 4; ++u) {
        s0[u] += std::fabs(x0[u]);
        s1[u] += std::fabs(x1[u]);
        s2[u] += std::fabs(x2[u]);
        s3[u] += std::fabs(x3[u]);
      }
    }
  } else if (metric == 3 || metric == 4) {
    for (; j + 16 <= d; j += 16) {
      v4f x0 = load4(a + j) - load4(b + j), x1 = load4(a + j + 4) - load4(b + j + 4);
      v4f x2 = load4(a + j + 8) - load4(b + j + 8), x3 = load4(a + j + 12) - load4(b + j + 12);
      for (int u = 0; u < 4; ++u) {
        const float a0 = std::fabs(x0[u]), a1 = std::fabs(x1[u]);
        const float a2 = std::fabs(x2[u]), a3 = std::fabs(x3[u]);
        s0[u] += metric == 3 ? std::sqrt(a0) : a0 * std::sqrt(a0);
        s1[u] += metric == 3 ? std::sqrt(a1) : a1 * std::sqrt(a1);
        s2[u] += metric == 3 ? std::sqrt(a2) : a2 * std::sqrt(a2);
        s3[u] += metric == 3 ? std::sqrt(a3) : a3 * std::sqrt(a3);
      }
    }
  } else if (metric == UHNSW_BASE_LP) {
    for (; j + 16 <= d; j += 16) {
      v4f x0 = load4(a + j) - load4(b + j), x1 = load4(a + j + 4) - load4(b + j + 4);
      v4f x2 = load4(a + j + 8) - load4(b + j + 8), x3 = load4(a + j + 12) - load4(b + j + 12);
      for (int u = 0; u < 4; ++u) {
        s0[u] += std::pow(std::fabs(x0[u]), bp);
        s1[u] += std::pow(std::fabs(x1[u]), bp);
        s2[u] += std::pow(std::fabs(x2[u]), bp);
        s3[u] += std::pow(std::fabs(x3[u]), bp);
      }
    }
  } else {
    for (; j + 16 <= d; j += 16) {
      v4f x0 = load4(a + j) - load4(b + j), x1 = load4(a + j + 4) - load4(b + j + 4);
      v4f x2 = load4(a + j + 8) - load4(b + j + 8), x3 = load4(a + j + 12) - load4(b + j + 12);
      s0 += x0 * x0;
      s1 += x1 * x1;
      s2 += x2 * x2;
      s3 += x3 * x3;
    }
  }
  v4f s = (s0 + s1) + (s2 + s3);
  float r = (s[0] + s[1]) + (s[2] + s[3]);
  for (; j < d; ++j) {
    float x = a[j] - b[j];
    const float a = std::fabs(x);
    r += metric == 1 ? a : metric == 3 ? std::sqrt(a) : metric == 4 ? a * std::sqrt(a)
         : metric == UHNSW_BASE_LP ? std::pow(a, bp) : x * x;
  }
  return r;
}

struct SpinLock {
  std::atomic<uint8_t> f{0};
  void lock() {
    while (f.exchange(1, std::memory_order_acquire)) {
      while (f.load(std::memory_order_relaxed)) std::this_thread::yield();
    }
  }
  void unlock() { f.store(0, std::memory_order_release); }
};

struct Visited {
  std::vector<uint16_t> mark;
  uint16_t gen = 0;
  explicit Visited(int64_t n) : mark(n, 0) {}
  void next() {
    if (++gen == 0) {
      std::fill(mark.begin(), mark.end(), 0);
      gen = 1;
    }
  }
  bool test_set(int32_t v) {
    if (mark[v] == gen) return true;
    mark[v] = gen;
    return false;
  }
};

struct Builder {
  int64_t n;
  int32_t d, metric, M, M0, efc;
  float bp = 0.f;                // the p of metric 5
  const float* base;
  std::vector<int32_t> level;
  std::vector<int32_t> links0;   // n x (M0 + 1): count, ids
  std::vector<int64_t> up_off;   // first upper row of node v (levels 1..level[v]), -1 if none
  std::vector<int32_t> links_up; // rows x (M + 1)
  std::unique_ptr<SpinLock[]> locks;
  std::mutex global;
  int32_t entry = 0;
  int32_t max_level = 0;

  int32_t* row(int32_t v, int32_t l) {
    if (l == 0) return &links0[(int64_t)v * (M0 + 1)];
    return &links_up[(up_off[v] + l - 1) * (int64_t)(M + 1)];
  }
  const float* vec(int32_t v) const { return base + (int64_t)v * d; }
  float dist(const float* x, int32_t v) const { return base_distance(x, vec(v), d, metric, bp); }

  // SEARCH-LAYER from the entry set `ep` (distances known) with beam `ef` at
  // level lc; returns the result set ascending by (d, id).
  void search_layer(const float* x, const std::vector<DI>& ep, int32_t ef, int32_t lc, Visited& vis,
                    std::vector<DI>& out, std::vector<int32_t>& nb_buf) {
    std::priority_queue<DI, std::vector<DI>, DIBestOnTop> C;
    std::priority_queue<DI, std::vector<DI>, DIWorstOnTop> W;
    vis.next();
    for (const DI& e : ep) {
      vis.test_set(e.id);
      C.push(e);
      W.push(e);
      if ((int32_t)W.size() > ef) W.pop();
    }
    const int32_t cap = lc == 0 ? M0 : M;
    nb_buf.resize(cap);
    while (!C.empty()) {
      DI c = C.top();
      C.pop();
      if (di_less(W.top(), c)) break;
      int32_t cnt;
      {
        std::lock_guard<SpinLock> g(locks[c.id]);
        const int32_t* r = row(c.id, lc);
        cnt = r[0];
        std::memcpy(nb_buf.data(), r + 1, sizeof(int32_t) * cnt);
      }
      for (int32_t a = 0; a < cnt; ++a) {
        if (a + 1 < cnt) __builtin_prefetch(vec(nb_buf[a + 1]));
        int32_t e = nb_buf[a];
        if (vis.test_set(e)) continue;
        DI de{dist(x, e), e};
        if ((int32_t)W.size() < ef || di_less(de, W.top())) {
          C.push(de);
          W.push(de);
          if ((int32_t)W.size() > ef) W.pop();
        }
      }
    }
    out.resize(W.size());
    for (int64_t i = (int64_t)W.size() - 1; i >= 0; --i) {
      out[i] = W.top();
      W.pop();
    }
  }

  // Neighbour-selection heuristic over `cand` ascending by distance to the
  // base point: keep e only if it is strictly nearer to the base point than
  // to every element already kept; at most m.
  int32_t select(const std::vector<DI>& cand, int32_t m, int32_t* out) const {
    int32_t r = 0;
    for (size_t i = 0; i < cand.size() && r < m; ++i) {
      const DI& e = cand[i];
      bool keep = true;
      for (int32_t j = 0; j < r; ++j) {
        if (!(e.d < base_distance(vec(e.id), vec(out[j]), d, metric, bp))) {
          keep = false;
          break;
        }
      }
      if (keep) out[r++] = e.id;
    }
    return r;
  }

  void insert(int32_t q, Visited& vis, std::vector<DI>& W, std::vector<DI>& ep,
              std::vector<DI>& tmp, std::vector<int32_t>& nb_buf, std::vector<int32_t>& sel) {
    const int32_t l = level[q];
    std::unique_lock<std::mutex> glock(global);
    int32_t L = max_level;
    int32_t cur = entry;
    if (l <= L) glock.unlock();  // only a new top node holds the lock throughout
    const float* x = vec(q);
    ep.assign(1, DI{dist(x, cur), cur});
    for (int32_t lc = L; lc > l; --lc) {
      search_layer(x, ep, 1, lc, vis, W, nb_buf);
      ep.assign(1, W[0]);
    }
    for (int32_t lc = std::min(L, l); lc >= 0; --lc) {
      search_layer(x, ep, efc, lc, vis, W, nb_buf);
      sel.resize(std::max(M, M0) + 1);
      int32_t r = select(W, M, sel.data());
      {
        std::lock_guard<SpinLock> g(locks[q]);
        int32_t* rq = row(q, lc);
        rq[0] = r;
        std::memcpy(rq + 1, sel.data(), sizeof(int32_t) * r);
      }
      const int32_t mmax = lc == 0 ? M0 : M;
      std::vector<int32_t> mine(sel.begin(), sel.begin() + r);
      for (int32_t e : mine) {
        std::lock_guard<SpinLock> g(locks[e]);
        int32_t* re = row(e, lc);
        int32_t cnt = re[0];
        if (cnt < mmax) {
          re[1 + cnt] = q;
          re[0] = cnt + 1;
          continue;
        }
        // e would exceed its cap: re-select among its links plus q
        tmp.clear();
        const float* xe = vec(e);
        for (int32_t a = 0; a < cnt; ++a) tmp.push_back(DI{dist(xe, re[1 + a]), re[1 + a]});
        tmp.push_back(DI{dist(xe, q), q});
        std::sort(tmp.begin(), tmp.end(), di_less);
        int32_t keep[UHNSW_MAX_DEGREE + 1];
        int32_t rr = select(tmp, mmax, keep);
        re[0] = rr;
        std::memcpy(re + 1, keep, sizeof(int32_t) * rr);
      }
      ep = W;
    }
    if (l > L) {
      entry = q;
      max_level = l;
    }
  }
};

}  // namespace

struct uhnsw_built {
  int32_t num_levels = 0;
  int32_t entry = 0;
  int32_t M = 0, M0 = 0;
  int64_t n = 0;
  std::vector<int32_t> count;
  std::vector<std::vector<int32_t>> nodes;
  std::vector<std::vector<int64_t>> offsets;
  std::vector<std::vector<int32_t>> nbrs;
};

namespace {

int build_host(const float* base, int64_t n, int32_t d, int32_t metric, float bp, int32_t M,
               int32_t ef_construction, const int32_t* levels, int32_t threads,
               uhnsw_built** out) {
  if (!base || !levels || n < 1 || n > INT32_MAX || d < 1 || d > UHNSW_MAX_DIM)
    return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph: bad base/levels/n/d");
  if (M < 2 || 2 * M > UHNSW_MAX_DEGREE || ef_construction < 1)
    return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph: need 2 <= M <= %d, efc >= 1",
                                UHNSW_MAX_DEGREE / 2);
  for (int64_t i = 0; i < n; ++i)
    if (levels[i] < 0 || levels[i] >= UHNSW_MAX_LEVELS)
      return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph: level of node %lld is %d",
                                  (long long)i, levels[i]);
  try {
    Builder B;
    B.n = n;
    B.d = d;
    B.metric = metric;
    B.bp = bp;
    B.M = M;
    B.M0 = 2 * M;
    B.efc = ef_construction;
    B.base = base;
    B.level.assign(levels, levels + n);
    B.links0.assign(n * (int64_t)(B.M0 + 1), 0);
    B.up_off.assign(n, -1);
    int64_t rows = 0;
    for (int64_t v = 0; v < n; ++v)
      if (levels[v] > 0) {
        B.up_off[v] = rows;
        rows += levels[v];
      }
    B.links_up.assign(rows * (int64_t)(M + 1), 0);
    B.locks.reset(new SpinLock[n]);
    B.entry = 0;
    B.max_level = levels[0];

    int32_t nt = threads > 0 ? threads : (int32_t)std::max(1u, std::thread::hardware_concurrency());
    std::atomic<int64_t> next(1);
    auto work = [&]() {
      Visited vis(n);
      std::vector<DI> W, ep, tmp;
      std::vector<int32_t> nb_buf, sel;
      for (;;) {
        int64_t q = next.fetch_add(1);
        if (q >= n) break;
        B.insert((int32_t)q, vis, W, ep, tmp, nb_buf, sel);
      }
    };
    if (nt == 1) {
      work();
    } else {
      std::vector<std::thread> pool;
      for (int32_t i = 0; i < nt; ++i) pool.emplace_back(work);
      for (auto& th : pool) th.join();
    }

    auto* g = new uhnsw_built();
    g->n = n;
    g->M = M;
    g->M0 = B.M0;
    g->num_levels = B.max_level + 1;
    g->entry = B.entry;
    g->count.assign(g->num_levels, 0);
    g->nodes.resize(g->num_levels);
    g->offsets.resize(g->num_levels);
    g->nbrs.resize(g->num_levels);
    for (int32_t l = 0; l < g->num_levels; ++l) {
      auto& off = g->offsets[l];
      auto& nb = g->nbrs[l];
      off.push_back(0);
      for (int64_t v = 0; v < n; ++v) {
        if (levels[v] < l) continue;
        if (l > 0) g->nodes[l].push_back((int32_t)v);
        const int32_t* r = B.row((int32_t)v, l);
        nb.insert(nb.end(), r + 1, r + 1 + r[0]);
        off.push_back((int64_t)nb.size());
      }
      g->count[l] = (int32_t)(off.size() - 1);
    }
    *out = g;
    return UHNSW_OK;
  } catch (const std::bad_alloc&) {
    return uhnsw_internal::fail(UHNSW_EOOM, "uhnsw_build_graph: out of host memory");
  }
}

}  // namespace

extern "C" int uhnsw_build_graph(const float* base, int64_t n, int32_t d, int32_t metric,
                                 int32_t M, int32_t ef_construction, const int32_t* levels,
                                 int32_t threads, uhnsw_built** out) {
  uhnsw_internal::clear_error();
  if (!out) return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph: out is NULL");
  *out = nullptr;
  if (metric < 1 || metric > 4)
    return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph: metric must be 1, 2, 3 or 4");
  return build_host(base, n, d, metric, 0.f, M, ef_construction, levels, threads, out);
}

extern "C" int uhnsw_build_graph_lp(const float* base, int64_t n, int32_t d, float p, int32_t M,
                                    int32_t ef_construction, const int32_t* levels,
                                    int32_t threads, int32_t on_device, uhnsw_built** out) {
  uhnsw_internal::clear_error();
  if (!out) return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph_lp: out is NULL");
  *out = nullptr;
  if (!(p > 0.f && p <= 2.f))
    return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_build_graph_lp: p=%g outside (0, 2]",
                                (double)p);
  const int32_t metric = uhnsw_internal::base_metric_of_p(p);
  if (on_device)
    return uhnsw_internal::build_graph_gpu(base, n, d, metric, p, M, ef_construction, levels, out);
  return build_host(base, n, d, metric, p, M, ef_construction, levels, threads, out);
}

namespace uhnsw_internal {
// CSR graph from the padded adjacency tables the GPU builder leaves.
uhnsw_built* make_built(int64_t n, int32_t M, int32_t M0, const int32_t* levels, int32_t entry,
                        int32_t top, const int32_t* ell0, const int32_t* up_off,
                        const int32_t* up_adj) {
  auto* g = new (std::nothrow) uhnsw_built();
  if (!g) return nullptr;
  try {
    g->n = n;
    g->M = M;
    g->M0 = M0;
    g->num_levels = top + 1;
    g->entry = entry;
    g->count.assign(g->num_levels, 0);
    g->nodes.resize(g->num_levels);
    g->offsets.resize(g->num_levels);
    g->nbrs.resize(g->num_levels);
    for (int32_t l = 0; l < g->num_levels; ++l) {
      auto& off = g->offsets[l];
      auto& nb = g->nbrs[l];
      off.push_back(0);
      const int32_t cap = l == 0 ? M0 : M;
      for (int64_t v = 0; v < n; ++v) {
        if (levels[v] < l) continue;
        if (l > 0) g->nodes[l].push_back((int32_t)v);
        const int32_t* r = l == 0 ? ell0 + v * M0 : up_adj + ((int64_t)up_off[v] + l - 1) * M;
        for (int32_t j = 0; j < cap && r[j] >= 0; ++j) nb.push_back(r[j]);
        off.push_back((int64_t)nb.size());
      }
      g->count[l] = (int32_t)(off.size() - 1);
    }
  } catch (const std::bad_alloc&) {
    delete g;
    return nullptr;
  }
  return g;
}
}  // namespace uhnsw_internal

extern "C" int uhnsw_built_graph(const uhnsw_built* b, uhnsw_graph* view) {
  uhnsw_internal::clear_error();
  if (!b || !view) return uhnsw_internal::fail(UHNSW_EINVAL, "uhnsw_built_graph: NULL argument");
  std::memset(view, 0, sizeof(*view));
  view->num_levels = b->num_levels;
  view->entry_point = b->entry;
  view->max_degree0 = b->M0;
  view->max_degree = b->M;
  view->level_count = b->count.data();
  for (int32_t l = 0; l < b->num_levels; ++l) {
    view->level_nodes[l] = l == 0 ? nullptr : b->nodes[l].data();
    view->level_offsets[l] = b->offsets[l].data();
    view->level_nbrs[l] = b->nbrs[l].data();
  }
  return UHNSW_OK;
}

extern "C" void uhnsw_built_free(uhnsw_built* b) { delete b; }
