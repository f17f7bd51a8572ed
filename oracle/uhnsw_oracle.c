/*
 * U-HNSW oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the U-HNSW query
 * path computes (arxiv 2605.02030, "U-HNSW: An Efficient Graph-based Solution
 * to ANNS Under Universal L_p Metrics"), written for obviously-correct
 * reading, not speed.  Every distance is evaluated in FP64 from the FP32
 * inputs.  Only the tests, the package's smoke check and the bench's CPU
 * baseline leg may load this library; the GPU path never links or calls it
 * and shares no code, header or table with it.
 *
 * Contents and the passage each part follows:
 *   oracle_lp_sum         S = sum_j |x_j - q_j|^p               (Section 2.1)
 *   oracle_exact_knn      exact top-K under L_p (the recall ground truth;
 *                         problem statement of Sections 1.1 and 2.1,
 *                         recall of Section 4.1.2)
 *   oracle_hnsw_build     HNSW construction under L1 (G1) or L2 (G2)
 *                         (Section 2.2; the published HNSW insertion,
 *                         Malkov & Yashunin, Algorithms 1, 2 and 4).
 *                         Pinned by hand-derived graphs and, at
 *                         efConstruction >= N, by brute-force insertion
 *                         (every reachable earlier node ranked); below that
 *                         the graph follows the beam, pinned on its own.
 *   oracle_hnsw_build_p   the same construction under any L_bp, 0 < bp <= 2
 *                         (the fixed-p HNSW of Section 4.3, one graph per p)
 *   oracle_hnsw_search    KnnSearch(q, t) on a CSR graph (Section 2.2 and
 *                         Section 3.1 "Candidate generation"; HNSW
 *                         Algorithms 2 and 5); oracle_hnsw_search_p under
 *                         any L_bp
 *   oracle_verify_exact   top-K by L_p over the whole candidate set C, with
 *                         or without abandoning a candidate whose partial
 *                         sum exceeds the running K-th best sum
 *   oracle_verify_paper   Algorithm 1, lines 6-10: batches of kappa with the
 *                         |R_new ∩ R| / K >= tau early stop (Section 3.1)
 *   oracle_hnsw_search_w  KnnSearch whose layer-0 beam expands `width`
 *                         entries per step: the GPU's fast mode, a GPU
 *                         adaptation (width = 1 is HNSW's own order)
 *   oracle_uhnsw_query    Algorithm 1 end to end, with the p <= cutoff
 *                         routing (Section 3.1) and the direct K-NN for
 *                         p in {1, 2} (Section 3 introduction); with graphs
 *                         under L0.5 and L1 and cutoff 0.6 it is U-HNSW-E
 *                         (Section 4.5), whose direct K-NN is for p in
 *                         {0.5, 1}; oracle_uhnsw_query_p takes the two
 *                         graphs' p instead of metric codes, and
 *                         oracle_uhnsw_query_w a search width as well
 *   oracle_uhnsw_query_trav  the same with the search on a rounded copy
 *                         of the rows (the FP16 / BF16 precision form) and
 *                         verification on the FP32 rows, counting the
 *                         search's near-tie comparisons
 *
 * Order used everywhere: lexicographic (distance, id), ids ascending on ties.
 * Base metrics (metric codes): 1 = L1, sum |d_j|; 2 = the squared L2 sum
 * d_j^2, which orders points exactly like L2; 3 = L0.5 without its root,
 * sum |d_j|^(1/2), which orders points exactly like L0.5; 4 = L1.5 without
 * its root, sum |d_j|^(3/2) (the fixed-p HNSW graph of Section 4.3 at
 * p = 1.5, where the paper finds plain HNSW faster).  The _p entry points
 * take the base p itself: a graph built under L_bp is built and searched
 * with S_bp = sum |d_j|^bp, which orders points exactly like L_bp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

/* ------------------------------------------------------------------ */
/* Distances (Section 2.1)                                             */
/* ------------------------------------------------------------------ */

/* S = sum_j |x_j - q_j|^p in FP64 (no root). */
double oracle_lp_sum(const float* x, const float* q, int32_t d, double p) {
  double s = 0.0;
  for (int32_t j = 0; j < d; ++j) {
    double diff = fabs((double)x[j] - (double)q[j]);
    s += pow(diff, p);
  }
  return s;
}

/* The base metric of a graph built under L_bp: S_bp = sum_j |d_j|^bp, with
 * the closed forms of p = 1, 2, 0.5 and 1.5 written out and pow() for any
 * other bp.  Every graph is built and searched with the S of its own bp. */
static double base_dist_p(const float* x, const float* q, int32_t d, double bp) {
  double s = 0.0;
  for (int32_t j = 0; j < d; ++j) {
    double diff = (double)x[j] - (double)q[j];
    double a = fabs(diff);
    if (bp == 1.0) s += a;
    else if (bp == 2.0) s += diff * diff;
    else if (bp == 0.5) s += sqrt(a);
    else if (bp == 1.5) s += a * sqrt(a);
    else s += pow(a, bp);
  }
  return s;
}

/* The p of a base metric code, and whether the code is one. */
static double metric_p(int32_t metric) {
  return metric == 1 ? 1.0 : metric == 2 ? 2.0 : metric == 3 ? 0.5 : 1.5;
}
static int valid_metric(int32_t metric) { return metric >= 1 && metric <= 4; }
static int valid_bp(double bp) { return bp > 0.0 && bp <= 2.0; }

/* Base metric by code: metric 1 -> L1 sum |d_j|; metric 2 -> squared L2 sum
 * d_j^2; metric 3 -> L0.5 sum |d_j|^(1/2); metric 4 -> L1.5 sum |d_j|^(3/2). */
double oracle_base_dist(const float* x, const float* q, int32_t d, int32_t metric) {
  return base_dist_p(x, q, d, metric_p(metric));
}

/* S^(1/bp): the distance a direct query on a graph built under L_bp returns */
static double base_root(double s, double bp) {
  return bp == 1.0 ? s : bp == 2.0 ? sqrt(s) : bp == 0.5 ? s * s : pow(s, 1.0 / bp);
}

/* Near-tie accounting of oracle_uhnsw_query_trav: while g_near is set, every
 * comparison of two different nodes' finite distances whose gap is at most
 * g_tie_tol times the larger one (equal values included) is counted.  (A
 * node compared with itself, as when the popped candidate is W's furthest
 * entry, decides nothing that a perturbation could change.)  A search that made no such
 * comparison takes the same decisions under any perturbation of its
 * distances smaller than half that tolerance.  Thread-local, so that the
 * queries of the thread driver count independently; NULL everywhere else. */
static __thread int64_t* g_near = NULL;
static __thread double g_tie_tol = 0.0;

/* (da, ia) precedes (db, ib) in the (distance, id) order */
static int pair_less(double da, int64_t ia, double db, int64_t ib) {
  if (g_near && ia != ib && isfinite(da) && isfinite(db)) {
    const double m = fabs(da) > fabs(db) ? fabs(da) : fabs(db);
    if (fabs(da - db) <= g_tie_tol * m) (*g_near)++;
  }
  if (da < db) return 1;
  if (da > db) return 0;
  return ia < ib;
}

/* Insert (s, id) into the sorted list (ds, is) holding *cnt <= cap entries;
 * the worst entry falls off when the list is full.  Returns 1 if inserted. */
static int sorted_insert(double* ds, int64_t* is, int32_t* cnt, int32_t cap, double s, int64_t id) {
  int32_t c = *cnt;
  if (c == cap && !pair_less(s, id, ds[c - 1], is[c - 1])) return 0;
  int32_t pos = (c == cap) ? c - 1 : c;
  while (pos > 0 && pair_less(s, id, ds[pos - 1], is[pos - 1])) {
    ds[pos] = ds[pos - 1];
    is[pos] = is[pos - 1];
    --pos;
  }
  ds[pos] = s;
  is[pos] = id;
  if (c < cap) *cnt = c + 1;
  return 1;
}

/* ------------------------------------------------------------------ */
/* O1: exact L_p top-K (problem statement, Sections 1.1 / 2.1)         */
/* ------------------------------------------------------------------ */

/* For each query i: the k ids minimising S_p(x, q_i) over all n base rows,
 * ascending by (S, id); rows beyond n are padded with id -1, S = +inf. */
int oracle_exact_knn(const float* base, int64_t n, int32_t d, const float* queries, int64_t nq,
                     const float* p, int32_t k, int64_t* out_ids, double* out_S) {
  if (k <= 0 || d <= 0 || n < 0 || nq < 0) return OR_EINVAL;
  for (int64_t i = 0; i < nq; ++i) {
    double* ds = out_S + i * k;
    int64_t* is = out_ids + i * k;
    int32_t cnt = 0;
    for (int32_t j = 0; j < k; ++j) { ds[j] = INFINITY; is[j] = -1; }
    const float* q = queries + i * (int64_t)d;
    for (int64_t x = 0; x < n; ++x) {
      double s = oracle_lp_sum(base + x * (int64_t)d, q, d, (double)p[i]);
      sorted_insert(ds, is, &cnt, k, s, x);
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Graph access: the builder's lists or a CSR graph                    */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t cnt;
  int32_t cap;
  int32_t* ids;
} nlist_t;

/* CSR form of one HNSW graph, the layout the library's loader also takes:
 * level l holds count[l] nodes (sorted global ids; level 0 may pass NULL
 * for "all nodes, identity"), offsets[count[l]+1] and global-id nbrs. */
typedef struct oracle_csr {
  int32_t num_levels;
  int32_t entry_point;
  int32_t max_degree0;
  int32_t max_degree;
  int64_t n;
  const int32_t* count;
  const int32_t* const* nodes;
  const int64_t* const* offsets;
  const int32_t* const* nbrs;
} oracle_csr;

typedef struct {
  /* builder form */
  nlist_t** links;        /* links[v][l], l <= level[v] */
  const int32_t* level;
  /* CSR form */
  const oracle_csr* csr;
} gview_t;

/* row of node v inside level l of a CSR graph (binary search; -1 if absent) */
static int64_t csr_row(const oracle_csr* g, int32_t l, int32_t v) {
  if (l == 0 && g->nodes[0] == NULL) return v;
  const int32_t* nodes = g->nodes[l];
  int64_t lo = 0, hi = g->count[l];
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (nodes[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  if (lo < g->count[l] && nodes[lo] == v) return lo;
  return -1;
}

static void neighbours(const gview_t* g, int32_t v, int32_t l, const int32_t** out, int32_t* cnt) {
  if (g->links) {
    nlist_t* L = &g->links[v][l];
    *out = L->ids;
    *cnt = L->cnt;
    return;
  }
  int64_t r = csr_row(g->csr, l, v);
  if (r < 0) { *out = NULL; *cnt = 0; return; }
  int64_t a = g->csr->offsets[l][r], b = g->csr->offsets[l][r + 1];
  *out = g->csr->nbrs[l] + a;
  *cnt = (int32_t)(b - a);
}

/* ------------------------------------------------------------------ */
/* SEARCH-LAYER (HNSW Algorithm 2), the routine behind KnnSearch       */
/* ------------------------------------------------------------------ */

typedef struct {
  double* d;
  int64_t* id;
  int32_t cnt;
  int32_t cap;
} pset_t;

typedef struct {
  uint32_t* mark;   /* visited marks, one per node */
  uint32_t gen;
  int64_t n;
} visited_t;

static int pset_grow(pset_t* s, int32_t need) {
  if (need <= s->cap) return 1;
  int32_t nc = s->cap ? s->cap * 2 : 64;
  while (nc < need) nc *= 2;
  double* nd = (double*)realloc(s->d, sizeof(double) * nc);
  if (!nd) return 0;
  s->d = nd;
  int64_t* ni = (int64_t*)realloc(s->id, sizeof(int64_t) * nc);
  if (!ni) return 0;
  s->id = ni;
  s->cap = nc;
  return 1;
}

static void visited_next(visited_t* v) {
  v->gen++;
  if (v->gen == 0) {
    memset(v->mark, 0, sizeof(uint32_t) * v->n);
    v->gen = 1;
  }
}

/*
 * W <- SEARCH-LAYER(q, ep, ef, lc):
 *   v <- ep; C <- ep; W <- ep
 *   while C not empty:
 *     c <- nearest of C (removed); f <- furthest of W
 *     if c is further than f: stop
 *     for each e in neighbourhood(c) at layer lc not in v:
 *       v <- v + e; f <- furthest of W
 *       if e is nearer than f or |W| < ef: C <- C + e; W <- W + e;
 *                                          if |W| > ef: drop furthest of W
 * W is kept sorted ascending (so "furthest" is its last entry); C is an
 * unsorted array scanned for its minimum.  `n_dist` counts base-distance
 * evaluations.  q is either a query vector or, during construction, the
 * inserted row.
 */
static int search_layer(const gview_t* g, const float* base, int32_t d, double bp,
                        const float* q, const int64_t* ep, const double* ep_d, int32_t n_ep,
                        int32_t ef, int32_t lc, visited_t* vis, pset_t* W, int64_t* n_dist) {
  pset_t C = {0};
  visited_next(vis);
  W->cnt = 0;
  if (!pset_grow(W, ef + 1)) return 0;
  if (!pset_grow(&C, n_ep + 1)) return 0;
  for (int32_t i = 0; i < n_ep; ++i) {
    vis->mark[ep[i]] = vis->gen;
    C.d[C.cnt] = ep_d[i];
    C.id[C.cnt] = ep[i];
    C.cnt++;
    sorted_insert(W->d, W->id, &W->cnt, ef, ep_d[i], ep[i]);
  }
  while (C.cnt > 0) {
    int32_t best = 0;
    for (int32_t i = 1; i < C.cnt; ++i)
      if (pair_less(C.d[i], C.id[i], C.d[best], C.id[best])) best = i;
    double cd = C.d[best];
    int64_t cid = C.id[best];
    C.d[best] = C.d[C.cnt - 1];
    C.id[best] = C.id[C.cnt - 1];
    C.cnt--;
    if (pair_less(W->d[W->cnt - 1], W->id[W->cnt - 1], cd, cid)) break;
    const int32_t* nb;
    int32_t nn;
    neighbours(g, (int32_t)cid, lc, &nb, &nn);
    for (int32_t a = 0; a < nn; ++a) {
      int64_t e = nb[a];
      if (e < 0) continue;
      if (vis->mark[e] == vis->gen) continue;
      vis->mark[e] = vis->gen;
      double de = base_dist_p(base + e * (int64_t)d, q, d, bp);
      if (n_dist) (*n_dist)++;
      if (W->cnt < ef || pair_less(de, e, W->d[W->cnt - 1], W->id[W->cnt - 1])) {
        if (!pset_grow(&C, C.cnt + 1)) return 0;
        C.d[C.cnt] = de;
        C.id[C.cnt] = e;
        C.cnt++;
        sorted_insert(W->d, W->id, &W->cnt, ef, de, e);
      }
    }
  }
  free(C.d);
  free(C.id);
  return 1;
}

/*
 * Layer search that expands `width` beam entries per step.  This is a GPU
 * adaptation, not the paper's search: with width = 1 it is HNSW's own order
 * (SEARCH-LAYER above expands the nearest unexpanded entry of W, and stops
 * when every entry of W is expanded), and with width > 1 a step takes
 * several parents before their neighbours are ranked:
 *   W <- ep (every entry unexpanded); v <- ep
 *   repeat:
 *     P <- the first `width` unexpanded entries of W, in W's order, now expanded
 *     if P is empty: stop
 *     N <- the neighbours at layer lc of each parent in P's order, in list
 *          order, that are not in v (each joins v as it is taken)
 *     W <- the ef nearest of W + N by (distance, id); entries of N unexpanded
 * W is kept sorted ascending with an expanded flag per entry.
 */
static int search_layer_wide(const gview_t* g, const float* base, int32_t d, double bp,
                             const float* q, int64_t ep, double ep_d, int32_t ef, int32_t width,
                             int32_t lc, visited_t* vis, pset_t* W, int64_t* n_dist) {
  visited_next(vis);
  if (!pset_grow(W, ef + 1)) return 0;
  unsigned char* ex = (unsigned char*)calloc((size_t)ef + 1, 1);
  int64_t* par = (int64_t*)malloc(sizeof(int64_t) * (size_t)width);
  if (!ex || !par) { free(ex); free(par); return 0; }
  W->cnt = 1;
  W->d[0] = ep_d;
  W->id[0] = ep;
  vis->mark[ep] = vis->gen;
  for (;;) {
    int32_t np = 0;
    for (int32_t i = 0; i < W->cnt && np < width; ++i)
      if (!ex[i]) { ex[i] = 1; par[np++] = W->id[i]; }
    if (np == 0) break;
    for (int32_t j = 0; j < np; ++j) {
      const int32_t* nb;
      int32_t nn;
      neighbours(g, (int32_t)par[j], lc, &nb, &nn);
      for (int32_t a = 0; a < nn; ++a) {
        int64_t e = nb[a];
        if (e < 0 || vis->mark[e] == vis->gen) continue;
        vis->mark[e] = vis->gen;
        double de = base_dist_p(base + e * (int64_t)d, q, d, bp);
        if (n_dist) (*n_dist)++;
        /* W <- the ef nearest of W + {e}, e unexpanded (the order in which the
         * step's candidates are added does not change the resulting set) */
        int32_t c = W->cnt;
        if (c == ef && !pair_less(de, e, W->d[c - 1], W->id[c - 1])) continue;
        int32_t pos = (c == ef) ? c - 1 : c;
        while (pos > 0 && pair_less(de, e, W->d[pos - 1], W->id[pos - 1])) {
          W->d[pos] = W->d[pos - 1];
          W->id[pos] = W->id[pos - 1];
          ex[pos] = ex[pos - 1];
          --pos;
        }
        W->d[pos] = de;
        W->id[pos] = e;
        ex[pos] = 0;
        if (c < ef) W->cnt = c + 1;
      }
    }
  }
  free(ex);
  free(par);
  return 1;
}

/* ------------------------------------------------------------------ */
/* SELECT-NEIGHBORS-HEURISTIC (HNSW Algorithm 4; no candidate          */
/* extension, pruned connections not kept)                             */
/* ------------------------------------------------------------------ */

/* cand (cand_d = distance to the base point b) sorted ascending; keep e only
 * if e is strictly nearer to b than to every element already kept. */
static int32_t select_heuristic(const float* base, int32_t d, double bp, const int64_t* cand,
                                const double* cand_d, int32_t nc, int32_t m, int32_t* out) {
  int32_t r = 0;
  for (int32_t i = 0; i < nc && r < m; ++i) {
    int64_t e = cand[i];
    int keep = 1;
    for (int32_t j = 0; j < r; ++j) {
      double der = base_dist_p(base + e * (int64_t)d, base + (int64_t)out[j] * d, d, bp);
      if (!(cand_d[i] < der)) { keep = 0; break; }
    }
    if (keep) out[r++] = (int32_t)e;
  }
  return r;
}

/* exposed for the hand-derived tests of the heuristic */
int32_t oracle_select_heuristic(const float* base, int32_t d, int32_t metric, const int64_t* cand,
                                const double* cand_d, int32_t nc, int32_t m, int32_t* out) {
  return select_heuristic(base, d, metric_p(metric), cand, cand_d, nc, m, out);
}

/* ------------------------------------------------------------------ */
/* O2: HNSW construction (Section 2.2; HNSW Algorithm 1)               */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  int32_t d, M, M0, efc;
  double bp;                       /* the graph's base metric is S_bp */
  int32_t entry, max_level;
  const float* base;
  int32_t* level;
  nlist_t** links;
} oracle_graph;

static int list_set(nlist_t* L, const int32_t* ids, int32_t cnt) {
  if (cnt > L->cap) return 0;
  memcpy(L->ids, ids, sizeof(int32_t) * cnt);
  L->cnt = cnt;
  return 1;
}

void oracle_graph_free(oracle_graph* g) {
  if (!g) return;
  if (g->links) {
    for (int64_t v = 0; v < g->n; ++v) {
      if (!g->links[v]) continue;
      for (int32_t l = 0; l <= g->level[v]; ++l) free(g->links[v][l].ids);
      free(g->links[v]);
    }
    free(g->links);
  }
  free(g->level);
  free(g);
}

/*
 * INSERT(q) for q = 0, 1, ..., n-1 in order, with the given levels:
 *   W <- empty; ep <- entry point; L <- its level; l <- level[q]
 *   for lc = L .. l+1:  W <- SEARCH-LAYER(q, ep, 1, lc); ep <- nearest of W
 *   for lc = min(L, l) .. 0:
 *     W <- SEARCH-LAYER(q, ep, efConstruction, lc)
 *     neighbours <- SELECT-NEIGHBORS-HEURISTIC(q, W, M)
 *     connect q -> neighbours and each neighbour e -> q;
 *     if e now has more than Mmax links (Mmax0 = M0 at layer 0, M above):
 *       e's links <- SELECT-NEIGHBORS-HEURISTIC(e, e's links, Mmax)
 *     ep <- W
 *   if l > L: entry point <- q
 */
oracle_graph* oracle_hnsw_build_p(const float* base, int64_t n, int32_t d, double bp, int32_t M,
                                  int32_t M0, int32_t efc, const int32_t* levels, int32_t* status) {
  *status = OR_EINVAL;
  if (n <= 0 || d <= 0 || !valid_bp(bp) || M < 2 || M0 < M || efc < 1) return NULL;
  oracle_graph* g = (oracle_graph*)calloc(1, sizeof(oracle_graph));
  if (!g) { *status = OR_ENOMEM; return NULL; }
  g->n = n; g->d = d; g->bp = bp; g->M = M; g->M0 = M0; g->efc = efc;
  g->base = base;
  g->level = (int32_t*)malloc(sizeof(int32_t) * n);
  g->links = (nlist_t**)calloc(n, sizeof(nlist_t*));
  visited_t vis = {(uint32_t*)calloc(n, sizeof(uint32_t)), 0, n};
  pset_t W = {0};
  int32_t cap = efc > M0 ? efc : M0;
  int64_t* ep = (int64_t*)malloc(sizeof(int64_t) * (cap + 1));
  double* epd = (double*)malloc(sizeof(double) * (cap + 1));
  int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (M0 + 2));
  double* cand_d = (double*)malloc(sizeof(double) * (M0 + 2));
  int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (M0 + 2));
  int32_t* sel2 = (int32_t*)malloc(sizeof(int32_t) * (M0 + 2));
  if (!g->level || !g->links || !vis.mark || !ep || !epd || !cand || !cand_d || !sel || !sel2) {
    *status = OR_ENOMEM;
    goto fail;
  }
  gview_t view = {g->links, g->level, NULL};
  for (int64_t q = 0; q < n; ++q) {
    int32_t l = levels[q];
    if (l < 0) { *status = OR_EINVAL; goto fail; }
    g->level[q] = l;
    g->links[q] = (nlist_t*)calloc(l + 1, sizeof(nlist_t));
    if (!g->links[q]) { *status = OR_ENOMEM; goto fail; }
    for (int32_t lc = 0; lc <= l; ++lc) {
      int32_t c = (lc == 0 ? M0 : M) + 1;
      g->links[q][lc].ids = (int32_t*)malloc(sizeof(int32_t) * c);
      g->links[q][lc].cap = c;
      if (!g->links[q][lc].ids) { *status = OR_ENOMEM; goto fail; }
    }
    const float* x = base + q * (int64_t)d;
    if (q == 0) {
      g->entry = 0;
      g->max_level = l;
      continue;
    }
    int32_t L = g->max_level;
    int32_t n_ep = 1;
    ep[0] = g->entry;
    epd[0] = base_dist_p(base + (int64_t)g->entry * d, x, d, bp);
    for (int32_t lc = L; lc > l; --lc) {
      if (!search_layer(&view, base, d, bp, x, ep, epd, n_ep, 1, lc, &vis, &W, NULL)) {
        *status = OR_ENOMEM;
        goto fail;
      }
      ep[0] = W.id[0];
      epd[0] = W.d[0];
      n_ep = 1;
    }
    for (int32_t lc = (L < l ? L : l); lc >= 0; --lc) {
      if (!search_layer(&view, base, d, bp, x, ep, epd, n_ep, efc, lc, &vis, &W, NULL)) {
        *status = OR_ENOMEM;
        goto fail;
      }
      int32_t r = select_heuristic(base, d, bp, W.id, W.d, W.cnt, M, sel);
      list_set(&g->links[q][lc], sel, r);
      int32_t mmax = (lc == 0) ? M0 : M;
      for (int32_t i = 0; i < r; ++i) {
        int32_t e = sel[i];
        nlist_t* Le = &g->links[e][lc];
        Le->ids[Le->cnt++] = (int32_t)q;       /* capacity is mmax + 1 */
        if (Le->cnt > mmax) {
          const float* xe = base + (int64_t)e * d;
          int32_t m = Le->cnt;
          for (int32_t a = 0; a < m; ++a) {
            int64_t id = Le->ids[a];
            double dd = base_dist_p(base + id * (int64_t)d, xe, d, bp);
            int32_t pos = a;
            while (pos > 0 && pair_less(dd, id, cand_d[pos - 1], cand[pos - 1])) {
              cand_d[pos] = cand_d[pos - 1];
              cand[pos] = cand[pos - 1];
              --pos;
            }
            cand_d[pos] = dd;
            cand[pos] = id;
          }
          int32_t rr = select_heuristic(base, d, bp, cand, cand_d, m, mmax, sel2);
          list_set(Le, sel2, rr);
        }
      }
      n_ep = W.cnt;
      for (int32_t i = 0; i < W.cnt; ++i) { ep[i] = W.id[i]; epd[i] = W.d[i]; }
    }
    if (l > L) {
      g->entry = (int32_t)q;
      g->max_level = l;
    }
  }
  free(vis.mark); free(W.d); free(W.id); free(ep); free(epd); free(cand); free(cand_d); free(sel); free(sel2);
  *status = OR_OK;
  return g;
fail:
  free(vis.mark); free(W.d); free(W.id); free(ep); free(epd); free(cand); free(cand_d); free(sel); free(sel2);
  oracle_graph_free(g);
  return NULL;
}

oracle_graph* oracle_hnsw_build(const float* base, int64_t n, int32_t d, int32_t metric, int32_t M,
                                int32_t M0, int32_t efc, const int32_t* levels, int32_t* status) {
  if (!valid_metric(metric)) { *status = OR_EINVAL; return NULL; }
  return oracle_hnsw_build_p(base, n, d, metric_p(metric), M, M0, efc, levels, status);
}

/* CSR export: number of levels, entry point, and per-level sizes / arrays. */
int32_t oracle_graph_num_levels(const oracle_graph* g) { return g->max_level + 1; }
int32_t oracle_graph_entry(const oracle_graph* g) { return g->entry; }

void oracle_graph_level_size(const oracle_graph* g, int32_t l, int64_t* n_nodes, int64_t* n_edges) {
  int64_t nn = 0, ne = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    if (g->level[v] < l) continue;
    nn++;
    ne += g->links[v][l].cnt;
  }
  *n_nodes = nn;
  *n_edges = ne;
}

void oracle_graph_level_copy(const oracle_graph* g, int32_t l, int32_t* nodes, int64_t* offsets,
                             int32_t* nbrs) {
  int64_t r = 0, e = 0;
  offsets[0] = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    if (g->level[v] < l) continue;
    nodes[r] = (int32_t)v;
    const nlist_t* L = &g->links[v][l];
    for (int32_t a = 0; a < L->cnt; ++a) nbrs[e++] = L->ids[a];
    offsets[++r] = e;
  }
}

/* ------------------------------------------------------------------ */
/* O3: KnnSearch(q, t) on a CSR graph (Section 3.1; HNSW Algorithm 5) */
/* ------------------------------------------------------------------ */

/*
 * ep <- entry point; for lc = top .. 1: W <- SEARCH-LAYER(q, ep, 1, lc);
 * ep <- nearest of W; W <- SEARCH-LAYER(q, ep, ef, 0); return the t nearest
 * of W ascending by (base distance, id).  Rows of out_ids beyond |W| are -1.
 */
int oracle_hnsw_search_p(const oracle_csr* g, const float* base, int32_t d, double bp,
                         const float* q, int32_t ef, int32_t t, int64_t* out_ids, double* out_d,
                         int64_t* n_dist) {
  if (ef < 1 || t < 1 || !valid_bp(bp)) return OR_EINVAL;
  gview_t view = {NULL, NULL, g};
  visited_t vis = {(uint32_t*)calloc(g->n, sizeof(uint32_t)), 0, g->n};
  pset_t W = {0};
  if (!vis.mark) return OR_ENOMEM;
  int64_t ep = g->entry_point;
  double epd = base_dist_p(base + ep * (int64_t)d, q, d, bp);
  if (n_dist) (*n_dist)++;
  for (int32_t lc = g->num_levels - 1; lc >= 1; --lc) {
    if (!search_layer(&view, base, d, bp, q, &ep, &epd, 1, 1, lc, &vis, &W, n_dist)) {
      free(vis.mark);
      return OR_ENOMEM;
    }
    ep = W.id[0];
    epd = W.d[0];
  }
  if (!search_layer(&view, base, d, bp, q, &ep, &epd, 1, ef, 0, &vis, &W, n_dist)) {
    free(vis.mark);
    return OR_ENOMEM;
  }
  for (int32_t i = 0; i < t; ++i) {
    out_ids[i] = i < W.cnt ? W.id[i] : -1;
    out_d[i] = i < W.cnt ? W.d[i] : INFINITY;
  }
  free(vis.mark);
  free(W.d);
  free(W.id);
  return OR_OK;
}

int oracle_hnsw_search(const oracle_csr* g, const float* base, int32_t d, int32_t metric,
                       const float* q, int32_t ef, int32_t t, int64_t* out_ids, double* out_d,
                       int64_t* n_dist) {
  if (!valid_metric(metric)) return OR_EINVAL;
  return oracle_hnsw_search_p(g, base, d, metric_p(metric), q, ef, t, out_ids, out_d, n_dist);
}

/*
 * KnnSearch with the layer-0 beam expanding `width` entries per step (the
 * GPU's fast mode, search_layer_wide): the upper levels as in
 * oracle_hnsw_search_p (beam 1), then layer 0 by search_layer_wide.  With
 * width = 1 it returns what oracle_hnsw_search_p returns.
 */
int oracle_hnsw_search_w(const oracle_csr* g, const float* base, int32_t d, double bp,
                         const float* q, int32_t ef, int32_t t, int32_t width, int64_t* out_ids,
                         double* out_d, int64_t* n_dist) {
  if (ef < 1 || t < 1 || width < 1 || !valid_bp(bp)) return OR_EINVAL;
  gview_t view = {NULL, NULL, g};
  visited_t vis = {(uint32_t*)calloc(g->n, sizeof(uint32_t)), 0, g->n};
  pset_t W = {0};
  if (!vis.mark) return OR_ENOMEM;
  int64_t ep = g->entry_point;
  double epd = base_dist_p(base + ep * (int64_t)d, q, d, bp);
  if (n_dist) (*n_dist)++;
  int ok = 1;
  for (int32_t lc = g->num_levels - 1; lc >= 1 && ok; --lc) {
    ok = search_layer(&view, base, d, bp, q, &ep, &epd, 1, 1, lc, &vis, &W, n_dist);
    if (ok) {
      ep = W.id[0];
      epd = W.d[0];
    }
  }
  if (ok) ok = search_layer_wide(&view, base, d, bp, q, ep, epd, ef, width, 0, &vis, &W, n_dist);
  if (ok) {
    for (int32_t i = 0; i < t; ++i) {
      out_ids[i] = i < W.cnt ? W.id[i] : -1;
      out_d[i] = i < W.cnt ? W.d[i] : INFINITY;
    }
  }
  free(vis.mark);
  free(W.d);
  free(W.id);
  return ok ? OR_OK : OR_ENOMEM;
}

/* ------------------------------------------------------------------ */
/* O4: verification of a candidate set (Section 3.1)                   */
/* ------------------------------------------------------------------ */

/*
 * Exact mode: the k candidates of C (ids, -1 = absent slot) with the smallest
 * (S, id), ascending.  With abandon != 0 a candidate's accumulation stops as
 * soon as its partial sum exceeds the current k-th best S (the result is the
 * same: partial sums of non-negative terms never decrease).  n_terms counts
 * |x_j - q_j|^p evaluations.
 */
int oracle_verify_exact(const float* base, int32_t d, const float* q, double p, const int32_t* cand,
                        int32_t t, int32_t k, int32_t abandon, int64_t* out_ids, double* out_S,
                        int64_t* n_terms) {
  if (k < 1 || t < 0) return OR_EINVAL;
  int32_t cnt = 0;
  for (int32_t j = 0; j < k; ++j) { out_S[j] = INFINITY; out_ids[j] = -1; }
  for (int32_t i = 0; i < t; ++i) {
    int64_t id = cand[i];
    if (id < 0) continue;
    const float* x = base + id * (int64_t)d;
    double thr = (cnt == k) ? out_S[k - 1] : INFINITY;
    double s = 0.0;
    int dropped = 0;
    for (int32_t j = 0; j < d; ++j) {
      s += pow(fabs((double)x[j] - (double)q[j]), p);
      if (n_terms) (*n_terms)++;
      if (abandon && s > thr) { dropped = 1; break; }
    }
    if (!dropped) sorted_insert(out_S, out_ids, &cnt, k, s, id);
  }
  return OR_OK;
}

/*
 * Paper mode: the early-terminated verification of Algorithm 1 (Section 3.1).
 * The current answer starts as the K best (by (S, id)) of the first K valid
 * candidates of C.  The rest of C is then taken in consecutive batches of
 * kappa valid candidates (the last batch may be shorter); after each batch
 * the answer becomes the K best of itself and the batch, and the search
 * stops as soon as the fraction of the new answer that was already in the
 * previous one reaches tau.  If C runs out first, the last answer is
 * returned.  The fraction is compared in IEEE single precision,
 * (float)overlap / (float)K >= tau.  n_lp counts candidates whose L_p sum was
 * computed; n_batches counts batches examined.
 */
int oracle_verify_paper(const float* base, int32_t d, const float* q, double p, const int32_t* cand,
                        int32_t t, int32_t k, int32_t kappa, float tau, int64_t* out_ids,
                        double* out_S, int64_t* n_lp, int64_t* n_batches) {
  if (k < 1 || kappa < 1 || t < 0) return OR_EINVAL;
  double* Rs = (double*)malloc(sizeof(double) * k);
  int64_t* Ri = (int64_t*)malloc(sizeof(int64_t) * k);
  double* Ns = (double*)malloc(sizeof(double) * k);
  int64_t* Ni = (int64_t*)malloc(sizeof(int64_t) * k);
  if (!Rs || !Ri || !Ns || !Ni) { free(Rs); free(Ri); free(Ns); free(Ni); return OR_ENOMEM; }
  int32_t rc = 0;
  for (int32_t j = 0; j < k; ++j) { Rs[j] = INFINITY; Ri[j] = -1; }
  int32_t i = 0;
  /* R <- first K (valid) points of C */
  while (i < t && rc < k) {
    int64_t id = cand[i++];
    if (id < 0) continue;
    double s = oracle_lp_sum(base + id * (int64_t)d, q, d, p);
    if (n_lp) (*n_lp)++;
    sorted_insert(Rs, Ri, &rc, k, s, id);
  }
  while (i < t) {
    /* next batch R' of kappa (valid) points */
    int32_t nc = rc;
    memcpy(Ns, Rs, sizeof(double) * k);
    memcpy(Ni, Ri, sizeof(int64_t) * k);
    int32_t taken = 0;
    while (i < t && taken < kappa) {
      int64_t id = cand[i++];
      if (id < 0) continue;
      taken++;
      double s = oracle_lp_sum(base + id * (int64_t)d, q, d, p);
      if (n_lp) (*n_lp)++;
      sorted_insert(Ns, Ni, &nc, k, s, id);
    }
    if (taken == 0) break;
    if (n_batches) (*n_batches)++;
    int32_t overlap = 0;
    for (int32_t a = 0; a < nc; ++a)
      for (int32_t b = 0; b < rc; ++b)
        if (Ni[a] == Ri[b]) { overlap++; break; }
    memcpy(Rs, Ns, sizeof(double) * k);
    memcpy(Ri, Ni, sizeof(int64_t) * k);
    rc = nc;
    if ((float)overlap / (float)k >= tau) break;
  }
  memcpy(out_S, Rs, sizeof(double) * k);
  memcpy(out_ids, Ri, sizeof(int64_t) * k);
  free(Rs); free(Ri); free(Ns); free(Ni);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 end to end                                               */
/* ------------------------------------------------------------------ */

/*
 * Routing (Algorithm 1, lines 1-5), for graphs ga and gb under base metrics
 * ma and mb (U-HNSW: L1 and L2; U-HNSW-E: L0.5 and L1): when p equals a
 * graph's base p exactly (in FP32), direct K-NN on that graph with
 * ef' = max(ef, k), and the returned distance is the base distance's root
 * S^(1/bp).  Otherwise ga if p <= cutoff (FP32 compare), else gb;
 * C <- KnnSearch(q, t) with t' = max(t or ef, k) and ef' = max(ef, t'); then
 * verify C (mode 0: exact with abandon; mode 1: Algorithm 1's batches).  The
 * returned distance is S^(1/p).  Counters: stats[0] = base-distance
 * evaluations (N_b), stats[1] = L_p candidates computed (N_p), stats[2] = L_p
 * terms.
 *
 * With `trav` given (rows of the same shape as `base`), the graph search
 * computes its base distances on `trav` (the precision form: a rounded copy
 * of the rows, here as FP32 values) and verification stays on `base`.  A
 * direct query (p == the graph's base p) then ranks its whole beam of ef'
 * by the exact base distance on `base`, so that its returned distances are
 * those of the FP32 rows.  With tie_tol > 0, stats[3] counts the near-tie
 * comparisons of the search (see pair_less); cand_out, if given, receives C
 * (the first t' beam entries, or the whole beam of a direct query on `trav`),
 * -1 padded.
 */
static int uhnsw_query_impl(const oracle_csr* ga, const oracle_csr* gb, double bpa, double bpb,
                            const float* base, const float* trav, int32_t d, const float* q,
                            float p, int32_t k, int32_t ef, int32_t t, float tau, int32_t kappa,
                            float cutoff, int32_t mode, int32_t width, double tie_tol,
                            int64_t* out_ids, double* out_dist, int64_t* cand_out,
                            int64_t* stats) {
  if (k < 1 || ef < 1 || width < 1 || !(p > 0.0f) || !(p <= 2.0f)) return OR_EINVAL;
  if (!valid_bp(bpa) || !valid_bp(bpb)) return OR_EINVAL;
  const int reduced = trav != NULL;
  if (!reduced) trav = base;
  int64_t nb = 0, np = 0, nterm = 0, near = 0;
  const float pa = (float)bpa, pb = (float)bpb;
  int use_a = (p == pa) ? 1 : (p == pb) ? 0 : (p <= cutoff);
  double bp = use_a ? bpa : bpb;
  int direct = p == (float)bp;
  const oracle_csr* g = use_a ? ga : gb;
  int32_t tt = direct ? k : (t > 0 ? t : ef);
  if (tt < k) tt = k;
  int32_t efp = ef > tt ? ef : tt;
  /* a direct query on the rounded copy keeps its whole beam for the re-rank */
  const int32_t nc = (direct && reduced) ? efp : tt;
  int64_t* C = (int64_t*)malloc(sizeof(int64_t) * nc);
  double* Cd = (double*)malloc(sizeof(double) * nc);
  int32_t* C32 = (int32_t*)malloc(sizeof(int32_t) * nc);
  double* S = (double*)malloc(sizeof(double) * k);
  if (!C || !Cd || !C32 || !S) { free(C); free(Cd); free(C32); free(S); return OR_ENOMEM; }
  if (tie_tol > 0.0) { g_near = &near; g_tie_tol = tie_tol; }
  int rc = width == 1 ? oracle_hnsw_search_p(g, trav, d, bp, q, efp, nc, C, Cd, &nb)
                      : oracle_hnsw_search_w(g, trav, d, bp, q, efp, nc, width, C, Cd, &nb);
  g_near = NULL;
  if (rc != OR_OK) { free(C); free(Cd); free(C32); free(S); return rc; }
  if (cand_out) for (int32_t j = 0; j < nc; ++j) cand_out[j] = C[j];
  if (direct && !reduced) {
    for (int32_t j = 0; j < k; ++j) {
      out_ids[j] = C[j];
      out_dist[j] = C[j] < 0 ? INFINITY : base_root(Cd[j], bp);
    }
  } else {
    for (int32_t j = 0; j < nc; ++j) C32[j] = (int32_t)C[j];
    if (mode == 0 || direct) {
      oracle_verify_exact(base, d, q, (double)p, C32, nc, k, 1, out_ids, S, &nterm);
      for (int32_t j = 0; j < nc; ++j) if (C32[j] >= 0) np++;
    } else {
      oracle_verify_paper(base, d, q, (double)p, C32, nc, k, kappa > 0 ? kappa : k,
                          tau > 0.0f ? tau : 0.92f, out_ids, S, &np, NULL);
      nterm = np * d;
    }
    for (int32_t j = 0; j < k; ++j)
      out_dist[j] = out_ids[j] < 0 ? INFINITY : pow(S[j], 1.0 / (double)p);
  }
  if (stats) { stats[0] = nb; stats[1] = np; stats[2] = nterm; }
  if (stats && tie_tol > 0.0) stats[3] = near;
  free(C); free(Cd); free(C32); free(S);
  return OR_OK;
}

int oracle_uhnsw_query_w(const oracle_csr* ga, const oracle_csr* gb, double bpa, double bpb,
                         const float* base, int32_t d, const float* q, float p, int32_t k,
                         int32_t ef, int32_t t, float tau, int32_t kappa, float cutoff,
                         int32_t mode, int32_t width, int64_t* out_ids, double* out_dist,
                         int64_t* stats) {
  return uhnsw_query_impl(ga, gb, bpa, bpb, base, NULL, d, q, p, k, ef, t, tau, kappa, cutoff,
                          mode, width, 0.0, out_ids, out_dist, NULL, stats);
}

/* Algorithm 1 in the precision form: the graph search on the rounded rows
 * `trav`, verification on `base` (see uhnsw_query_impl); stats has 4 slots,
 * the last the number of near-tie comparisons of the search at tie_tol. */
int oracle_uhnsw_query_trav(const oracle_csr* ga, const oracle_csr* gb, double bpa, double bpb,
                            const float* base, const float* trav, int32_t d, const float* q,
                            float p, int32_t k, int32_t ef, int32_t t, float tau, int32_t kappa,
                            float cutoff, int32_t mode, int32_t width, double tie_tol,
                            int64_t* out_ids, double* out_dist, int64_t* cand_out,
                            int64_t* stats) {
  if (!trav || !(tie_tol >= 0.0)) return OR_EINVAL;
  return uhnsw_query_impl(ga, gb, bpa, bpb, base, trav, d, q, p, k, ef, t, tau, kappa, cutoff,
                          mode, width, tie_tol, out_ids, out_dist, cand_out, stats);
}

int oracle_uhnsw_query_p(const oracle_csr* ga, const oracle_csr* gb, double bpa, double bpb,
                         const float* base, int32_t d, const float* q, float p, int32_t k,
                         int32_t ef, int32_t t, float tau, int32_t kappa, float cutoff,
                         int32_t mode, int64_t* out_ids, double* out_dist, int64_t* stats) {
  return oracle_uhnsw_query_w(ga, gb, bpa, bpb, base, d, q, p, k, ef, t, tau, kappa, cutoff, mode,
                              1, out_ids, out_dist, stats);
}

int oracle_uhnsw_query(const oracle_csr* ga, const oracle_csr* gb, int32_t ma, int32_t mb,
                       const float* base, int32_t d, const float* q, float p, int32_t k,
                       int32_t ef, int32_t t, float tau, int32_t kappa, float cutoff,
                       int32_t mode, int64_t* out_ids, double* out_dist, int64_t* stats) {
  if (!valid_metric(ma) || !valid_metric(mb)) return OR_EINVAL;
  return oracle_uhnsw_query_p(ga, gb, metric_p(ma), metric_p(mb), base, d, q, p, k, ef, t, tau,
                              kappa, cutoff, mode, out_ids, out_dist, stats);
}
