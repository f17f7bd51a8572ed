/*
 * uhnsw.h: C ABI of the GB300 U-HNSW query path.
 *
 * U-HNSW (arxiv 2605.02030) answers a query (q, p) with the K nearest base
 * vectors under that query's own L_p distance, 0.5 <= p <= 2 (Sections 1.1
 * and 2.1), from two HNSW graphs: G1 built under L1 and G2 built under L2
 * (Section 3.1).  A query with p <= cutoff (1.4 by default) searches G1,
 * otherwise G2 ("Candidate generation", Algorithm 1 lines 1-5); the t nearest
 * under the base metric form the candidate set C, which is re-ranked under
 * L_p ("Candidate verification", Algorithm 1 lines 6-10).  p == 1 and p == 2
 * search G1 / G2 for the K nearest directly, without verification (Section 3,
 * introduction).  In general a query whose p equals a graph's base p is
 * answered directly on that graph; U-HNSW-E (Section 4.5) loads graphs under
 * L0.5 and L1 (uhnsw_load_opts.base_metric) and routes with cutoff 0.6.
 *
 * Conventions for every entry point:
 *   - Return value: UHNSW_OK (0) or a negative UHNSW_E* code; nothing throws
 *     across the ABI.  uhnsw_last_error() returns a message for the calling
 *     thread's last failure.
 *   - Arguments are validated before any work is queued; on failure nothing
 *     is written.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     device memory of the current device (e.g. torch tensors' data_ptr()).
 *     All inputs stay owned by the caller.  uhnsw_load copies what it needs.
 *   - Device work is queued on the caller's stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream); results are valid once that
 *     stream has synchronised.  Calls on one index may be queued on several
 *     streams concurrently, and from several host threads on one stream,
 *     unless stated otherwise.  The index keeps a small state for every
 *     stream that has searched it (persistent-queue counters and ordering
 *     workspace, host-search staging) until uhnsw_free: reuse a fixed set
 *     of streams rather than a new stream per call.
 *   - Order of results: ascending by (distance, id).  Missing results are
 *     padded with id -1 and distance +inf.
 *   - Every device wait inside the library is bounded; a wait that gives up
 *     records UHNSW_ETIMEOUT in the query's status (never traps).
 */
#ifndef UHNSW_H_
#define UHNSW_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UHNSW_MAX_LEVELS 16
#define UHNSW_MAX_EF 512   /* largest beam ef' = max(ef, t, k) */
#define UHNSW_MAX_DIM 2048
#define UHNSW_MAX_DEGREE 128

#define UHNSW_OK 0
#define UHNSW_EINVAL (-1)    /* bad argument or malformed graph */
#define UHNSW_EOOM (-2)      /* device or host allocation failed */
#define UHNSW_ECUDA (-3)     /* a CUDA runtime call failed (no device, ...) */
#define UHNSW_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define UHNSW_ECAPACITY (-5) /* a size above a documented limit */

typedef enum { UHNSW_F32 = 0, UHNSW_F16 = 1, UHNSW_BF16 = 2 } uhnsw_dtype;

typedef enum {
  UHNSW_VERIFY_EXACT = 0, /* top-K by L_p over all of C, with partial-sum abandon */
  UHNSW_VERIFY_PAPER = 1  /* Algorithm 1 lines 6-10: batches of kappa, stop at tau */
} uhnsw_verify_mode;

typedef struct uhnsw_index uhnsw_index;

/*
 * One HNSW graph in CSR form per level (Section 2.2: a multi-layer proximity
 * graph).  All arrays are HOST memory owned by the caller and only read
 * during uhnsw_load.  Level l lists the nodes present at that level as sorted
 * global ids level_nodes[l][0..level_count[l]) (level 0 may pass NULL, meaning
 * all n nodes in id order), their adjacency rows
 * level_nbrs[l][level_offsets[l][i] .. level_offsets[l][i+1]) as global ids,
 * with at most max_degree0 links at level 0 and max_degree above.  Every node
 * of level l > 0 must also be present at level l-1; entry_point must be a
 * node of the top level num_levels-1.
 */
typedef struct {
  int32_t num_levels;
  int32_t entry_point;
  int32_t max_degree0;
  int32_t max_degree;
  const int32_t* level_count;
  const int32_t* level_nodes[UHNSW_MAX_LEVELS];
  const int64_t* level_offsets[UHNSW_MAX_LEVELS];
  const int32_t* level_nbrs[UHNSW_MAX_LEVELS];
} uhnsw_graph;

/* Base metric of a graph (the metric it was built under and is searched
 * with).  UHNSW_BASE_L2 is the squared L2 sum and UHNSW_BASE_L05 the L0.5 sum
 * without its root; each orders points exactly like its L_p metric.
 * UHNSW_BASE_LP is the sum for any other p in (0, 2] (the fixed-p HNSW of
 * Section 4.3, one graph per p), evaluated as 2^(p log2 |d_j|). */
typedef enum {
  UHNSW_BASE_L1 = 1,   /* sum |d_j|,       p = 1   */
  UHNSW_BASE_L2 = 2,   /* sum d_j^2,       p = 2   */
  UHNSW_BASE_L05 = 3,  /* sum |d_j|^(1/2), p = 0.5 */
  UHNSW_BASE_L15 = 4,  /* sum |d_j|^(3/2), p = 1.5 (a fixed-p HNSW graph, Section 4.3) */
  UHNSW_BASE_LP = 5    /* sum |d_j|^p,     p = uhnsw_load_opts.base_p of the slot */
} uhnsw_base_metric;

typedef struct {
  /* storage of the copy the beam search reads (the FP32 master copy is kept
   * for verification and returned distances either way) */
  uhnsw_dtype traverse_dtype;
  /* base metrics of the two graph slots; 0 => UHNSW_BASE_L1 for the first
   * (g1) and UHNSW_BASE_L2 for the second (g2), which is U-HNSW.  U-HNSW-E
   * (Section 4.5) loads a graph built under L0.5 as g1 and one built under
   * L1 as g2 ({UHNSW_BASE_L05, UHNSW_BASE_L1}) and searches with cutoff 0.6.
   * The first slot's base p must be below the second's. */
  int32_t base_metric[2];
  /* the p of a slot whose base_metric is UHNSW_BASE_LP, 0 < p <= 2 (read for
   * that slot only; p = 1, 2, 0.5 or 1.5 act as their own codes) */
  float base_p[2];
  int32_t reserved[3];
} uhnsw_load_opts;

/* per-query counters written when uhnsw_search_opts.stats is set */
enum {
  UHNSW_STAT_NB = 0,        /* base-metric distance evaluations (N_b of Eq. 1) */
  UHNSW_STAT_NP = 1,        /* candidates whose L_p sum was started (N_p of Eq. 1) */
  UHNSW_STAT_TERMS = 2,     /* |x_j - q_j|^p terms accumulated */
  UHNSW_STAT_EXPANSIONS = 3,/* beam entries expanded at layer 0 */
  UHNSW_STAT_RESETS = 4,    /* visited-table resets */
  UHNSW_STAT_STATUS = 5,    /* 0 or a negative UHNSW_E* code for this query */
  UHNSW_STAT_GRAPH = 6,     /* graph slot searched: 1 = g1 (G1, L1), 2 = g2 (G2, L2) */
  UHNSW_STAT_ADJ = 7,       /* adjacency rows read (upper levels and layer 0) */
  UHNSW_NSTATS = 8
};

typedef struct {
  int32_t t;             /* |C|, candidates verified; 0 => ef (the whole beam); raised to k */
  int32_t kappa;         /* batch size of Algorithm 1; 0 => k */
  float tau;             /* early-termination threshold of Algorithm 1; 0 => 0.92;
                            a negative value stops after the first batch */
  float cutoff;          /* routing: p <= cutoff searches the first graph (G1); 0 => 1.4 */
  int32_t verify_mode;   /* uhnsw_verify_mode */
  int32_t search_width;  /* beam entries expanded per step, 0..8; <= 1 => exactly HNSW's
                            order (the deterministic mode).  w > 1 (the fast mode): each
                            step takes the first w unexpanded entries of the beam as
                            parents, gathers their unvisited neighbours in parent order
                            and keeps the ef nearest of the beam and the new entries; the
                            results differ from HNSW's order and are judged by recall */
  int32_t persistent;    /* 1: persistent launch pulling queries from a device queue.  The
                            queue is ordered by graph and p form, so that the queries in
                            flight on an SM run the same code.  With per-query ef it is
                            also bucketed by beam (<= 64, 128, 256, 512), one launch per
                            bucket sized for its beam.  Each stream has a queue of its
                            own (created on its first persistent search), so persistent
                            searches on different streams may overlap on the GPU: a
                            launch's blocks fill the SMs that the previous batch's
                            finished blocks leave. */
  int32_t use_graph;     /* 1: capture the launch sequence once per call shape, then replay */
  int32_t ef_max;        /* bound on ef' over the batch when per-query ef is given; 0 => 512 */
  int32_t query_threads; /* threads per query: 32 = one warp per query (4 queries per
                            block), 128 = one block per query; a launch that does not fit
                            in shared memory fails with UHNSW_ECAPACITY.  0 => the
                            configuration uhnsw_autotune chose for this beam / k bucket,
                            else 32; then a beam bucket whose warp-kernel layout does not
                            fit runs the block kernel. */
  int32_t* stats;        /* device [nq][UHNSW_NSTATS] int32, or NULL */
  int32_t stage_bytes;   /* warp kernel: shared memory per query for the FP32 rows being
                            verified (a multiple of 4 rows); 0 => as many rows as fit in
                            the visited table's bytes (the two share one region), a
                            multiple of 4 from 4 to 16 */
  int32_t team_lanes;    /* warp kernel: lanes sharing one row (4, 8, 16 or 32); 0 => the
                            default shape for the row's width (e.g. 4 lanes x 3 chunks
                            for 96 FP16 dimensions, 8 x 2 for 128) */
  void* kernel_events;   /* NULL, or a host array of two cudaEvent_t that uhnsw_search
                            records on its stream right before the first search-kernel
                            launch and right after the last one: the search kernels' own
                            duration, without the queue-ordering kernels of a persistent
                            launch.  Such a call runs without CUDA-graph replay. */
  const int32_t* t_per_query;  /* device [nq] or NULL: query i verifies t_i candidates in
                                  place of t (0 => ef); ef' grows with t_i as above, so a
                                  batch with per-query t needs ef_max (0 => 512).  The knob
                                  of the t / tau trade-off (Section 3.2); uhnsw_plan_t
                                  derives t per p from idealized recall. */
  const float* tau_per_query;  /* device [nq] or NULL: query i's tau in place of tau (0 =>
                                  0.92, negative => stop after the first batch) */
  int32_t hash_bits;     /* visited table of 1 << hash_bits slots per query; 0 => the
                            smallest power of two >= 4 (ef' + search_width * M0), at least
                            2^9.  Allowed: from the smallest power of two >= 2 (ef' +
                            search_width * M0) up to 2^15 (else UHNSW_EINVAL).  The size
                            does not change any result (a table past half full is cleared
                            and refilled with the beam, which cannot change the beam); a
                            smaller table re-evaluates more nodes, a larger one takes
                            shared memory from other queries. */
  int32_t verify_groups; /* verification in the warp-per-query kernels: 32-dimension
                            groups accumulated between two tests of a candidate's partial
                            sum against the running k-th best sum, 1..16; 0 => 2 in
                            uhnsw_search, 1 in uhnsw_verify (the block-per-query kernel
                            tests after every group).  Every lane
                            accumulates its elements in the same order whatever the
                            value, so sums and results do not depend on it; it trades
                            drop-test work for candidates summed further before they are
                            dropped. */
} uhnsw_search_opts;

/*
 * Upload an index: base vectors plus two graphs, G1 (L1) and G2 (L2) unless
 * opts->base_metric says otherwise.
 *   base      host, n x d float32 row-major; copied to an FP32 master copy and,
 *             if opts->traverse_dtype != UHNSW_F32, a rounded FP16/BF16 copy.
 *             Rows are zero-padded on the device to a multiple of 8 elements.
 *   g1, g2    host CSR graphs over the same n nodes (either may be NULL: a
 *             query routed to a missing graph fails with UHNSW_EINVAL status).
 *   opts      may be NULL (FP32 traversal).
 *   out       receives the index handle; free it with uhnsw_free.
 * Layer 0 of each graph is stored as a padded [n][max_degree0] table, upper
 * levels as [rows][max_degree] tables.  Uses the current CUDA device.
 * Errors: EINVAL (d or n out of range, malformed CSR), EOOM, ECUDA.
 */
int uhnsw_load(const float* base, int64_t n, int32_t d, const uhnsw_graph* g1,
               const uhnsw_graph* g2, const uhnsw_load_opts* opts, uhnsw_index** out);

/*
 * Algorithm 1 for a batch of nq queries.
 *   q          device, nq x d float32 row-major
 *   p          device [nq] float32, each in (0, 2]
 *   k          device [nq] int32 in [1, k_max], or NULL (all k_max)
 *   ef         device [nq] int32 >= 1, or NULL (all ef_default)
 *   k_max      row stride of the outputs, 1 <= k_max <= UHNSW_MAX_EF
 *   out_ids    device, nq x k_max int64
 *   out_dist   device, nq x k_max float32 (L_p distance S^(1/p))
 *   opts       may be NULL (defaults above)
 * The beam of a query holds ef' = max(ef, t', k) entries, t' = max(t or ef, k)
 * for general p, t' = k when p is a graph's base p.  For such a p the first k
 * beam entries are returned directly when the beam ran on the FP32 rows or on an
 * FP16/BF16 copy that holds every value exactly (checked at load); with an
 * inexact copy the whole beam is re-ranked by its FP32 base distance, so
 * returned distances are always FP32 ones.  ef' above the launch bound
 * (opts->ef_max, or ef_default) or UHNSW_MAX_EF, an invalid p or k, fails that
 * query alone (status EINVAL in stats, outputs padded).
 * Errors: EINVAL (host-checkable arguments), ECUDA.
 */
int uhnsw_search(uhnsw_index* idx, const float* q, const float* p, const int32_t* k,
                 const int32_t* ef, int64_t nq, int32_t k_max, int32_t ef_default,
                 const uhnsw_search_opts* opts, int64_t* out_ids, float* out_dist,
                 void* stream);

/*
 * uhnsw_search with HOST arrays: q (nq x d), p, k, ef (or NULL), the outputs
 * and opts->t_per_query / tau_per_query (if set) are host memory (pinned
 * memory makes the copies asynchronous).  The call
 * copies the inputs to device staging buffers that the index holds for
 * `stream`, runs the search on `stream` and copies the results back; it
 * returns after the stream has synchronised.  opts->use_graph is ignored.
 * Calls on different streams may run concurrently; calls on one stream from
 * several threads are serialised by the index.
 */
int uhnsw_search_host(uhnsw_index* idx, const float* q, const float* p, const int32_t* k,
                      const int32_t* ef, int64_t nq, int32_t k_max, int32_t ef_default,
                      const uhnsw_search_opts* opts, int64_t* out_ids, float* out_dist,
                      void* stream);

/*
 * uhnsw_search_host without the final wait: returns once the copies in, the
 * search and the copies out are queued on `stream`.  The host inputs must
 * stay unchanged and the outputs unread until `stream` has synchronised (an
 * event recorded after the call marks completion).  With pinned host buffers
 * the copies run asynchronously, so batches queued on two streams overlap
 * one batch's copies and search with the other's.  A call whose staging must
 * grow first waits for the stream's earlier work.  Not capturable in a CUDA
 * graph.  Errors as uhnsw_search_host.
 */
int uhnsw_search_host_async(uhnsw_index* idx, const float* q, const float* p, const int32_t* k,
                            const int32_t* ef, int64_t nq, int32_t k_max, int32_t ef_default,
                            const uhnsw_search_opts* opts, int64_t* out_ids, float* out_dist,
                            void* stream);

/*
 * Candidate verification alone (Algorithm 1 lines 6-10, or the exact mode) on
 * caller-given candidate sets, for testing the re-ranking step in isolation.
 *   q      device nq x d float32;  p device [nq] float32 in (0, 2]
 *   cand   device nq x t int32 base ids in C's order (-1 = absent slot; no
 *          duplicates within a row)
 *   k      results per query, 1 <= k <= UHNSW_MAX_EF
 *   opts   uses verify_mode, kappa, tau and stats (NP / TERMS / STATUS); may be NULL
 *   out_ids / out_dist   device nq x k int64 / float32
 * Errors: EINVAL, ECUDA.
 */
int uhnsw_verify(uhnsw_index* idx, const float* q, const float* p, const int32_t* cand, int32_t t,
                 int32_t k, int64_t nq, const uhnsw_search_opts* opts, int64_t* out_ids,
                 float* out_dist, void* stream);

/*
 * Exhaustive L_p k-NN over all n base vectors of the FP32 master copy (the
 * exact answer the recall of Section 4.1.2 is measured against), computed on
 * the GPU.
 *   q device nq x d float32; p device [nq]; k in [1, 256];
 *   out_ids / out_dist device nq x k.
 * Uses a device workspace owned by the index (grown on demand, freed by
 * uhnsw_free); not safe to run concurrently on one index.
 * Errors: EINVAL, EOOM, ECUDA.
 */
int uhnsw_exact(uhnsw_index* idx, const float* q, const float* p, int64_t nq, int32_t k,
                int64_t* out_ids, float* out_dist, void* stream);

/*
 * Idealized recall of candidate sets (Section 3.2; the experiment the paper
 * uses to choose t).  For each query, counts[i][t-1] = |T_K ∩ B_t| for
 * t = 1 .. t_max, where T_K is the exact top-K under the query's own L_p and
 * B_t the exact top-t under the base metric of the graph the query is routed
 * to (cutoff as in uhnsw_search_opts, 0 => 1.4).  counts / K is the recall
 * that verifying the true top-t base-metric points would reach.
 *   q, p     device, nq x d and [nq]
 *   counts   device int32 [nq][t_max]; 1 <= K <= t_max <= 256
 * Allocates its scratch with cudaMalloc and returns after `stream` has
 * synchronised.  Errors: EINVAL, ECUDA.
 */
int uhnsw_idealized_recall(uhnsw_index* idx, const float* q, const float* p, int64_t nq,
                           int32_t K, int32_t t_max, float cutoff, int32_t* counts, void* stream);

/*
 * A t per p for a target recall, from idealized-recall curves (host code).
 * Bin b holds p in (p_lo + b w, p_lo + (b+1) w] (values outside go to the end
 * bins; a p within 1e-4 w of an upper edge counts as on it); out_t[b] is the smallest t whose mean idealized recall over the
 * sample queries of that bin reaches `target` (t_max if none does, 0 for an
 * empty bin).  Pass out_t's entries as uhnsw_search_opts.t_per_query for the
 * queries of each bin, with tau a little above the target (the paper takes
 * 0.92 for a target of 0.9).
 *   counts   host int32 [n][t_max] from uhnsw_idealized_recall; p host [n]
 * Errors: EINVAL.
 */
int uhnsw_plan_t(const int32_t* counts, const float* p, int64_t n, int32_t K, int32_t t_max,
                 float target, float p_lo, float bin_width, int32_t nbins, int32_t* out_t);

/*
 * uhnsw_exact for callers that cannot allocate device memory.  Such callers
 * include a serving loop that runs on a fixed, pre-reserved memory budget; a
 * process whose device memory is owned by another framework's caching
 * allocator; and latency-critical code that must not hit the device-wide
 * synchronisation a cudaMalloc or cudaFree can cause.  The paper has no
 * counterpart: this is an interface detail of this library.
 *
 * Identical arguments, results and errors as uhnsw_exact, except:
 *   - The per-slice partial lists live in one file-scope device array of
 *     UHNSW_EXACT_STATIC_BYTES bytes.  Every GPU that loads this library holds
 *     it until the process exits.  The call allocates nothing: no cudaMalloc,
 *     no cudaFree, no allocating library routine.
 *   - Sizes: nq * k * 8 bytes must not exceed UHNSW_EXACT_STATIC_BYTES;
 *     larger requests fail with UHNSW_ECAPACITY before any work is queued.
 *     Smaller requests may use fewer slices than uhnsw_exact; the result is
 *     the same.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it.  Make that first call before any
 *     stream capture begins.  The device must be the index's device.
 *   - All calls share the array.  It keeps the last call's contents; every
 *     slot a call reads is written by that call first, so nothing needs
 *     clearing.  Calls whose work overlaps on the GPU (several streams, or
 *     several host threads) race on the array: serialise them.
 */
#define UHNSW_EXACT_STATIC_BYTES (32 * 1024 * 1024)
int uhnsw_exact_static(uhnsw_index* idx, const float* q, const float* p, int64_t nq, int32_t k,
                       int64_t* out_ids, float* out_dist, void* stream);

/*
 * Autotuner of the launch configuration (the batched form's team size and
 * staging width).  Times every candidate on the caller's sample batch (device
 * q [nq][d], p [nq]; k and ef for all) with 1 warm-up and 3 timed launches on
 * `stream`, and records the fastest for the bucket (traversal dtype, beam
 * next_pow2(max(ef, k)), k next_pow2(k)) in the index; uhnsw_search with
 * opts->query_threads == 0 then uses it.  Candidates: the warp-per-query
 * kernel with each compiled team width that covers a row (8, 16, 32 lanes),
 * 4, 8 or 16 staged verification rows, the default visited table or one
 * twice its size, and a drop test every 1, 2 or 4 verification groups; the
 * block-per-query kernel with either table size.  The candidates run the same algorithm in the same
 * order; their distances can differ only by the FP32 summation order of the
 * team width (table size, staging and drop-test interval change no sum).
 * hash_bits and verify_groups set in `base` are kept, not searched.  `base` supplies the other options
 * (may be NULL); `best` (may be NULL) receives the chosen options and
 * `best_ms` (may be NULL) its median time.  The paper has no counterpart
 * (its queries run one at a time on a CPU).  Synchronises `stream`.
 * Errors: EINVAL, ECUDA.
 */
int uhnsw_autotune(uhnsw_index* idx, const float* q, const float* p, int64_t nq, int32_t k,
                   int32_t ef, const uhnsw_search_opts* base, void* stream,
                   uhnsw_search_opts* best, float* best_ms);

/* Writes / reads the tuned configurations as text lines
 * "dtype d ef_bucket k_bucket query_threads team_lanes stage_bytes hash_bits
 * verify_groups"; load keeps only lines matching this index's dtype and d
 * (lines of seven fields, without the last two, load with both 0). */
int uhnsw_autotune_save(const uhnsw_index* idx, const char* path);
int uhnsw_autotune_load(uhnsw_index* idx, const char* path);

/*
 * Index facts: n, d, padded row length, bytes held on the device, and the
 * device pointers of the layer-0 tables (for diagnostics).  Any out pointer
 * may be NULL.
 */
int uhnsw_index_info(const uhnsw_index* idx, int64_t* n, int32_t* d, int32_t* d_pad,
                     int64_t* device_bytes, int32_t* max_degree0);

/* Reads and clears the index's sticky device error word (synchronises the
 * device).  Returns UHNSW_OK or the first recorded code. */
int uhnsw_device_status(uhnsw_index* idx);

/* Frees every device and host allocation of the index (NULL is a no-op). */
void uhnsw_free(uhnsw_index* idx);

/* Message of the calling thread's last failed call ("" if none). */
const char* uhnsw_last_error(void);

/* ------------------------------------------------------------------------
 * Measurement probes: the peak rates that roofline fractions are stated
 * against, measured on the current device (not part of the query path; the
 * paper has no counterpart).  Each launches once untimed, then once between
 * two events on `stream`, and synchronises it.  Errors: EINVAL, ECUDA.
 * ---------------------------------------------------------------------- */

/* SFU rate of the general-p verification term 2^(p log2 |d|): blocks_per_sm
 * (1..64) blocks of 256 threads per SM, each thread running 8 independent
 * chains of `iters` links x <- 2^(c log2 x) (lg2.approx, ex2.approx).
 * *elapsed_ms = the timed launch; *ops = SFU operations it executed
 * (2 x 8 x iters x threads).  Allocates a small sink buffer. */
int uhnsw_probe_sfu(int32_t blocks_per_sm, int32_t iters, float* elapsed_ms, double* ops,
                    void* stream);

/* Random-row gather bandwidth: every warp of blocks_per_sm blocks of 256
 * threads per SM reads `per_warp` (a positive multiple of 128) rows of
 * `row_bytes` (a multiple of 16) bytes, chosen by a hash of (warp, i), with
 * 16-byte loads, four rows per lane group in flight.  buf: device, 16-byte
 * aligned, rows x row_bytes bytes (rows < 2^32).  A buffer smaller than L2
 * measures L2 gathers (after the untimed launch has warmed it); a larger one
 * measures HBM gathers.  *bytes = row bytes read by the timed launch.
 * Allocates a small sink buffer. */
int uhnsw_probe_gather(const void* buf, int64_t rows, int32_t row_bytes, int32_t per_warp,
                       int32_t blocks_per_sm, float* elapsed_ms, double* bytes, void* stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching over a resident index.  The paper answers one
 * query at a time (Section 4.1.2 measures per-query time); this server lets
 * requests that arrive while others are on the GPU join the next batch.
 * ---------------------------------------------------------------------- */

typedef struct uhnsw_server uhnsw_server;

typedef struct {
  int32_t max_batch;     /* queries per launch; 0 => 1024 */
  int32_t streams;       /* batches in flight at once (one stream each); 0 => 4 */
  int64_t state_budget;  /* bytes of search state (beam, visited table, verification lists
                            of every admitted, unfinished query) admitted at once;
                            0 => 2 * max_batch queries at ef_max / k_max */
  int32_t k_max;         /* largest k accepted; 0 => 100 */
  int32_t ef_max;        /* largest ef accepted; 0 => 512 */
  int32_t max_delay_us;  /* a partial batch waits at most this long for more requests
                            while other batches run; 0 => 200 */
  int32_t reserved;
  uhnsw_search_opts search; /* options of every launch (stats, use_graph, ef_max ignored) */
} uhnsw_server_opts;

typedef struct {
  int64_t completed;     /* requests finished since the server started */
  int64_t batches;       /* launches */
  double mean_batch;     /* queries per launch */
  int64_t peak_inflight; /* most queries admitted and unfinished at once */
  int64_t peak_state;    /* most search-state bytes admitted at once (<= state_budget
                            unless a single request exceeds it) */
  double mean_us, p50_us, p99_us, max_us; /* submit -> result on the host, over the last
                                             2^20 finished requests */
  int32_t error;         /* first failure of a launch (0 if none) */
  int32_t reserved;
} uhnsw_server_report;

/*
 * Starts a server on `idx` (which must outlive it) with a dispatcher and a
 * completion thread; allocates max_batch-query device and pinned host slots
 * per stream.  Uses the current device.  Errors: EINVAL, EOOM, ECUDA.
 */
int uhnsw_server_create(uhnsw_index* idx, const uhnsw_server_opts* opts, uhnsw_server** out);

/* Queues one request (q: host, d floats; copied) and returns its ticket.
 * Thread-safe.  Errors: EINVAL (p, k or ef outside the server's limits). */
int uhnsw_server_submit(uhnsw_server* s, const float* q, float p, int32_t k, int32_t ef,
                        uint64_t* ticket);

/* Non-blocking: *done = 1 and the k results copied out (ticket released) once
 * finished, else *done = 0. */
int uhnsw_server_poll(uhnsw_server* s, uint64_t ticket, int64_t* ids, float* dist, int32_t* done);

/* Blocks until the request finishes (or timeout_ms: UHNSW_ETIMEOUT).  A
 * ticket released meanwhile by another poll / wait gives UHNSW_EINVAL. */
int uhnsw_server_wait(uhnsw_server* s, uint64_t ticket, int64_t* ids, float* dist,
                      int32_t timeout_ms);

/*
 * Request loop: submits nq requests (host arrays q [nq][d], p, k, ef) at the
 * times arrival_us[i] (microseconds after the call starts, ascending), then
 * waits for all of them.  Results go to out_ids / out_dist [nq][k_max]
 * (padded with -1 / +inf past each k), latency_us[i] = submit -> result.
 * Any output pointer may be NULL.
 */
int uhnsw_server_replay(uhnsw_server* s, const float* q, const float* p, const int32_t* k,
                        const int32_t* ef, int64_t nq, const double* arrival_us,
                        int64_t* out_ids, float* out_dist, double* latency_us,
                        int32_t timeout_ms);

int uhnsw_server_stats(uhnsw_server* s, uhnsw_server_report* out);

/* Stops the threads, waits for batches in flight and frees the slots. */
void uhnsw_server_destroy(uhnsw_server* s);

/* ------------------------------------------------------------------------
 * Index construction (Section 2.2, the HNSW insertion the paper builds G1 and
 * G2 with): host-side and multi-threaded; not part of the query path.
 * ---------------------------------------------------------------------- */

typedef struct uhnsw_built uhnsw_built;

/*
 * Build one HNSW graph on the host.
 *   base      host n x d float32 row-major (read during the call only)
 *   metric    a uhnsw_base_metric: 1 = L1 (G1), 2 = squared L2 (G2), 3 = L0.5
 *             (G0.5 of U-HNSW-E), 4 = L1.5
 *   M         links per inserted node; layer-0 lists hold up to 2M
 *   ef_construction   beam width of the insertion search
 *   levels    host [n] int32, the level of each node (drawn by the caller)
 *   threads   worker threads (<= 0: all hardware threads); with 1 thread the
 *             insertion order, and so the graph, is deterministic
 *   out       receives the graph; read it with uhnsw_built_graph, free it with
 *             uhnsw_built_free
 * Errors: EINVAL, EOOM.
 */
int uhnsw_build_graph(const float* base, int64_t n, int32_t d, int32_t metric, int32_t M,
                      int32_t ef_construction, const int32_t* levels, int32_t threads,
                      uhnsw_built** out);

/*
 * The same construction on the current CUDA device (Section 2.2's graphs,
 * built for inputs too large for the host builder).  Nodes are inserted in
 * batches: a batch searches the graph of the nodes before it (one warp per
 * new node, efConstruction beam, the neighbour heuristic), then its reverse
 * links are applied row by row, re-selecting a row past its cap with the
 * heuristic.  A batch holds 1/16 of the nodes already inserted (1 to 65,536),
 * and its nodes do not link to each other directly, so the graph differs
 * from a one-at-a-time build; it is the same on every run.  Arguments as
 * uhnsw_build_graph (host arrays), with 1 <= ef_construction <= 512.  Device
 * memory: about n (4 d + 8 M + 520) bytes while it runs.  Returns after the
 * device work has finished.  Errors: EINVAL, EOOM, ECUDA, ECAPACITY.
 */
int uhnsw_build_graph_gpu(const float* base, int64_t n, int32_t d, int32_t metric, int32_t M,
                          int32_t ef_construction, const int32_t* levels, uhnsw_built** out);

/*
 * Build one HNSW graph under L_p for any 0 < p <= 2 (the fixed-p HNSW of
 * Section 4.3: a graph per p, searched directly at that p).  The graph is
 * built with S_p = sum_j |d_j|^p, which orders points exactly like L_p; p =
 * 1, 2, 0.5 and 1.5 use their own closed forms (metric codes 1-4), any other
 * p a power (std::pow on the host, the fast power intrinsic on the device).
 * Load it with base_metric UHNSW_BASE_LP and base_p = p in its slot.
 *   on_device  0: uhnsw_build_graph on the host with `threads` workers;
 *              1: uhnsw_build_graph_gpu on the current CUDA device
 * Other arguments as uhnsw_build_graph.  Errors: EINVAL (p outside (0, 2],
 * or as the builder chosen), EOOM, ECUDA, ECAPACITY.
 */
int uhnsw_build_graph_lp(const float* base, int64_t n, int32_t d, float p, int32_t M,
                         int32_t ef_construction, const int32_t* levels, int32_t threads,
                         int32_t on_device, uhnsw_built** out);

/* Fills `view` with host pointers into the built graph (valid until
 * uhnsw_built_free); level 0 lists every node, so level_nodes[0] is NULL. */
int uhnsw_built_graph(const uhnsw_built* b, uhnsw_graph* view);

void uhnsw_built_free(uhnsw_built* b);

#ifdef __cplusplus
}
#endif

#endif /* UHNSW_H_ */
