/*
 * U-HNSW oracle, TEST INFRASTRUCTURE ONLY: a batch driver that runs the
 * oracle's own Algorithm 1 (oracle_uhnsw_query in uhnsw_oracle.c, unchanged)
 * over a batch of queries on several host threads, so that the CPU baseline
 * can be timed on all of a machine's cores.  Each query is answered by one
 * single-threaded call; thread j takes queries j, j + T, j + 2T, ...  The
 * oracle keeps no global state, so the calls are independent and the results
 * equal a one-thread loop query for query.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct oracle_csr oracle_csr;

int oracle_uhnsw_query(const oracle_csr* ga, const oracle_csr* gb, int32_t ma, int32_t mb,
                       const float* base, int32_t d, const float* q, float p, int32_t k,
                       int32_t ef, int32_t t, float tau, int32_t kappa, float cutoff,
                       int32_t mode, int64_t* out_ids, double* out_dist, int64_t* stats);

typedef struct {
  const oracle_csr *ga, *gb;
  int32_t ma, mb;
  const float* base;
  int32_t d;
  const float* Q;
  const float* P;
  int64_t nq;
  int32_t k, ef, t;
  float tau;
  int32_t kappa;
  float cutoff;
  int32_t mode;
  int64_t* out_ids;
  double* out_dist;
  int32_t nthreads;
  int32_t tid;
  int status;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* j = (batch_job*)arg;
  j->status = 0;
  for (int64_t i = j->tid; i < j->nq; i += j->nthreads) {
    int rc = oracle_uhnsw_query(j->ga, j->gb, j->ma, j->mb, j->base, j->d, j->Q + i * j->d,
                                j->P[i], j->k, j->ef, j->t, j->tau, j->kappa, j->cutoff, j->mode,
                                j->out_ids + i * j->k, j->out_dist + i * j->k, NULL);
    if (rc != 0) {
      j->status = rc;
      break;
    }
  }
  return NULL;
}

/* Q [nq][d], P [nq]; out_ids / out_dist [nq][k].  Returns 0, the first
 * failing query's status, or -2 when a thread cannot be started. */
int oracle_uhnsw_batch_threads(const oracle_csr* ga, const oracle_csr* gb, int32_t ma, int32_t mb,
                               const float* base, int32_t d, const float* Q, const float* P,
                               int64_t nq, int32_t k, int32_t ef, int32_t t, float tau,
                               int32_t kappa, float cutoff, int32_t mode, int32_t nthreads,
                               int64_t* out_ids, double* out_dist) {
  if (nthreads < 1) nthreads = 1;
  batch_job* jobs = (batch_job*)calloc((size_t)nthreads, sizeof(batch_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -2;
  }
  int started = 0, status = 0;
  for (int32_t i = 0; i < nthreads; ++i) {
    batch_job j = {ga, gb, ma, mb, base, d, Q, P, nq, k, ef, t, tau, kappa, cutoff, mode,
                   out_ids, out_dist, nthreads, i, 0};
    jobs[i] = j;
  }
  for (int32_t i = 0; i < nthreads; ++i) {
    if (pthread_create(&th[i], NULL, batch_worker, &jobs[i]) != 0) {
      status = -2;
      break;
    }
    started++;
  }
  for (int32_t i = 0; i < started; ++i) pthread_join(th[i], NULL);
  for (int32_t i = 0; i < started && status == 0; ++i)
    if (jobs[i].status != 0) status = jobs[i].status;
  free(jobs);
  free(th);
  return status;
}
