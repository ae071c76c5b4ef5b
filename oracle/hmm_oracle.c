/*
 * hmm_oracle.c -- plain FP64 log-space CPU oracle (see hmm_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py, never by the product path.
 *
 * Every recursion below is the textbook definition written out in log space
 * with a max-shifted log-sum-exp, one sequence at a time, one model at a time,
 * with no blocking, fusion or rescaling (Rabiner 1989 eqs. 19-21, 24-25,
 * 32-35, 37-38, 40). The only parallelism is over whole sequences, with
 * pthreads; per-thread count buffers are summed in thread order.
 */
#include "hmm_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* log-space helpers                                                         */
/* ------------------------------------------------------------------------ */

static double safe_log(double p) { return p > 0.0 ? log(p) : -INFINITY; }

/* log(sum_i exp(x_i)), max-shifted; all -inf gives -inf. */
static double log_sum_exp(const double* x, int n) {
  double m = -INFINITY;
  for (int i = 0; i < n; ++i)
    if (x[i] > m) m = x[i];
  if (m == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += exp(x[i] - m);
  return m + log(s);
}

typedef struct {
  int N, M;
  const double* lpi; /* [N]   */
  const double* lA;  /* [N][N] */
  const double* lB;  /* [N][M] */
} lmodel_t;

typedef struct {
  int K, N, M;
  double* lpi; /* [K][N] */
  double* lA;  /* [K][N][N] */
  double* lB;  /* [K][N][M] */
} lparams_t;

static int make_lparams(lparams_t* p, int K, int N, int M, const double* pi,
                        const double* A, const double* B) {
  p->K = K;
  p->N = N;
  p->M = M;
  p->lpi = (double*)malloc(sizeof(double) * (size_t)K * N);
  p->lA = (double*)malloc(sizeof(double) * (size_t)K * N * N);
  p->lB = (double*)malloc(sizeof(double) * (size_t)K * N * M);
  if (!p->lpi || !p->lA || !p->lB) return ORC_ERR_ARG;
  for (size_t i = 0; i < (size_t)K * N; ++i) p->lpi[i] = safe_log(pi[i]);
  for (size_t i = 0; i < (size_t)K * N * N; ++i) p->lA[i] = safe_log(A[i]);
  for (size_t i = 0; i < (size_t)K * N * M; ++i) p->lB[i] = safe_log(B[i]);
  return ORC_OK;
}

static void free_lparams(lparams_t* p) {
  free(p->lpi);
  free(p->lA);
  free(p->lB);
}

static lmodel_t model_k(const lparams_t* p, int k) {
  lmodel_t m;
  m.N = p->N;
  m.M = p->M;
  m.lpi = p->lpi + (size_t)k * p->N;
  m.lA = p->lA + (size_t)k * p->N * p->N;
  m.lB = p->lB + (size_t)k * p->N * p->M;
  return m;
}

static int symbols_ok(const int32_t* o, int64_t T, int M) {
  for (int64_t t = 0; t < T; ++t)
    if (o[t] < 0 || o[t] >= M) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* single-sequence recursions                                                */
/* ------------------------------------------------------------------------ */

/* Forward variable in log space (Rabiner eqs. 19-21):
 *   la_1(i) = log pi_i + log b_i(o_1)
 *   la_t(j) = LSE_i(la_{t-1}(i) + log a_ij) + log b_j(o_t)
 *   log P(O) = LSE_i la_T(i).
 * la_all, if not NULL, receives la_t for every t ([T][N]). */
static double seq_forward(const lmodel_t* m, const int32_t* o, int64_t T, double* la_all,
                          double* work /* 3N */) {
  const int N = m->N, M = m->M;
  if (T == 0) return 0.0;
  double* prev = work;
  double* cur = work + N;
  double* tmp = work + 2 * N;
  for (int i = 0; i < N; ++i) prev[i] = m->lpi[i] + m->lB[(size_t)i * M + o[0]];
  if (la_all) memcpy(la_all, prev, sizeof(double) * N);
  for (int64_t t = 1; t < T; ++t) {
    for (int j = 0; j < N; ++j) {
      for (int i = 0; i < N; ++i) tmp[i] = prev[i] + m->lA[(size_t)i * N + j];
      cur[j] = log_sum_exp(tmp, N) + m->lB[(size_t)j * M + o[t]];
    }
    double* sw = prev;
    prev = cur;
    cur = sw;
    if (la_all) memcpy(la_all + (size_t)t * N, prev, sizeof(double) * N);
  }
  return log_sum_exp(prev, N);
}

/* Viterbi in log space (Rabiner eqs. 32-35), with the smallest index taken on
 * ties, plus the score of the second-best complete path (list Viterbi that
 * keeps the two best partial paths into every state).
 *   d_1(i)   = log pi_i + log b_i(o_1)
 *   d_t(j)   = max_i(d_{t-1}(i) + log a_ij) + log b_j(o_t)
 *   psi_t(j) = smallest maximising i
 *   q_T = smallest argmax_j d_T(j); q_t = psi_{t+1}(q_{t+1}). */
static double seq_viterbi(const lmodel_t* m, const int32_t* o, int64_t T, int32_t* path,
                          double* second, int32_t* psi /* [T][N] */,
                          double* work /* 4N */) {
  const int N = m->N, M = m->M;
  if (T == 0) {
    if (second) *second = -INFINITY;
    return 0.0;
  }
  double* d1 = work;          /* best partial path score into each state */
  double* d2 = work + N;      /* second best */
  double* n1 = work + 2 * N;
  double* n2 = work + 3 * N;
  for (int i = 0; i < N; ++i) {
    d1[i] = m->lpi[i] + m->lB[(size_t)i * M + o[0]];
    d2[i] = -INFINITY;
    psi[i] = 0;
  }
  for (int64_t t = 1; t < T; ++t) {
    for (int j = 0; j < N; ++j) {
      double best = -INFINITY, sec = -INFINITY;
      int arg = 0;
      for (int i = 0; i < N; ++i) {
        const double la = m->lA[(size_t)i * N + j];
        const double v1 = d1[i] + la;
        const double v2 = d2[i] + la;
        /* candidate v1 */
        if (v1 > best) {
          sec = best;
          best = v1;
          arg = i;
        } else if (v1 > sec) {
          sec = v1;
        }
        /* candidate v2 can only ever be a second best: v2 <= v1 <= best */
        if (v2 > sec) sec = v2;
      }
      const double lb = m->lB[(size_t)j * M + o[t]];
      n1[j] = best + lb;
      n2[j] = sec + lb;
      psi[(size_t)t * N + j] = arg;
    }
    memcpy(d1, n1, sizeof(double) * N);
    memcpy(d2, n2, sizeof(double) * N);
  }
  double best = -INFINITY, sec = -INFINITY;
  int q = 0;
  for (int j = 0; j < N; ++j) {
    if (d1[j] > best) {
      sec = best;
      best = d1[j];
      q = j;
    } else if (d1[j] > sec) {
      sec = d1[j];
    }
    if (d2[j] > sec) sec = d2[j];
  }
  if (second) *second = sec;
  if (path) {
    if (best == -INFINITY) {
      for (int64_t t = 0; t < T; ++t) path[t] = 0;
    } else {
      path[T - 1] = q;
      for (int64_t t = T - 1; t > 0; --t) {
        q = psi[(size_t)t * N + q];
        path[t - 1] = q;
      }
    }
  }
  return best;
}

/* Expected counts of one sequence, weighted by w, added into cpi/cA/cB
 * (Rabiner eqs. 24-25 backward variable, 37 xi, 38 gamma):
 *   lb_T(i) = 0, lb_t(i) = LSE_j(log a_ij + log b_j(o_{t+1}) + lb_{t+1}(j))
 *   gamma_t(i)  = exp(la_t(i) + lb_t(i) - log P)
 *   xi_t(i,j)   = exp(la_t(i) + log a_ij + log b_j(o_{t+1}) + lb_{t+1}(j) - log P)
 *   C_pi += w gamma_1, C_A += w sum_{t<T} xi_t, C_B[:,k] += w sum_{t:o_t=k} gamma_t.
 * Returns log P. */
static double seq_counts(const lmodel_t* m, const int32_t* o, int64_t T, double w,
                         double* cpi, double* cA, double* cB, double* la /* [T][N] */,
                         double* lbv /* [T][N] */, double* work /* 3N */) {
  const int N = m->N, M = m->M;
  if (T == 0) return 0.0;
  const double lp = seq_forward(m, o, T, la, work);
  if (lp == -INFINITY) return lp; /* impossible: no counts */
  double* tmp = work;
  for (int i = 0; i < N; ++i) lbv[(size_t)(T - 1) * N + i] = 0.0;
  for (int64_t t = T - 2; t >= 0; --t) {
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j)
        tmp[j] = m->lA[(size_t)i * N + j] + m->lB[(size_t)j * M + o[t + 1]] +
                 lbv[(size_t)(t + 1) * N + j];
      lbv[(size_t)t * N + i] = log_sum_exp(tmp, N);
    }
  }
  for (int64_t t = 0; t < T; ++t) {
    for (int i = 0; i < N; ++i) {
      const double g = exp(la[(size_t)t * N + i] + lbv[(size_t)t * N + i] - lp);
      if (t == 0) cpi[i] += w * g;
      cB[(size_t)i * M + o[t]] += w * g;
      if (t + 1 < T) {
        for (int j = 0; j < N; ++j) {
          const double x = la[(size_t)t * N + i] + m->lA[(size_t)i * N + j] +
                           m->lB[(size_t)j * M + o[t + 1]] + lbv[(size_t)(t + 1) * N + j] - lp;
          cA[(size_t)i * N + j] += w * exp(x);
        }
      }
    }
  }
  return lp;
}

/* ------------------------------------------------------------------------ */
/* thread pool over contiguous unit ranges                                   */
/* ------------------------------------------------------------------------ */

typedef void (*range_fn)(void* ctx, int tid, int64_t begin, int64_t end);

typedef struct {
  range_fn fn;
  void* ctx;
  int tid;
  int64_t begin, end;
} range_job_t;

static void* range_trampoline(void* arg) {
  range_job_t* j = (range_job_t*)arg;
  j->fn(j->ctx, j->tid, j->begin, j->end);
  return NULL;
}

static void parallel_ranges(int nthreads, int64_t n, range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads == 1) {
    fn(ctx, 0, 0, n);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  range_job_t* jobs = (range_job_t*)malloc(sizeof(range_job_t) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].tid = t;
    jobs[t].begin = n * t / nthreads;
    jobs[t].end = n * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, range_trampoline, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ------------------------------------------------------------------------ */
/* batch drivers                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  const lparams_t* lp;
  const int32_t* symbols;
  const int64_t* offsets;
  const int32_t* lengths;
  int S;
  const int32_t* model_of_seq;
  double* out;       /* loglik or score */
  int32_t* argmax;   /* forward: argmax; viterbi: best model */
  int32_t* path;
  double* margin;
  const double* weight;
  double* cnt; /* per-thread count buffers */
  int bad_symbol;
} batch_ctx_t;

static int64_t max_len_of(const int32_t* lengths, int S) {
  int64_t mx = 0;
  for (int s = 0; s < S; ++s)
    if (lengths[s] > mx) mx = lengths[s];
  return mx;
}

static void forward_range(void* vctx, int tid, int64_t begin, int64_t end) {
  (void)tid;
  batch_ctx_t* c = (batch_ctx_t*)vctx;
  const int K = c->lp->K, N = c->lp->N;
  double* work = (double*)malloc(sizeof(double) * 3 * N);
  for (int64_t s = begin; s < end; ++s) {
    const int32_t* o = c->symbols + c->offsets[s];
    const int64_t T = c->lengths[s];
    const int ok = symbols_ok(o, T, c->lp->M);
    if (!ok) c->bad_symbol = 1;
    if (c->model_of_seq) {
      lmodel_t m = model_k(c->lp, c->model_of_seq[s]);
      c->out[s] = ok ? seq_forward(&m, o, T, NULL, work) : NAN;
    } else {
      int any_nan = 0;
      for (int k = 0; k < K; ++k) {
        lmodel_t m = model_k(c->lp, k);
        const double v = ok ? seq_forward(&m, o, T, NULL, work) : NAN;
        c->out[s * K + k] = v;
        if (isnan(v)) any_nan = 1;
      }
      /* argmax with the smallest k on ties (Sec. 2.7: the recognised activity
       * is the best-scoring per-activity model) */
      double best = c->out[s * K];
      int arg = 0;
      for (int k = 1; k < K; ++k)
        if (c->out[s * K + k] > best) {
          best = c->out[s * K + k];
          arg = k;
        }
      if (c->argmax) c->argmax[s] = any_nan ? -1 : arg;
    }
  }
  free(work);
}

int orc_forward(int K, int N, int M, const double* pi, const double* A, const double* B,
                const int32_t* symbols, const int64_t* offsets, const int32_t* lengths,
                int S, const int32_t* model_of_seq, double* loglik, int32_t* argmax,
                int nthreads) {
  if (K < 1 || N < 1 || M < 1 || S < 0) return ORC_ERR_ARG;
  lparams_t lp;
  if (make_lparams(&lp, K, N, M, pi, A, B) != ORC_OK) return ORC_ERR_ARG;
  batch_ctx_t c;
  memset(&c, 0, sizeof(c));
  c.lp = &lp;
  c.symbols = symbols;
  c.offsets = offsets;
  c.lengths = lengths;
  c.S = S;
  c.model_of_seq = model_of_seq;
  c.out = loglik;
  c.argmax = argmax;
  parallel_ranges(nthreads, S, forward_range, &c);
  free_lparams(&lp);
  return c.bad_symbol ? ORC_ERR_SYMBOL : ORC_OK;
}

static void viterbi_range(void* vctx, int tid, int64_t begin, int64_t end) {
  (void)tid;
  batch_ctx_t* c = (batch_ctx_t*)vctx;
  const int K = c->lp->K, N = c->lp->N;
  const int64_t Tmax = max_len_of(c->lengths, c->S);
  double* work = (double*)malloc(sizeof(double) * 4 * N);
  int32_t* psi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(Tmax > 0 ? Tmax : 1) * N);
  for (int64_t s = begin; s < end; ++s) {
    const int32_t* o = c->symbols + c->offsets[s];
    const int64_t T = c->lengths[s];
    const int ok = symbols_ok(o, T, c->lp->M);
    if (!ok) c->bad_symbol = 1;
    int best_k;
    if (c->model_of_seq) {
      best_k = c->model_of_seq[s];
    } else {
      /* scores for every model, then the smallest k among the maximal */
      double best = -INFINITY;
      int any_nan = 0;
      best_k = 0;
      for (int k = 0; k < K; ++k) {
        lmodel_t m = model_k(c->lp, k);
        const double v = ok ? seq_viterbi(&m, o, T, NULL, NULL, psi, work) : NAN;
        c->out[s * K + k] = v;
        if (isnan(v)) any_nan = 1;
        if (k == 0 || v > best) {
          if (k == 0) best = v;
          else {
            best = v;
            best_k = k;
          }
        }
      }
      if (any_nan) best_k = -1;
    }
    if (c->argmax) c->argmax[s] = best_k;
    if (best_k < 0 || !ok) {
      if (c->model_of_seq) c->out[s] = NAN;
      if (c->margin) c->margin[s] = NAN;
      if (c->path)
        for (int64_t t = 0; t < T; ++t) c->path[c->offsets[s] + t] = -1;
      continue;
    }
    lmodel_t m = model_k(c->lp, best_k);
    double second = -INFINITY;
    const double v = seq_viterbi(&m, o, T, c->path ? c->path + c->offsets[s] : NULL, &second,
                                 psi, work);
    if (c->model_of_seq) c->out[s] = v;
    if (c->margin) c->margin[s] = (second == -INFINITY) ? INFINITY : v - second;
  }
  free(work);
  free(psi);
}

int orc_viterbi(int K, int N, int M, const double* pi, const double* A, const double* B,
                const int32_t* symbols, const int64_t* offsets, const int32_t* lengths,
                int S, const int32_t* model_of_seq, double* score, int32_t* best_model,
                int32_t* path, double* margin, int nthreads) {
  if (K < 1 || N < 1 || M < 1 || S < 0) return ORC_ERR_ARG;
  lparams_t lp;
  if (make_lparams(&lp, K, N, M, pi, A, B) != ORC_OK) return ORC_ERR_ARG;
  batch_ctx_t c;
  memset(&c, 0, sizeof(c));
  c.lp = &lp;
  c.symbols = symbols;
  c.offsets = offsets;
  c.lengths = lengths;
  c.S = S;
  c.model_of_seq = model_of_seq;
  c.out = score;
  c.argmax = best_model;
  c.path = path;
  c.margin = margin;
  parallel_ranges(nthreads, S, viterbi_range, &c);
  free_lparams(&lp);
  return c.bad_symbol ? ORC_ERR_SYMBOL : ORC_OK;
}

static void fb_range(void* vctx, int tid, int64_t begin, int64_t end) {
  batch_ctx_t* c = (batch_ctx_t*)vctx;
  const int K = c->lp->K, N = c->lp->N, M = c->lp->M;
  const int64_t Tmax = max_len_of(c->lengths, c->S);
  const size_t per = (size_t)N + (size_t)N * N + (size_t)N * M;
  double* cnt = c->cnt + (size_t)tid * K * per;
  double* work = (double*)malloc(sizeof(double) * 3 * N);
  const size_t tn = (size_t)(Tmax > 0 ? Tmax : 1) * N;
  double* la = (double*)malloc(sizeof(double) * tn);
  double* lbv = (double*)malloc(sizeof(double) * tn);
  for (int64_t s = begin; s < end; ++s) {
    const int32_t* o = c->symbols + c->offsets[s];
    const int64_t T = c->lengths[s];
    const int ok = symbols_ok(o, T, M);
    if (!ok) c->bad_symbol = 1;
    const int k0 = c->model_of_seq ? c->model_of_seq[s] : 0;
    const int k1 = c->model_of_seq ? k0 + 1 : K;
    for (int k = k0; k < k1; ++k) {
      const size_t oi = c->model_of_seq ? (size_t)s : (size_t)s * K + k;
      if (!ok) {
        c->out[oi] = NAN;
        continue;
      }
      const double w = c->weight ? c->weight[oi] : 1.0;
      lmodel_t m = model_k(c->lp, k);
      double* base = cnt + (size_t)k * per;
      c->out[oi] = seq_counts(&m, o, T, w, base, base + N, base + N + (size_t)N * N, la, lbv,
                              work);
    }
  }
  free(work);
  free(la);
  free(lbv);
}

int orc_forward_backward(int K, int N, int M, const double* pi, const double* A,
                         const double* B, const int32_t* symbols, const int64_t* offsets,
                         const int32_t* lengths, int S, const int32_t* model_of_seq,
                         const double* weight, double* loglik, double* cnt_pi,
                         double* cnt_A, double* cnt_B, int nthreads) {
  if (K < 1 || N < 1 || M < 1 || S < 0) return ORC_ERR_ARG;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > S && S > 0) nthreads = S;
  lparams_t lp;
  if (make_lparams(&lp, K, N, M, pi, A, B) != ORC_OK) return ORC_ERR_ARG;
  const size_t per = (size_t)N + (size_t)N * N + (size_t)N * M;
  batch_ctx_t c;
  memset(&c, 0, sizeof(c));
  c.lp = &lp;
  c.symbols = symbols;
  c.offsets = offsets;
  c.lengths = lengths;
  c.S = S;
  c.model_of_seq = model_of_seq;
  c.out = loglik;
  c.weight = weight;
  c.cnt = (double*)calloc((size_t)nthreads * K * per, sizeof(double));
  parallel_ranges(nthreads, S, fb_range, &c);
  for (int k = 0; k < K; ++k) {
    for (int i = 0; i < N; ++i) cnt_pi[(size_t)k * N + i] = 0.0;
    for (size_t e = 0; e < (size_t)N * N; ++e) cnt_A[(size_t)k * N * N + e] = 0.0;
    for (size_t e = 0; e < (size_t)N * M; ++e) cnt_B[(size_t)k * N * M + e] = 0.0;
    for (int t = 0; t < nthreads; ++t) {
      const double* base = c.cnt + ((size_t)t * K + k) * per;
      for (int i = 0; i < N; ++i) cnt_pi[(size_t)k * N + i] += base[i];
      for (size_t e = 0; e < (size_t)N * N; ++e) cnt_A[(size_t)k * N * N + e] += base[N + e];
      for (size_t e = 0; e < (size_t)N * M; ++e)
        cnt_B[(size_t)k * N * M + e] += base[N + (size_t)N * N + e];
    }
  }
  free(c.cnt);
  free_lparams(&lp);
  return c.bad_symbol ? ORC_ERR_SYMBOL : ORC_OK;
}

/* g_ij = C_ij - p_ij * sum_j' C_ij' for every row of every table: the chain
 * rule through p_i. = softmax(theta_i.), using d log P / d p_ij = C_ij / p_ij. */
static void rows_grad(const double* p, const double* C, double* g, size_t rows, int width) {
  for (size_t r = 0; r < rows; ++r) {
    double tot = 0.0;
    for (int c = 0; c < width; ++c) tot += C[r * width + c];
    for (int c = 0; c < width; ++c) g[r * width + c] = C[r * width + c] - p[r * width + c] * tot;
  }
}

void orc_softmax_grad(int K, int N, int M, const double* pi, const double* A,
                      const double* B, const double* cnt_pi, const double* cnt_A,
                      const double* cnt_B, double* g_pi, double* g_A, double* g_B) {
  rows_grad(pi, cnt_pi, g_pi, (size_t)K, N);
  rows_grad(A, cnt_A, g_A, (size_t)K * N, N);
  rows_grad(B, cnt_B, g_B, (size_t)K * N, M);
}

static void rows_normalise(const double* p, const double* C, double* out, size_t rows,
                           int width) {
  for (size_t r = 0; r < rows; ++r) {
    double tot = 0.0;
    for (int c = 0; c < width; ++c) tot += C[r * width + c];
    for (int c = 0; c < width; ++c)
      out[r * width + c] = tot > 0.0 ? C[r * width + c] / tot : p[r * width + c];
  }
}

void orc_mstep(int K, int N, int M, const double* pi, const double* A, const double* B,
               const double* cnt_pi, const double* cnt_A, const double* cnt_B,
               double* pi_out, double* A_out, double* B_out) {
  rows_normalise(pi, cnt_pi, pi_out, (size_t)K, N);
  rows_normalise(A, cnt_A, A_out, (size_t)K * N, N);
  rows_normalise(B, cnt_B, B_out, (size_t)K * N, M);
}
