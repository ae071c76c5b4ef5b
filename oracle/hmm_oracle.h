/*
 * hmm_oracle.h -- plain FP64 log-space CPU oracle for discrete-HMM scoring,
 * decoding and expected counts.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this library: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg do. It shares no code, header, table or helper with the CUDA
 * library under paper_1310_3322_gb300/csrc/.
 *
 * What it computes (the paper, Sec. 2.7, names the Forward, Viterbi and
 * Baum-Welch kernels of its HMM recognition stage but prints no equations;
 * the definitions followed are the textbook ones, Rabiner, "A Tutorial on
 * Hidden Markov Models and Selected Applications in Speech Recognition",
 * Proc. IEEE 77(2), 1989):
 *   forward      log P(O | lambda)                   Rabiner eqs. 19-21
 *   viterbi      max_Q log P(O, Q | lambda), Q*      Rabiner eqs. 32-35
 *   second best  log P of the second-best full path (list Viterbi)
 *   counts       sum_s w_s E[n_pi], E[n_ij], E[n_jk]  Rabiner eqs. 24-25, 37-38
 *   softmax grad d(sum_s w_s log P)/d(row logits)    chain rule through softmax
 *   M-step       row-normalised counts                Rabiner eq. 40
 *
 * Conventions (shared with the CUDA path by specification only):
 *   pi[K][N], A[K][N][N] (row i = from-state, a_ij = P(q_{t+1}=j | q_t=i)),
 *   B[K][N][M] (row j = P(symbol | state j)), all FP64 probabilities.
 *   Sequence s: symbols[offsets[s] .. offsets[s]+lengths[s]), 0-based in [0,M).
 *   model_of_seq == NULL scores every sequence against every model (outputs
 *   [S][K]); otherwise only against model_of_seq[s] (outputs [S]).
 *   log 0 = -inf. T = 0 gives log P = 0 and an empty path. Ties in the Viterbi
 *   predecessor, final state and model argmax resolve to the smallest index.
 *   An impossible sequence gives -inf and contributes no counts.
 *
 * Return value of the batch functions: 0, or ORC_ERR_SYMBOL if some symbol was
 * out of range (that sequence's outputs are NaN), or ORC_ERR_ARG.
 */
#ifndef HMM_ORACLE_H
#define HMM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_SYMBOL (-5)

int orc_forward(int K, int N, int M, const double* pi, const double* A, const double* B,
                const int32_t* symbols, const int64_t* offsets, const int32_t* lengths,
                int S, const int32_t* model_of_seq, double* loglik, int32_t* argmax,
                int nthreads);

/* score: [S][K] or [S]. best_model: [S] (argmax_k score, or model_of_seq[s]).
 * path: written at symbols' positions for best_model[s] (may be NULL).
 * margin: [S] log P(best path) - log P(second-best path) of the decoded pair
 * (may be NULL; +inf when only one path has non-zero probability). */
int orc_viterbi(int K, int N, int M, const double* pi, const double* A, const double* B,
                const int32_t* symbols, const int64_t* offsets, const int32_t* lengths,
                int S, const int32_t* model_of_seq, double* score, int32_t* best_model,
                int32_t* path, double* margin, int nthreads);

/* weight: [S] (labelled) or [S][K] (all models), NULL = 1.
 * loglik: [S] or [S][K]. Counts are overwritten: cnt_pi[K][N], cnt_A[K][N][N],
 * cnt_B[K][N][M]. */
int orc_forward_backward(int K, int N, int M, const double* pi, const double* A,
                         const double* B, const int32_t* symbols, const int64_t* offsets,
                         const int32_t* lengths, int S, const int32_t* model_of_seq,
                         const double* weight, double* loglik, double* cnt_pi,
                         double* cnt_A, double* cnt_B, int nthreads);

/* Gradient of sum_s w_s log P with respect to the row logits of pi, A, B when
 * each row is the softmax of its logits: g = C - p * rowsum(C). */
void orc_softmax_grad(int K, int N, int M, const double* pi, const double* A,
                      const double* B, const double* cnt_pi, const double* cnt_A,
                      const double* cnt_B, double* g_pi, double* g_A, double* g_B);

/* Baum-Welch re-estimation from counts. A row with zero total count keeps the
 * row given in pi/A/B. */
void orc_mstep(int K, int N, int M, const double* pi, const double* A, const double* B,
               const double* cnt_pi, const double* cnt_A, const double* cnt_B,
               double* pi_out, double* A_out, double* B_out);

#ifdef __cplusplus
}
#endif
#endif
