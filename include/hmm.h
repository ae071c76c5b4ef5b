/*
 * hmm.h -- C-ABI of the GB300 (sm_103a) discrete-HMM recognition hot path.
 *
 * The paper (arXiv 1310.3322, Sec. 2.7) builds its activity-recognition stage
 * on three GPU kernels -- Forward, Viterbi and Baum-Welch -- over discrete
 * HMMs, one HMM per activity, all run in parallel with the recognised activity
 * the best-scoring model (Sec. 3, item 3; Sec. 4.1 lists the stage's
 * parameters: number of hidden states, symbols, actions). The paper prints no
 * equations; the operations below follow the textbook recursions (Rabiner,
 * Proc. IEEE 77(2), 1989).
 *
 * Conventions shared by every entry point
 *   - Models: K discrete HMMs with N states and M symbols.
 *       pi [K][N]     initial-state probabilities
 *       A  [K][N][N]  a_ij = P(q_{t+1} = j | q_t = i), row-major, row = from-state
 *       B  [K][N][M]  b_j(m) = P(o_t = m | q_t = j), row-major
 *     FP32, non-negative and finite (rows are not required to sum to 1).
 *   - Sequences (hmm_seqs_t): sequence s is symbols[offsets[s] ..
 *     offsets[s] + lengths[s]), symbols 0-based in [0, M). If model_of_seq is
 *     NULL every sequence is scored against all K models and per-pair outputs
 *     are [S][K] (row-major, s-major); otherwise sequence s is scored against
 *     model_of_seq[s] only and per-pair outputs are [S].
 *   - Unless stated otherwise, every pointer argument is a DEVICE pointer,
 *     owned by the caller, at least 4-byte aligned (8 for int64), and must stay
 *     valid until the work on `stream` completes.
 *   - The library never allocates device memory: each call that needs scratch
 *     space takes a caller-owned device workspace of at least
 *     hmm_workspace_size() bytes (256-byte aligned). Calls that share a
 *     workspace must be ordered on one stream.
 *   - Every call is asynchronous on `stream` (NULL = legacy default stream),
 *     launches only kernels and memsets (no host synchronisation), and can be
 *     captured into a CUDA graph.
 *   - Return value: HMM_OK, or a negative HMM_ERR_* code found by host-side
 *     checks before anything is launched (nothing is enqueued then), or
 *     HMM_ERR_CUDA if a launch failed. hmm_last_error() describes the last
 *     failure of the calling thread.
 *   - Problems found on the device (a symbol out of range, a negative or
 *     non-finite parameter, an inconsistent offset/length/model index) never
 *     trap: the device status word in the workspace gets a HMM_STATUS_* bit,
 *     the affected outputs are NaN (paths -1), and hmm_get_device_status()
 *     reads the word.
 *   - Log-likelihoods and scores are natural logarithms (nats). An impossible
 *     sequence gives -inf (path filled with 0). T = 0 gives 0 (empty path).
 *     Ties in a Viterbi predecessor, the final state or a model argmax take the
 *     smallest index.
 */
#ifndef HMMGB_HMM_H
#define HMMGB_HMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* hmm_stream_t;

/* Return codes. */
#define HMM_OK 0
#define HMM_ERR_ARG (-1)          /* bad pointer, size, alignment or dimension */
#define HMM_ERR_CUDA (-2)         /* a CUDA runtime call or launch failed */
#define HMM_ERR_WORKSPACE (-3)    /* workspace NULL, misaligned or too small */
#define HMM_ERR_UNSUPPORTED (-4)  /* valid request this build does not implement */
#define HMM_ERR_DEVICE (-5)       /* hmm_get_device_status: a status bit is set */

/* Device status bits (hmm_get_device_status). */
#define HMM_STATUS_SYMBOL 0x1     /* a symbol outside [0, M) */
#define HMM_STATUS_PARAM 0x2      /* a negative, NaN or infinite parameter */
#define HMM_STATUS_SEQ 0x4        /* offset/length out of range, bad model index,
                                     or sum of lengths above total_obs (Viterbi) */
#define HMM_STATUS_TIMEOUT 0x8    /* a bounded device-side wait gave up (the
                                     tensor-core kernels); outputs are invalid */

typedef enum {
  HMM_FP32 = 0,      /* FP32 SIMT recursion (exact power-of-two rescaling) */
  HMM_BF16_MMA = 1,  /* tensor-core alpha*A, BF16 operands (A and B rounded to BF16),
                        FP32 accumulation */
  HMM_TF32_MMA = 2,  /* tensor-core alpha*A, TF32 operands, FP32 accumulation */
  HMM_AUTO = 3       /* the library's choice for the given N */
} hmm_precision_t;

typedef enum {
  HMM_OP_FORWARD = 0,
  HMM_OP_VITERBI = 1,
  HMM_OP_FORWARD_BACKWARD = 2,
  HMM_OP_FORWARD_SCAN = 3  /* hmm_forward_scan with the automatic chunk length */
} hmm_op_t;

typedef struct {
  int32_t K; /* number of models (activities), >= 1 */
  int32_t N; /* states per model, 1 .. hmm_max_states(op) */
  int32_t M; /* symbols, >= 1 */
} hmm_dims_t;

typedef struct {
  const int32_t* symbols;      /* device [total_obs] */
  const int64_t* offsets;      /* device [S], start of each sequence in symbols */
  const int32_t* lengths;      /* device [S], T_s >= 0 */
  const int32_t* model_of_seq; /* device [S] in [0, K), or NULL = all models */
  int32_t S;                   /* host: number of sequences, >= 0 */
  int32_t max_len;             /* host: upper bound on every lengths[s]; sizes
                                  the adjoint's checkpoint buffers */
  int64_t total_obs;           /* host: number of elements of symbols */
  /* Model sets (one HMM set per role, Sec. 5.7), used when model_of_seq is
   * NULL and model_base is not: sequence s is scored against models
   * [model_base[s], model_base[s] + model_span) only, and every per-model
   * output ([S][K] above) becomes [S][model_span] with indices relative to
   * the set. FP32 forward and Viterbi only; zero-initialised fields (NULL, 0)
   * mean "every model". */
  const int32_t* model_base;   /* device [S], model_base[s] + model_span <= K */
  int32_t model_span;          /* host: models per set, 1 .. K */
} hmm_seqs_t;

/* Workspace bytes that `op` needs for these dimensions and sequences (host
 * only; reads only the host fields of *seqs). */
int hmm_workspace_size(hmm_dims_t dims, const hmm_seqs_t* seqs, hmm_op_t op, size_t* bytes);

/* Largest N that `op` accepts at `precision` in this build. */
int hmm_max_states(hmm_op_t op, hmm_precision_t precision);

/* Forward algorithm (Sec. 2.7 "Forward"; Rabiner eqs. 19-21 with per-step
 * rescaling, Sec. V-A): loglik = log P(O_s | lambda_k) for every scored pair.
 *   loglik  [S][K] (model_of_seq NULL) or [S]
 *   argmax  [S] or NULL: recognised activity = argmax_k loglik[s][k] (Sec. 3
 *           item 3), smallest k on ties, -1 if any of the row is NaN. Only
 *           written when model_of_seq is NULL.
 * HMM_FP32 (N <= 64): the alpha recursion runs in FP32 with exact
 * power-of-two rescaling every step; the exponent sum is an integer and the
 * final log is taken in FP64. HMM_BF16_MMA (32 < N <= 512) / HMM_TF32_MMA
 * (32 < N <= 128), every sequence against every model: alpha*A on the tensor
 * cores with BF16 (u = 2^-8) or TF32 (u = 2^-11, round to nearest) operands
 * and FP32 accumulation, |delta log P| <= 2 u T (TF32) or 3 u T (BF16) against
 * FP64. The BF16 path
 * computes with the model's A and B both rounded to BF16 (round to nearest
 * even, once per call); the TF32 path rounds A only. Above 128
 * states (the cited cuHMM kernel's 512-state workload, Sec. 5.6) each
 * 128-sequence tile runs on a thread-block cluster of N_pad / 64 CTAs, each
 * holding its 64-column slices of A and of the emission table resident, the
 * rows exchanged through distributed shared memory every step; where the
 * emission slice does not fit (N_pad = 512 with M > 173) one CTA per tile
 * streams A^T from a BF16 image the call builds in the workspace. HMM_AUTO: tensor cores (BF16) above N = 64; for
 * N <= 32 and a batch of few long sequences (max_len >= 4096, pairs * N_pad^3
 * <= 2^21) the parallel-in-time forward of hmm_forward_scan, when the
 * workspace holds its chunk products (hmm_workspace_size(HMM_OP_FORWARD)
 * counts them for such batches); FP32 SIMT otherwise. */
int hmm_forward(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                const hmm_seqs_t* seqs, hmm_precision_t precision, float* loglik,
                int32_t* argmax, void* workspace, size_t workspace_bytes, hmm_stream_t stream);

/* hmm_forward for callers that cannot provide a device workspace. (The paper
 * has no counterpart; this is an integration convenience of this library.)
 *
 * Some callers cannot allocate device memory when they score: real-time or
 * embedded hosts that forbid cudaMalloc after start-up, plug-in hosts that
 * own every device allocation, code that must never touch an allocator on its
 * recognition path. This call takes its scratch from a fixed array compiled
 * into the library (HMM_STATIC_SCRATCH_BYTES in the device memory of every GPU
 * that loads the library, held until the process exits) and is otherwise
 * hmm_forward: same arguments except the workspace, same outputs, same device
 * status bits. It allocates nothing and calls no allocating routine.
 *   - What must fit is the scratch of the sequential recursion: the value of
 *     hmm_workspace_size(HMM_OP_FORWARD) for every batch except the few-long-
 *     sequence batches that HMM_AUTO sends to the parallel-in-time forward,
 *     for which that query also counts the chunk products (this call takes
 *     that variant only when the products fit too, else the sequential
 *     recursion). Larger requests return HMM_ERR_WORKSPACE and enqueue
 *     nothing; about 8 MiB covers e.g. 65536 sequences with K=10, N=32, M=256.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current) and keeps it for the life of the
 *     process; make that first call before any stream capture on the device.
 *     A device reset (cudaDeviceReset) invalidates the kept address: do not
 *     call this entry point on a device after resetting it.
 *   - Every call on a device shares the one array, and the next call
 *     overwrites what the last one left there: calls that may overlap on the
 *     GPU (different streams, or threads without ordering) race and give wrong
 *     results. Serialise them on one stream.
 *   - The device status word lives in the shared array and is not readable
 *     through hmm_get_device_status; bad inputs still give NaN outputs. */
#define HMM_STATIC_SCRATCH_BYTES (8 * 1024 * 1024)
int hmm_forward_static(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                       const hmm_seqs_t* seqs, hmm_precision_t precision, float* loglik,
                       int32_t* argmax, hmm_stream_t stream);

/* Parallel-in-time forward for few, very long sequences (not in the paper:
 * an associative-scan reformulation of the same Forward, Sec. 2.7 / Rabiner
 * eqs. 19-21). alpha_{T-1} = alpha_0 M_1 ... M_{T-1} with the step matrices
 * M_t = A diag(b(o_t)); the steps 1 .. T-1 of every sequence are cut into
 * chunks of `chunk` steps whose products are computed independently (row i
 * of a chunk product is the recursion started from state i, each row with its
 * own power-of-two exponent), then every pair combines its chunks in order.
 * Outputs, argmax, model_of_seq / model sets and the device status bits are
 * those of hmm_forward with HMM_FP32 (N <= 32 here); only the rounding order
 * differs. It does N times the arithmetic of hmm_forward, in exchange for a
 * dependency chain of chunk + T / chunk steps instead of T: worth it when a
 * batch has too few (sequence, model) pairs to fill the GPU.
 *   chunk  steps per chunk, 1 .. 65536, or 0 = ceil(sqrt(2 max_len)) rounded
 *          up to a multiple of 16 (the chain-length balance point).
 * The workspace holds N_pad^2 + N_pad floats per (chunk, model) pair:
 * hmm_forward_scan_workspace_size() (host only) gives the bytes for a chunk
 * length; hmm_workspace_size(HMM_OP_FORWARD_SCAN) those of the automatic one.
 * A batch whose chunks exceed that storage (overlapping sequences whose
 * lengths sum past total_obs) has the excess sequences marked bad
 * (HMM_STATUS_SEQ, NaN). */
int hmm_forward_scan(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                     const hmm_seqs_t* seqs, int32_t chunk, float* loglik, int32_t* argmax,
                     void* workspace, size_t workspace_bytes, hmm_stream_t stream);
int hmm_forward_scan_workspace_size(hmm_dims_t dims, const hmm_seqs_t* seqs, int32_t chunk,
                                    size_t* bytes);

/* Viterbi algorithm (Sec. 2.7 "Viterbi"; Rabiner eqs. 32-35):
 *   score       [S][K] or [S]: max_Q log P(O_s, Q | lambda_k)
 *   best_model  [S] or NULL: the decoded model, argmax_k score[s][k] (smallest
 *               k on ties, -1 if a score is NaN), or model_of_seq[s]
 *   path        [total_obs] or NULL: the best state path of the decoded model,
 *               path[offsets[s] + t] = q_t (sequences must not overlap)
 * Requires sum_s lengths[s] <= total_obs (backpointer storage: one byte per
 * padded state and step). FP32 SIMT max-plus for N <= 128 (above 64 states
 * one warp per pair with log A staged in shared memory). */
int hmm_viterbi(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                const hmm_seqs_t* seqs, float* score, int32_t* best_model, int32_t* path,
                void* workspace, size_t workspace_bytes, hmm_stream_t stream);

/* Forward-backward adjoint (Sec. 2.7 "Baum-Welch", its E-step; Rabiner
 * eqs. 24-25, 37-38): weighted expected counts
 *   cnt_pi[k][i]   = sum_s w_s gamma_1(i)
 *   cnt_A[k][i][j] = sum_s w_s sum_{t<T} xi_t(i,j)
 *   cnt_B[k][j][m] = sum_s w_s sum_{t: o_t = m} gamma_t(j)
 * over the pairs scored against model k, which are exactly the gradient of
 * sum_s w_s log P with respect to log pi, log A, log B. Alpha is checkpointed
 * every ceil(sqrt(T)) steps and recomputed segment by segment.
 *   weight  [S] or [S][K] (the layout of loglik), NULL = all 1
 *   loglik  [S] or [S][K]
 *   counts  overwritten; summed in a fixed order (bitwise reproducible).
 * precision: HMM_FP32 runs the FP32 SIMT adjoint (N <= 64); HMM_BF16_MMA the
 * tensor-core adjoint (32 < N <= 128, M <= 256: BF16 operands, A and B
 * rounded to BF16 as in hmm_forward, FP32 accumulation, per-row messages
 * renormalised every step, checkpoint stride
 * capped at 16 while T <= 8192) as two kernels: the forward and the backward
 * recursion of every 128-row tile run as independent chains keeping
 * checkpoints of both, then every range of a tile's checkpoint segments is a
 * separate work item (recompute, backward, counts); HMM_AUTO chooses the
 * tensor cores above N = 32. Its errors against FP64 are of order the BF16 unit roundoff 2^-8
 * relative per count (|delta log P| <= 2^-7 T).
 * Above 128 states (N <= 512, the cited cuHMM shape of Sec. 5.6) the
 * tensor-core forward and backward passes (on clusters, as the forward) keep
 * every step's rescaled alpha and beta rows in the workspace (4 K total_obs
 * N_pad floats), and the counts are formed from them: xi as one fixed-order
 * contraction over all steps on the tensor cores, its two operands rounded
 * to TF32 (relative error <= 2^-11 each, FP32 accumulation). This path
 * scores every sequence against every model (model_of_seq only with K = 1)
 * and needs the cluster forward's emission slice in shared memory (M <= 173
 * at 512 padded states); other requests return HMM_ERR_UNSUPPORTED. The
 * emission and initial counts sum the gamma rows of each symbol (rows sorted
 * by symbol, fixed-size pieces, pieces summed in order). Same error bounds.
 * HMM_TF32_MMA (64 < N <= 128, M <= 256): the forward and the backward
 * recursion of every tile of the same tile plan with TF32 operands (A
 * rounded to TF32, round to nearest; B in FP32; FP32 accumulation), keeping
 * every step's rescaled alpha and beta rows (4 rows x total_obs x 128 floats
 * when labelled, K times that otherwise: size the workspace with
 * hmm_forward_backward_workspace_size), then the counts from the rows as
 * above (xi's operands rounded to TF32). |delta log P| <= 2 u T, u = 2^-11,
 * counts within 2^-8 relative.
 * Impossible or invalid pairs contribute no counts. */
int hmm_forward_backward(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                         const hmm_seqs_t* seqs, const float* weight,
                         hmm_precision_t precision, float* loglik, float* cnt_pi,
                         float* cnt_A, float* cnt_B, void* workspace, size_t workspace_bytes,
                         hmm_stream_t stream);

/* Workspace bytes hmm_forward_backward needs at `precision` (host only; for
 * anything but HMM_TF32_MMA the same as hmm_workspace_size with
 * HMM_OP_FORWARD_BACKWARD). Errors as hmm_workspace_size. */
int hmm_forward_backward_workspace_size(hmm_dims_t dims, const hmm_seqs_t* seqs,
                                        hmm_precision_t precision, size_t* bytes);

/* Row-wise softmax of logits into probabilities (the parameterisation used for
 * learning): pi[k] = softmax(logit_pi[k]), A[k][i] = softmax(logit_A[k][i]),
 * B[k][j] = softmax(logit_B[k][j]). Outputs may not alias inputs. */
int hmm_softmax_rows(hmm_dims_t dims, const float* logit_pi, const float* logit_A,
                     const float* logit_B, float* pi, float* A, float* B, hmm_stream_t stream);

/* Gradient of sum_s w_s log P with respect to the row logits, from the
 * probabilities and the counts of hmm_forward_backward:
 *   g = C - p * rowsum(C)   for every row of pi, A and B.
 * Outputs may alias the counts. */
int hmm_softmax_grad(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                     const float* cnt_pi, const float* cnt_A, const float* cnt_B, float* g_pi,
                     float* g_A, float* g_B, hmm_stream_t stream);

/* Baum-Welch re-estimation, the M-step (Sec. 2.7 "Baum-Welch"; Rabiner
 * eq. 40): from the expected counts of hmm_forward_backward (unit weights),
 *   pi_out[k][i]   = cnt_pi[k][i] / sum_i cnt_pi[k][i]
 *   A_out[k][i][j] = cnt_A[k][i][j] / sum_j cnt_A[k][i][j]
 *   B_out[k][j][m] = cnt_B[k][j][m] / sum_m cnt_B[k][j][m]
 * A row whose counts sum to zero keeps the old row of pi / A / B. Outputs may
 * alias pi, A, B (in-place re-estimation); all pointers are device pointers.
 * Alternating hmm_forward_backward and hmm_mstep never lowers sum_s log P
 * (up to rounding): the paper's learning loop. */
int hmm_mstep(hmm_dims_t dims, const float* pi, const float* A, const float* B,
              const float* cnt_pi, const float* cnt_A, const float* cnt_B, float* pi_out,
              float* A_out, float* B_out, hmm_stream_t stream);

/* One Adam step (Kingma & Ba 2015) on n parameters, in place:
 *   t = *step_counter + 1;  g = grad_scale * grad;
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   param -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
 *   *step_counter = t.
 * step_counter is a DEVICE int32 (steps taken so far, 0 before the first),
 * so a captured CUDA graph advances the bias correction on every replay.
 * Use grad_scale < 0 to ascend a log-likelihood gradient. */
int hmm_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, float grad_scale, int32_t* step_counter,
                  hmm_stream_t stream);

/* Copies the device status word of the last call that used `workspace` into
 * *status (HOST pointer), synchronising `stream`. Returns HMM_OK when the
 * word is 0, HMM_ERR_DEVICE when a bit is set. */
int hmm_get_device_status(const void* workspace, hmm_stream_t stream, int32_t* status);

/* Autotuner hook: lanes of a warp that cooperate on one (sequence, model)
 * pair, per tunable kernel and padded state count n_pad (4, 8, 16, 32, 64).
 * `op` is HMM_OP_FORWARD, HMM_OP_VITERBI (the score kernel),
 * HMM_OP_FORWARD_BACKWARD or HMM_TUNE_VITERBI_PATHS (the path kernel); or
 * HMM_TUNE_FB_RANGES, whose value is the number of ranges the segments of one
 * pair are split into by the FP32 SIMT adjoint (1, the default: forward,
 * recompute and backward in one kernel; more: forward and backward recursions
 * as independent chains keeping checkpoints of both, then each range of
 * segments a separate work item with its own count slot -- shorter chains,
 * for batches of few long sequences that leave the GPU idle; the workspace
 * grows with the value). The value must be
 * one this build instantiates (hmm_tuning_candidates, whose first entry is
 * the default); 0 restores the default. Process-wide; not thread-safe against
 * concurrent launches. The choice changes only the speed and the rounding
 * order of the counts: every candidate computes the same recursion. */
#define HMM_TUNE_VITERBI_PATHS 3
#define HMM_TUNE_FB_RANGES 4
int hmm_set_tuning(int32_t op, int32_t n_pad, int32_t lanes_per_pair);
int hmm_get_tuning(int32_t op, int32_t n_pad, int32_t* lanes_per_pair);
/* Writes up to cap candidate lane counts for (op, n_pad) into out (HOST
 * pointer); returns how many there are, or a negative error code. */
int hmm_tuning_candidates(int32_t op, int32_t n_pad, int32_t* out, int32_t cap);

/* Failure detection of the tensor-core kernels (HMM_BF16_MMA / HMM_TF32_MMA
 * forward and adjoint). Their threads hand each time step to one another
 * through shared-memory mbarriers; every such wait polls at most `polls`
 * times and then gives up: the kernel sets HMM_STATUS_TIMEOUT in the
 * workspace's status word, first waits (with the default limit) for the
 * matrix products and copies it has already started, frees its tensor memory
 * and returns; the outputs of that call are invalid (log-likelihoods of the
 * rows it gave up on are NaN). No wait ever traps or spins forever.
 *   polls < 0  the default, 2^24 polls (seconds: far beyond any healthy step)
 *   polls = 0  no poll at all: every such wait gives up at once -- the way the
 *              give-up path is tested
 *   polls > 0  that many polls (the first never suspends the thread; the
 *              others may, for a hardware-defined time), capped at 2^32 - 1
 * Process-wide, read when a call launches its kernels (a captured graph keeps
 * the value of its capture); returns HMM_OK. hmm_get_wait_limit returns the
 * limit in force. */
int hmm_set_wait_limit(int64_t polls);
uint32_t hmm_get_wait_limit(void);

/* FP32 FMA throughput probe: the measured denominator of the roofline of the
 * FP32 (SIMT) kernels, which are bound by FP32 issue (not part of the
 * paper's method). blocks x threads threads (threads a multiple of 32, at
 * most 1024) each run `iters` rounds of 16 independent FMA chains: mode 0
 * scalar fma.rn.f32 (blocks*threads*iters*32 flop per launch), mode 1 the
 * packed two-lane fma.rn.f32x2 (twice that). out [blocks] (device) receives
 * per-block sums of the chains. The caller times the launch; returns
 * HMM_ERR_ARG for bad arguments. */
int hmm_fma_probe(int32_t blocks, int32_t threads, int64_t iters, int32_t mode, float* out,
                  hmm_stream_t stream);

/* Kernel timing (host-side tracing). While enabled, every kernel launch of
 * the library is bracketed by two CUDA events recorded on the launch stream;
 * hmm_timing_read() synchronises those events and reports, per kernel kind,
 * the number of launches and their summed duration since the last reset.
 * Kinds: 0 setup, 1 forward, 2 viterbi-scores, 3 viterbi-paths, 4 adjoint
 * (for the two-kernel adjoints, the tensor-core one and the FP32 one with
 * segment ranges: their segment-range kernel), 5 count-reduce,
 * 6 softmax-rows, 7 softmax-grad, 8 adam, 9 mstep, 10 scan-chunks,
 * 11 scan-combine, 12 adjoint-pass (the two-kernel adjoints' forward and
 * backward passes). Not for use inside CUDA-graph capture; not thread-safe
 * against concurrent launches. */
#define HMM_TIMING_KINDS 13
int hmm_timing_enable(int on);
int hmm_timing_reset(void);
int hmm_timing_read(int32_t kind, int64_t* launches, double* total_ms);

/* Thread-local description of the last error of this thread ("" if none). */
const char* hmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HMMGB_HMM_H */
