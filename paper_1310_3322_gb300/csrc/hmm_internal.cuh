// hmm_internal.cuh -- shared internals of the sm_103a HMM library: workspace
// layout, kernel argument blocks, and the small device helpers every kernel
// uses (group reductions, packed FP32x2 arithmetic, exact power-of-two
// rescaling, the length bucketing of the scheduler).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hmm.h"

namespace hmmgb {

constexpr int kWarpsPerBlock = 4;      // SIMT kernels: 128-thread blocks
constexpr int kPlanThreads = 1024;     // setup kernel block size
constexpr int kLenBuckets = 1024;      // scheduler length buckets
constexpr int kReduceChunk = 32;       // sequences per first-level count reduction
constexpr int kReduceTile = 256;       // count entries per reduction block
constexpr float kViterbiQuant = 32768.f;  // Viterbi offsets are multiples of 2^-15

// ---------------------------------------------------------------------------
// workspace layout (all offsets 256-byte aligned)
// ---------------------------------------------------------------------------
struct WsHeader {
  int32_t status;      // HMM_STATUS_* bits
  int32_t queue[7];    // persistent-kernel work counters
  int32_t pad[56];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

struct WsLayout {
  size_t order, seqlen, done, bpoff, best, pip, Ap, Btp, bp, partial, red1, total;
  size_t Btp16;          // the emission table as BF16 bits (the BF16 path)
  size_t phist, punits;  // setup plan over many blocks
  size_t vgorder, vgcount;  // Viterbi paths above 64 states: grouping by model
  int NP;
  int64_t bp_cap;      // bytes of backpointer storage
  int64_t slots;       // adjoint partial slots
  int64_t slot_floats; // floats per slot (NP + NP*NP + NP*M)
  int nchunks;         // first-level reduction chunks
  // tensor-core adjoint
  size_t m_sorted, m_tmp, m_keys, m_tiles, m_ntiles, m_ckpt, m_scr, m_gexp, m_gbuf, m_pscr;
  size_t wimg;         // tensor-core forward above 128 states: BF16 A^T images
  size_t sc_coff, sc_P, sc_E;  // parallel-in-time forward: chunk offsets, products
  size_t w_X, w_Bh, w_V, w_G, w_xe, w_sym, w_Cp;  // adjoint above 128 states
  size_t w_ecb, w_eh, w_eb, w_epb, w_el, w_ep;      // its emission-count sort and pieces
  size_t t_pos, t_mrow, t_rpos;                                       // TF32 adjoint: row offsets
  int w_nsplit, w_ncc;
  int64_t w_ech;
  int64_t w_rtot;
  int64_t sc_cap;              // chunk slots per model slot
  size_t s_ckA, s_ckB, s_ckE, s_sig, s_skip;  // SIMT adjoint with segment ranges
  int s_planes;        // largest number of ranges per pair the workspace holds
  int64_t m_ckpt_bytes, m_scr_bytes, m_gexp_bytes;
  int m_grid;
  // the tensor-core adjoint's two kernels: work lists, per-tile Y checkpoints
  // and last-step row sums
  size_t m_pass, m_ptmp, m_npass, m_rtile, m_rseg, m_rmodel, m_rlen, m_nrng, m_cky, m_slast;
  size_t m_psum;
  int m_pass_cap, m_rng_cap, m_spr, m_group;
};

// ---------------------------------------------------------------------------
// kernel argument blocks
// ---------------------------------------------------------------------------
struct SeqArgs {
  const int32_t* symbols;
  const int64_t* offsets;
  const int32_t* model_of_seq;  // NULL = all models
  const int32_t* model_base;    // all-models mode with model sets: first model of s's set
  int span;                     // models scored per sequence in all-models mode (K or the set size)
  const int32_t* seqlen;        // validated lengths (-1 = invalid pair)
  const int32_t* order;         // sequences sorted by decreasing length
  int S;
  int K;
  int M;
  int N;                        // states (the padded count is the kernel's NP)
};

struct ModelArgs {
  const float* pip;   // [K][NP]
  const float* Ap;    // [K][NP][NP]
  const float* Btp;   // [K][M][NP]  (emission table transposed: symbol-major)
  const uint16_t* Btp16;  // [K][M][NP]  the same as BF16 bits (BF16 path only)
};

struct SetupArgs {
  int K, N, M, NP, S;
  int64_t total_obs;
  int max_len;         // sequences longer than this are rejected
  int log_mode;        // 1: tables hold natural logs (Viterbi), 0: probabilities
  int bf16_b;          // 1: the emission table holds B rounded to BF16 (the BF16 path)
  int want_bpoff;      // 1: compute backpointer offsets (Viterbi)
  int skip_order;      // 1: validate only (the caller builds its own schedule)
  int ndone;           // entries of `done` to clear
  const float* pi;
  const float* A;
  const float* B;
  const int32_t* lengths;
  const int64_t* offsets;
  const int32_t* model_of_seq;
  const int32_t* model_base;  // model sets: model_base[s] + span <= K
  int span;
  float* pip;
  float* Ap;
  float* Btp;
  uint16_t* Btp16;     // bf16_b: Btp's values as BF16 bits
  int32_t* seqlen;
  int32_t* order;
  int32_t* done;
  int64_t* bpoff;
  int64_t bp_cap_rows;   // rows of NP bytes available for backpointers
  int32_t* phist;        // S > 4096: per-plan-block length-bucket counts [nb][1024]
  int64_t* punits;       // S > 4096: per-plan-block prefix units [2][nb]
  int scan_chunk;        // > 0: chunk offsets of the parallel-in-time forward
  int64_t* coff;         // [S + 1] exclusive prefix of ceil((T_s - 1) / scan_chunk)
  int64_t coff_cap;      // chunk slots available (sequences past it are rejected)
  int32_t* status;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#define HMM_FULL_MASK 0xffffffffu

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(HMM_FULL_MASK, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(HMM_FULL_MASK, v, o));
  return v;
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Three-input FP32 maximum (sm_100+ PTX form).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// 2^k as a float, for k in [-126, 127].
__device__ __forceinline__ float exp2i(int k) { return __int_as_float((k + 127) << 23); }

// For finite s > 0 returns e with s * 2^-e in [1, 2). When s is below 2^-120
// the caller first multiplies by 2^64 (see rescale_pow2).
__device__ __forceinline__ int frexp2(float s) { return ((__float_as_int(s) >> 23) & 0xff) - 127; }

// Length bucket of the scheduler: exact below 256, then 32 buckets per octave.
__device__ __forceinline__ int length_bucket(int T) {
  if (T < 256) return T < 0 ? 0 : T;
  const int e = 31 - __clz(T);
  int b = 256 + (e - 8) * 32 + ((T >> (e - 5)) & 31);
  return b < kLenBuckets ? b : kLenBuckets - 1;
}

__device__ __forceinline__ void set_status(int32_t* status, int bits) { atomicOr(status, bits); }

// Vector loads/stores of J consecutive floats (J in {1,2,4,8}), 4*J-byte aligned.
template <int J>
__device__ __forceinline__ void load_vec(float (&d)[J], const float* p) {
  if constexpr (J == 1) {
    d[0] = __ldg(p);
  } else if constexpr (J == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    d[0] = v.x; d[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < J / 4; ++q) {
      float4 v = __ldg(reinterpret_cast<const float4*>(p) + q);
      d[4 * q] = v.x; d[4 * q + 1] = v.y; d[4 * q + 2] = v.z; d[4 * q + 3] = v.w;
    }
  }
}

template <int J>
__device__ __forceinline__ void store_vec(float* p, const float (&s)[J]) {
  if constexpr (J == 1) {
    p[0] = s[0];
  } else if constexpr (J == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(s[0], s[1]);
  } else {
#pragma unroll
    for (int q = 0; q < J / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(s[4 * q], s[4 * q + 1], s[4 * q + 2], s[4 * q + 3]);
  }
}

template <int J>
__device__ __forceinline__ void load_vec_smem(float (&d)[J], const float* p) {
  if constexpr (J == 1) {
    d[0] = p[0];
  } else if constexpr (J == 2) {
    float2 v = *reinterpret_cast<const float2*>(p);
    d[0] = v.x; d[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < J / 4; ++q) {
      float4 v = reinterpret_cast<const float4*>(p)[q];
      d[4 * q] = v.x; d[4 * q + 1] = v.y; d[4 * q + 2] = v.z; d[4 * q + 3] = v.w;
    }
  }
}

// Sum of J registers as a balanced tree (short dependency chain).
template <int J>
__device__ __forceinline__ float tree_sum(const float (&x)[J]) {
  if constexpr (J == 1) {
    return x[0];
  } else {
    float t[J / 2];
#pragma unroll
    for (int i = 0; i < J / 2; ++i) t[i] = x[2 * i] + x[2 * i + 1];
    return tree_sum<J / 2>(t);
  }
}

template <int J>
__device__ __forceinline__ float tree_max(const float (&x)[J]) {
  if constexpr (J == 1) {
    return x[0];
  } else {
    float t[J / 2];
#pragma unroll
    for (int i = 0; i < J / 2; ++i) t[i] = fmaxf(x[2 * i], x[2 * i + 1]);
    return tree_max<J / 2>(t);
  }
}

// out[jj] = sum_i x_i a_{i, j0+jj}: x is the per-pair shared-memory row (NP
// floats, 16-byte aligned), a2[i2][jj] = (a_{2 i2, j}, a_{2 i2 + 1, j}) the
// register-resident column slice. Packed FP32x2 FMAs over pairs of rows; NS
// independent accumulator sets keep at least four FMA chains in flight.
// NV < NP (states NV .. NP-1 are padding: x and a are exactly 0 there) skips
// the padded row pairs and, when one lane owns every column (J == NP), the
// padded columns: the skipped terms are exact zeros, so the sums are bitwise
// those of the full product.
template <int NP, int J, int NV = NP>
__device__ __forceinline__ void matvec_cols(const float* xb, const float2 (&a2)[NP / 2][J],
                                            float (&out)[J]) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  constexpr int JC = (J == NP) ? NV : J;  // columns computed
  float2 acc[NS][J];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[s][jj] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    if (4 * q >= NV) continue;
    const float4 xv = *reinterpret_cast<const float4*>(xb + 4 * q);
    const float2 lo = make_float2(xv.x, xv.y), hi = make_float2(xv.z, xv.w);
    const int s = q % NS;
#pragma unroll
    for (int jj = 0; jj < JC; ++jj) acc[s][jj] = __ffma2_rn(lo, a2[2 * q][jj], acc[s][jj]);
    if (4 * q + 2 < NV) {
#pragma unroll
      for (int jj = 0; jj < JC; ++jj) acc[s][jj] = __ffma2_rn(hi, a2[2 * q + 1][jj], acc[s][jj]);
    }
  }
#pragma unroll
  for (int jj = 0; jj < J; ++jj) {
    float2 t = acc[0][jj];
#pragma unroll
    for (int s = 1; s < NS; ++s) t = __fadd2_rn(t, acc[s][jj]);
    out[jj] = t.x + t.y;
  }
}

// out[jj] = max_i (x_i + la_{i, j0+jj}) (max-plus product; exact, so the
// grouping into NS partial maxima does not change the result). NV as in
// matvec_cols (padded entries are -inf and never win).
template <int NP, int J, int NV = NP>
__device__ __forceinline__ void maxplus_cols(const float* xb, const float2 (&a2)[NP / 2][J],
                                             float (&out)[J]) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  constexpr int JC = (J == NP) ? NV : J;
  float m[NS][J];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int jj = 0; jj < J; ++jj) m[s][jj] = -INFINITY;
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    if (4 * q >= NV) continue;
    const float4 xv = *reinterpret_cast<const float4*>(xb + 4 * q);
    const float2 lo = make_float2(xv.x, xv.y), hi = make_float2(xv.z, xv.w);
    const int s = q % NS;
#pragma unroll
    for (int jj = 0; jj < JC; ++jj) {
      const float2 v = __fadd2_rn(lo, a2[2 * q][jj]);
      m[s][jj] = fmax3(m[s][jj], v.x, v.y);
    }
    if (4 * q + 2 < NV) {
#pragma unroll
      for (int jj = 0; jj < JC; ++jj) {
        const float2 w = __fadd2_rn(hi, a2[2 * q + 1][jj]);
        m[s][jj] = fmax3(m[s][jj], w.x, w.y);
      }
    }
  }
#pragma unroll
  for (int jj = 0; jj < J; ++jj) {
    float t = m[0][jj];
#pragma unroll
    for (int s = 1; s < NS; ++s) t = fmaxf(t, m[s][jj]);
    out[jj] = t;
  }
}

// As maxplus_cols, also returning the smallest maximising i per column.
template <int NP, int J>
__device__ __forceinline__ void maxarg_cols(const float* xb, const float2 (&a2)[NP / 2][J],
                                            float (&out)[J], int (&arg)[J]) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  float m[NS][J];
  int a[NS][J];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int jj = 0; jj < J; ++jj) { m[s][jj] = -INFINITY; a[s][jj] = 0; }
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 xv = *reinterpret_cast<const float4*>(xb + 4 * q);
    const float2 lo = make_float2(xv.x, xv.y), hi = make_float2(xv.z, xv.w);
    const int s = q % NS;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
      const float2 v = __fadd2_rn(lo, a2[2 * q][jj]);
      if (v.x > m[s][jj]) { m[s][jj] = v.x; a[s][jj] = 4 * q; }
      if (v.y > m[s][jj]) { m[s][jj] = v.y; a[s][jj] = 4 * q + 1; }
    }
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
      const float2 w = __fadd2_rn(hi, a2[2 * q + 1][jj]);
      if (w.x > m[s][jj]) { m[s][jj] = w.x; a[s][jj] = 4 * q + 2; }
      if (w.y > m[s][jj]) { m[s][jj] = w.y; a[s][jj] = 4 * q + 3; }
    }
  }
#pragma unroll
  for (int jj = 0; jj < J; ++jj) {
    float t = m[0][jj];
    int ta = a[0][jj];
#pragma unroll
    for (int s = 1; s < NS; ++s)
      if (m[s][jj] > t || (m[s][jj] == t && a[s][jj] < ta)) { t = m[s][jj]; ta = a[s][jj]; }
    out[jj] = t;
    arg[jj] = ta;
  }
}

// Exact power-of-two rescaling of a group-distributed vector so that its sum
// lies in [1, 2). `gsum` is the group-wide sum (> 0, finite); returns the
// base-2 exponent removed (the caller adds it to its running total).
template <int J>
__device__ __forceinline__ int rescale_pow2(float (&x)[J], float gsum) {
  int shift = 0;
  if (gsum < 0x1p-120f) {  // keep the factor representable
#pragma unroll
    for (int jj = 0; jj < J; ++jj) x[jj] *= 0x1p64f;
    gsum *= 0x1p64f;
    shift = -64;
  } else if (gsum >= 0x1p120f) {
#pragma unroll
    for (int jj = 0; jj < J; ++jj) x[jj] *= 0x1p-64f;
    gsum *= 0x1p-64f;
    shift = 64;
  }
  const int e = frexp2(gsum);
  const float f = exp2i(-e);
#pragma unroll
  for (int jj = 0; jj < J; ++jj) x[jj] *= f;
  return e + shift;
}

// ---------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
cudaError_t launch_setup(const SetupArgs& a, cudaStream_t st);
cudaError_t launch_softmax_rows(int K, int N, int M, const float* lpi, const float* lA,
                                const float* lB, float* pi, float* A, float* B, cudaStream_t st);
cudaError_t launch_softmax_grad(int K, int N, int M, const float* pi, const float* A,
                                const float* B, const float* cpi, const float* cA,
                                const float* cB, float* gpi, float* gA, float* gB,
                                cudaStream_t st);
cudaError_t launch_mstep(int K, int N, int M, const float* pi, const float* A, const float* B,
                         const float* cpi, const float* cA, const float* cB, float* opi,
                         float* oA, float* oB, cudaStream_t st);
cudaError_t launch_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr,
                        float b1, float b2, float eps, float gs, int32_t* step, cudaStream_t st);

struct FwdLaunch {
  SeqArgs seq;
  ModelArgs mod;
  float* loglik;
  int32_t* argmax;
  int32_t* done;
  int32_t* queue;
  int32_t* status;
  int n_items;
};
cudaError_t launch_forward(int NP, int G, const FwdLaunch& a, cudaStream_t st);

struct VitLaunch {
  SeqArgs seq;
  ModelArgs mod;     // log tables
  float* score;
  int32_t* best;     // decoded model per sequence (workspace or caller's)
  int32_t* path;
  int32_t* done;
  int32_t* queue;    // two counters: [0] scores, [1] paths
  int32_t* status;
  const int64_t* bpoff;
  uint8_t* bp;
  int n_items_score;
  int n_items_path;
  int32_t* gorder;   // above 64 states: sequences grouped by decoded model (or NULL)
  int32_t* gcount;   // above 64 states: items of gorder
};
cudaError_t launch_viterbi_scores(int NP, int G, const VitLaunch& a, cudaStream_t st);
cudaError_t launch_viterbi_paths(int NP, int G, const VitLaunch& a, cudaStream_t st);
// 64 < N <= 128 (viterbi_wide.cu): one warp per pair, log A in shared memory
cudaError_t launch_viterbi_scores_wide(const VitLaunch& a, cudaStream_t st);
cudaError_t launch_viterbi_paths_wide(const VitLaunch& a, cudaStream_t st);

struct FbLaunch {
  SeqArgs seq;
  ModelArgs mod;
  const float* weight;
  float* loglik;
  float* partial;
  int64_t slot_floats;
  int32_t* queue;
  int32_t* status;
  int n_items;
  int ckpt;          // checkpoint stride C
  int nck;           // checkpoints per pair (ceil(max_len / C))
};
cudaError_t launch_fb(int NP, int G, const FbLaunch& a, cudaStream_t st);
size_t fb_smem_bytes(int NP, int G, int C, int NC, int M, int warps);

// FP32 SIMT adjoint with segment-parallel counts (fb_seg.cu): a pass kernel
// (forward and backward recursions as independent chains, checkpoints of
// both) and a segment kernel (one work item per range of segments of a pair).
struct FbSegLaunch {
  SeqArgs seq;
  ModelArgs mod;
  const float* weight;
  float* loglik;
  float* partial;      // [spar][npairs][slot_floats]
  int64_t slot_floats;
  float* ckA;          // [npairs][nck][NP] alpha at t = c C (power-of-two scaled)
  float* ckB;          // [npairs][nck][NP] beta at t = c C (power-of-two scaled)
  int32_t* ckE;        // [npairs][nck] exponent removed from alpha at t = c C
  float* sig;          // [npairs] sum of alpha_{T-1}
  int32_t* skip;       // [npairs] 1: no counts (empty, impossible or invalid, zero weight)
  int32_t* queue;      // [2] work counters of the two kernels
  int32_t* status;
  int npairs;          // S (labelled) or S * K
  int n_items_pass;    // 2 * pair-group items (forward and backward)
  int n_items_seg;     // pair-group items * spar
  int ckpt, nck;       // segment length C, segments of the longest sequence
  int spar, spg;       // ranges per pair, segments per range
};
// phase 0: the forward and backward passes; phase 1: the segment ranges
cudaError_t launch_fb_seg(int NP, int G, const FbSegLaunch& a, int phase, cudaStream_t st);

// Parallel-in-time forward (scan.cu): per-chunk products of the step
// matrices A diag(b(o_t)), then one ordered combine per pair.
constexpr int kScanDead = -(1 << 30);      // row exponent: the row is all zero
constexpr int kScanBad = -(1 << 30) - 1;   // row exponent: invalid symbol / overflow
constexpr int kScanMaxChunk = 1 << 16;     // largest steps per chunk
struct ScanLaunch {
  SeqArgs seq;
  ModelArgs mod;
  const int64_t* coff;  // [S + 1] first chunk of each sequence, coff[S] = all chunks
  float* P;             // [span][cap][NP][NP] chunk products, row-normalised
  int32_t* E;           // [span][cap][NP] base-2 exponent of each row
  int64_t cap;          // chunk slots per model slot
  int L;                // steps per chunk
  float* loglik;
  int32_t* argmax;
  int32_t* done;
  int32_t* queue;       // [0] chunk items, [1] pair items
  int32_t* status;
  int n_pair_items;     // warps' worth of pairs in the combine
};
// phase 0: chunk products (max_chunks bounds the device's chunk count);
// phase 1: combine
cudaError_t launch_scan(int NP, const ScanLaunch& a, int64_t max_chunks, int phase,
                        cudaStream_t st);
size_t fb_seg_smem_bytes(int NP, int G, int C, int M, int warps);

struct MmaFwdLaunch {
  SeqArgs seq;
  ModelArgs mod;      // probability tables padded to NP (64 or 128)
  float* loglik;      // [S][K]
  int32_t* argmax;    // [S] or NULL
  int32_t* done;      // per tile pair
  int32_t* queue;
  int32_t* status;
  int n_items;        // ceil(n_tiles / tiles per CTA) * K
  int n_tiles;        // ceil(S / 128)
  uint32_t wait_limit;  // polls before a step's mbarrier wait gives up
};
cudaError_t launch_forward_mma(int NP, bool tf32, const MmaFwdLaunch& a, cudaStream_t st);
int mma_tiles_per_cta(int NP);  // 128-row tiles one CTA of the tensor-core forward holds

// Launch arguments of the tensor-core recursions above 128 states: the
// cluster kernels of mma_cluster.cu (tiles of 32, 64 or 128 rows on N_pad / 64
// CTAs, forward and the adjoint's passes) and the streamed-A^T forward of
// mma_wide.cu (one 128-row tile per CTA, A^T from a BF16 image built per
// call), which serves only what the cluster cannot take.
struct MmaWideLaunch {
  SeqArgs seq;
  ModelArgs mod;      // probability tables padded to NP (256 or 512)
  uint8_t* img;       // [K][NP * NP] BF16 image of A^T, chunk-major
  float* loglik;      // [S][K]
  int32_t* argmax;    // [S] or NULL
  int32_t* done;      // per tile
  int32_t* queue;
  int32_t* status;
  int n_items;        // n_tiles * K
  int n_tiles;        // ceil(S / rows)
  int rows;           // rows per tile: 128 (the cluster kernel: 32, 64 or 128)
  // per-step rows for the adjoint above 128 states (xs NULL: recognition only)
  float* xs;             // [K][rtot][NP] forward: scaled alpha_t; backward: scaled beta_t
  int32_t* xe;           // backward: [K][rtot] power of two removed at each step
  const int64_t* roff;   // [S] first row of each sequence (exclusive prefix of lengths)
  int64_t rtot;          // rows per model
  uint32_t wait_limit;   // polls before a step's mbarrier wait gives up
};
// The forward above 128 states over a cluster of N_pad / 64 CTAs, each with its
// column slice of A resident (mma_cluster.cu); serves M symbols when its
// emission slice fits beside them.
bool forward_cluster_fits(int NP, int M);
// The cluster kernels' rows per tile for S sequences x K models x dirs passes.
int cluster_tile_rows(int NP, int S, int K, int dirs);
cudaError_t launch_forward_cluster(int NP, const MmaWideLaunch& a, cudaStream_t st);
// Both passes of the adjoint above 128 states on clusters, in one launch:
// clusters [0, f.n_items) the forward items of f (rows alpha_t kept in f.xs),
// the others the backward items of b (rows beta_t in b.xs, their exponents in
// b.xe); needs forward_cluster_fits.
cudaError_t launch_cluster_passes(int NP, const MmaWideLaunch& f, const MmaWideLaunch& b,
                                  cudaStream_t st);
// Counts of the adjoint above 128 states from the two passes' rows (fb_wide.cu).
struct FbWideArgs {
  int K, N, M, NP, S;
  int labelled;          // model_of_seq given (K == 1)
  int64_t rtot;          // rows per model
  float* X;              // [K][rtot][NP] forward rows, overwritten by U if u_in_x
  int u_in_x;            // 1: U replaces X; 0: the contraction reads X, V carries w / z
  const float* Bh;       // [K][rtot][NP] backward rows
  float* V;              // [K][rtot][NP]
  float* G;              // [K][rtot][NP] gamma rows (weighted)
  const int32_t* xe;     // [K][rtot] backward exponents
  int32_t* sym;          // [K][rtot] symbol code of each row
  const int64_t* roff;   // [S]
  const int32_t* seqlen; // [S] validated lengths
  const int64_t* offsets;
  const int32_t* symbols;
  const float* Btp;      // [K][M][NP] padded emission table
  const float* weight;   // [S] or [S][K], or NULL
  const float* A;        // caller's [K][N][N]
  float* Cp;             // [K][nsplit][NP][NP]
  int nsplit;
  // emission counts: model k's rows in chunks of ech rows, chunks of all
  // models numbered from cbase[k]; bucket (k, m) = row symbol m, (k, M) = t 0
  int32_t* cbase;        // [K + 1] first chunk of each model
  int32_t* ehist;        // [M + 1][ncc] entries per (bucket, chunk), then offsets
  int32_t* ebase;        // [K (M + 1) + 1] first entry of each bucket
  int32_t* epbase;       // [K (M + 1) + 1] first piece of each bucket
  int32_t* elist;        // [2 nrows] rows of each bucket in ascending order
  float* epart;          // [pieces][NP] gamma sums of the pieces
  int ncc;               // chunk capacity (>= cbase[K])
  int64_t ech;           // rows per chunk
  float* cnt_pi;
  float* cnt_A;
  float* cnt_B;
  int32_t* status;
  int64_t nrows;            // rows of the buffers the combine kernel visits
  // rows in the plan's order (TF32 adjoint, N_pad = 128); NULL: by sequence
  const int64_t* pos_row;   // [positions] first row of the plan's position p
  int32_t* row_pos;         // [rtot] position of each row (filled by launch_fbw_counts)
  const int32_t* sorted;    // [positions] sequence at position p
  const int32_t* n_valid;   // device count of positions
  const int32_t* model_of_seq;  // labelled: [S]
  const int64_t* mrow;      // [2 (K + 1)] model k's rows [mrow[k], mrow[K + 1 + k])
};
cudaError_t launch_fbw_counts(const FbWideArgs& a, cudaStream_t st);
// Emission-count buffers of launch_fbw_counts for `nrows` rows (element
// counts; cbase has K + 1, epbase as many as ebase).
struct FbwEmisSizes {
  int64_t ech, ncc, ehist, ebase, elist, epart;
};
FbwEmisSizes fbw_emis_sizes(int K, int M, int NP, int64_t nrows);

// The recognition forward above 128 states with A^T streamed, one CTA per
// tile (loglik, argmax; xs NULL): where the cluster kernel has no room.
cudaError_t launch_forward_wide(int NP, const MmaWideLaunch& a, cudaStream_t st);

// Plan of the tensor-core adjoint: the rows of every 128-row tile share one
// model, and the tile composition is a deterministic function of the input
// (stable sort by model, then decreasing length, then sequence index), so the
// per-tile count sums are bitwise reproducible.
struct MmaPlanArgs {
  int S, K, labelled;
  const int32_t* seqlen;        // validated lengths (-1 = invalid)
  const int32_t* model_of_seq;  // labelled mode
  float* loglik;                // rows in no tile: 0 (T = 0) or NaN (invalid)
  int32_t* sorted;              // [S] tile rows, in tile order
  int32_t* tmp;                 // [S] scratch
  uint32_t* key;                // [max(S, cap)] sort keys of `sorted` (model << 10 | length key)
  uint32_t* key_tmp;            // [max(S, cap)] scratch
  int32_t* tile_start;          // [cap] first row (index into sorted)
  int32_t* tile_rows;           // [cap] rows in the tile (1..128)
  int32_t* tile_model;          // [cap]
  int32_t* tile_len;            // [cap] longest row (-1 for unused entries)
  int32_t* tile_order;          // [cap] tiles by decreasing length
  int32_t* tile_tmp;            // [cap] scratch
  int32_t* group_start;         // [K] labelled: first sorted position of each model
  int32_t* group_end;           // [K] ... and one past its last
  int n_tiles_cap;
  int32_t* n_tiles;             // device count
  int32_t* bcnt;                // [ceil(S / 4096)] valid rows per block, then offsets
  int32_t* hist;                // [256][ceil(S / 4096)] digit counts, then offsets
  int32_t* n_valid;             // device count of rows with T >= 1
  // work lists of the two adjoint kernels (plan_items_kernel)
  int group;                    // tiles per pass group (the pass kernel's tiles per CTA)
  int spr;                      // checkpoint segments per range item
  int32_t* pass_tiles;          // [pass_cap][group] tile ids (-1: none), longest group first
  int32_t* pass_tmp;            // [2][pass_cap] scratch
  int32_t* n_pass;              // device count of pass groups
  int pass_cap;
  int32_t* rng_tile;            // [rng_cap] tile of each range item (longest tiles first)
  int32_t* rng_seg;             // [rng_cap] first | last segment << 16
  int32_t* rng_model;           // [rng_cap] model (0 for unused entries)
  int32_t* rng_len;             // [rng_cap] the tile's length (-1 for unused entries)
  int32_t* n_rng;               // device count of range items
  int rng_cap;
};
// Plan scratch bytes for S sequences (bcnt, hist, n_valid).
inline size_t mma_plan_scratch_bytes(int64_t S) {
  const int64_t nb = (S + 4095) / 4096 > 0 ? (S + 4095) / 4096 : 1;
  return (size_t)(nb + 256 * nb + 8) * 4;
}
cudaError_t launch_mma_plan(const MmaPlanArgs& a, cudaStream_t st);

// The adjoint's pass kernel (mma_pass.cu): for every group of tiles of one
// model, the forward recursion (direction 0: checkpoints of alpha, per-step
// exponents, log P and the last row sum) or the backward recursion run as the
// forward one with A in place of A^T in reversed time (direction 1:
// checkpoints of the beta-side operand Y_t = b(o_t) . beta_t, scaled).
struct MmaPassLaunch {
  SeqArgs seq;
  ModelArgs mod;                // probability tables padded to NP
  const int32_t* sorted;        // plan: tile rows
  const int32_t* tile_start;
  const int32_t* tile_rows;
  const int32_t* tile_model;
  const int32_t* tile_len;
  const int32_t* pass_tiles;    // [groups][NT] tile ids (-1: none)
  const int32_t* n_pass;        // device count of groups; items = 2 * groups
  int labelled;
  float* loglik;                // [S] or [S][K]
  uint8_t* ckx;                 // per tile: alpha images at t = c C, c = 0 .. NS - 1
  uint8_t* cky;                 // per tile: Y images at t = c C, c = 1 .. NS - 1
  int64_t ck_stride;            // bytes per tile (of each of ckx, cky)
  int8_t* gexp;                 // per tile: [max_len][128] forward scale exponents
  int64_t gexp_stride;          // bytes per tile
  float* s_last;                // per tile: [128] row sum at the row's last step (0: none,
                                // NaN: invalid row)
  int32_t* queue;
  int32_t* status;
  uint32_t wait_limit;
  // TF32 adjoint (mma_pass_tf32.cu): every step's rows instead of checkpoints
  float* xs;                    // [rows][NP] scaled alpha_t
  float* bhs;                   // [rows][NP] scaled beta_t
  int32_t* xe;                  // [rows] backward exponents
  const int64_t* rp;            // [S] first row of each sequence (plan order)
  int64_t rtot;                 // rows of a model's block (every sequence x every model)
};
// The TF32 adjoint's passes (row offsets first: rp, pos_row [positions],
// mrow [2 (K + 1)]); fb_tf32_supported: its shared memory fits.
bool fb_tf32_supported(int NP, int M);
cudaError_t launch_fb_pass_tf32(int NP, const MmaPassLaunch& a, const int32_t* n_valid,
                                int64_t* pos_row, int64_t* mrow, cudaStream_t st);
// Tiles per CTA of the pass kernel for a batch of up to `tiles` tiles (the
// plan's pass groups have this many tiles).
int fb_pass_tiles_per_cta(int NP, int tiles);
cudaError_t launch_fb_pass(int NP, int tiles_per_cta, const MmaPassLaunch& a, cudaStream_t st);

// The adjoint's second kernel (mma_fb.cu): one work item per (tile, range of
// checkpoint segments), from the pass kernel's checkpoints.
struct MmaFbLaunch {
  SeqArgs seq;
  ModelArgs mod;                // probability tables padded to NP
  const float* weight;          // [S] or [S][K], NULL = 1
  const int32_t* sorted;
  const int32_t* tile_start;
  const int32_t* tile_rows;
  const int32_t* tile_model;
  const int32_t* tile_len;
  const int32_t* rng_tile;      // [items] tile of each item
  const int32_t* rng_seg;       // [items] first | last segment << 16
  const int32_t* n_rng;         // device count of items
  int labelled;
  float* slots;                 // [item][slot_floats] per-item counts
  int64_t slot_floats;
  const uint8_t* ckx;           // per tile: alpha checkpoint images (the pass kernel's)
  const uint8_t* cky;           // per tile: Y checkpoint images
  int64_t ck_stride;
  const int8_t* gexp;           // per tile: [max_len][128] forward scale exponents
  int64_t gexp_stride;
  const float* s_last;          // per tile: [128] row sum at the row's last step
  uint8_t* scr;                 // per CTA: recomputed segment images
  float* gbuf;                  // per CTA: [128][NP] gamma_1 rows
  float* psum;                  // per CTA: [2][4][128] row partial sums
  int64_t scr_bytes;            // per-CTA stride of scr
  int32_t* queue;
  int32_t* status;
  uint32_t wait_limit;          // polls before a step's mbarrier wait gives up
};
cudaError_t launch_fb_mma(int NP, int M, int grid, const MmaFbLaunch& a, cudaStream_t st);
// Checkpoint stride of a tile whose longest row has L steps, and the per-CTA
// buffer sizes of the tensor-core adjoint for sequences up to max_len.
__host__ __device__ inline int fb_mma_segment(int L) {
  long long c = (long long)sqrtf((float)(L > 1 ? L : 1));
  if (c < 1) c = 1;
  while (c * c < L) ++c;                       // ceil(sqrt(L))
  while (c > 1 && (c - 1) * (c - 1) >= L) --c;
  if (L <= 8192 && c > 16) c = 16;             // recompute buffer sized for L2
  return (int)c;
}
int fb_mma_ctas_per_sm(int NP, int M);
bool fb_mma_supported(int NP, int M);

struct ReduceLaunch {
  const float* partial;  // [planes][S (or S * K)][slot_floats]
  float* red1;
  const int32_t* model_of_seq;
  const int32_t* seqlen;
  int S, K, N, M, NP;
  int planes;
  int64_t slot_floats;
  int nchunks;
  float* cnt_pi;
  float* cnt_A;
  float* cnt_B;
};
cudaError_t launch_reduce(const ReduceLaunch& a, cudaStream_t st);

// Instantiated lane counts per (op, NP); the first entry is the default.
int candidates(int op, int NP, int* out, int cap);
int plan_blocks(int S);  // plan blocks of the setup for S sequences
size_t forward_ws_sequential(const hmm_dims_t& d, const hmm_seqs_t& q);
int num_sms();
// Polls a tensor-core kernel's per-step mbarrier wait makes before it gives
// up (hmm_set_wait_limit; the drain waits after a give-up keep kDrainPolls).
uint32_t wait_limit_polls();
constexpr uint32_t kDrainPolls = 1u << 24;

}  // namespace hmmgb
