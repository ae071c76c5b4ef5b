// viterbi_wide.cu -- Viterbi decoding above 64 states (up to 128), FP32 SIMT
// (Sec. 2.7 "Viterbi"; Rabiner 1989 eqs. 32-35).
//
// The same recursion, shifts and tie-breaks as viterbi.cu, with one warp per
// (sequence, model) pair and four consecutive states j per lane. The log
// transition matrix (128 x 128 FP32, 64 KB) no longer fits a lane's
// registers, so it is staged in shared memory per work item and every step
// reads it row by row: lane l takes log a_{i, 4l .. 4l+3} as one 16-byte load
// (conflict-free across the warp) and delta_{t-1}(i) as a broadcast, four
// rows at a time.
//
//  * scores: all-models items are (group of 16 sequences, model): four warps
//    of four pairs each share the model's matrix, every row read from shared
//    memory serving four pairs; labelled pairs and model sets use one-warp
//    blocks (one pair, one matrix).
//  * paths: one-warp blocks (the decoded model differs per sequence); the
//    smallest maximising predecessor of each state is stored as one byte per
//    (t, j), 128 bytes per step written by the warp as one line, and the
//    backtrack walks 32 rows at a time from registers with one shuffle per
//    step, as in viterbi.cu.
#include "hmm_internal.cuh"

namespace hmmgb {

namespace {

constexpr int kVW = 128;  // padded states served here

__device__ __forceinline__ float nan_w() { return __int_as_float(0x7fc00000); }

// Shift the warp's 128-state vector (4 per lane) by its maximum rounded to a
// multiple of 2^-15; false when every entry is -inf.
__device__ __forceinline__ bool shift_max(float (&x)[4], long long& Q, bool apply) {
  float m = group_max<32>(fmaxf(fmaxf(x[0], x[1]), fmaxf(x[2], x[3])));
  if (!apply) return true;
  if (m == -INFINITY) return false;
  const int q = __float2int_rn(m * kViterbiQuant);
  const float qf = (float)q * (1.f / kViterbiQuant);
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) x[jj] -= qf;
  Q += q;
  return true;
}

// Stages the log transition matrix of model k (padded rows) in shared memory.
__device__ __forceinline__ void stage_la(float* lA, const float* Ap, int k, int nthreads) {
  const float4* src = reinterpret_cast<const float4*>(Ap + (size_t)k * kVW * kVW);
  float4* dst = reinterpret_cast<float4*>(lA);
  for (int i = threadIdx.x; i < kVW * kVW / 4; i += nthreads) dst[i] = __ldg(src + i);
}

// m[jj] = max_i (x_i + la_{i, j0+jj}); with ARG also the smallest maximising i.
// The sums are packed FP32x2 adds (rounded like scalar adds) and, without
// ARG, two rows fold into one three-input max: the maximum is exact in any
// grouping, so both variants return the same values.
template <bool ARG>
__device__ __forceinline__ void maxplus_smem(const float* xb, const float* lA, int j0,
                                             float (&m)[4], int (&arg)[4]) {
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) { m[jj] = -INFINITY; arg[jj] = 0; }
#pragma unroll 4
  for (int i4 = 0; i4 < kVW / 4; ++i4) {
    const float4 xv = *reinterpret_cast<const float4*>(xb + 4 * i4);
    const float xi[4] = {xv.x, xv.y, xv.z, xv.w};
    float2 v01[4], v23[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 la = *reinterpret_cast<const float4*>(lA + (4 * i4 + u) * kVW + j0);
      const float2 xx = make_float2(xi[u], xi[u]);
      v01[u] = fadd2(xx, make_float2(la.x, la.y));
      v23[u] = fadd2(xx, make_float2(la.z, la.w));
    }
    if constexpr (ARG) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * i4 + u;
        const float v[4] = {v01[u].x, v01[u].y, v23[u].x, v23[u].y};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (v[jj] > m[jj]) { m[jj] = v[jj]; arg[jj] = i; }
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; u += 2) {
        m[0] = fmax3(m[0], v01[u].x, v01[u + 1].x);
        m[1] = fmax3(m[1], v01[u].y, v01[u + 1].y);
        m[2] = fmax3(m[2], v23[u].x, v23[u + 1].x);
        m[3] = fmax3(m[3], v23[u].y, v23[u + 1].y);
      }
    }
  }
}

}  // namespace

// m[p][jj] = max_i (x_p(i) + la_{i, j0+jj}) for P pairs of one model: every
// row of log A read from shared memory serves all P pairs. Same values as
// maxplus_smem (exact maxima, identically rounded sums).
template <int P>
__device__ __forceinline__ void maxplus_smem_multi(const float* xb, const float* lA, int j0,
                                                   float (&m)[P][4]) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) m[p][jj] = -INFINITY;
#pragma unroll 2
  for (int i4 = 0; i4 < kVW / 4; ++i4) {
    float4 xv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) xv[p] = *reinterpret_cast<const float4*>(xb + p * 2 * kVW + 4 * i4);
#pragma unroll
    for (int uu = 0; uu < 4; uu += 2) {
      const float4 l0 = *reinterpret_cast<const float4*>(lA + (4 * i4 + uu) * kVW + j0);
      const float4 l1 = *reinterpret_cast<const float4*>(lA + (4 * i4 + uu + 1) * kVW + j0);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float x0 = uu == 0 ? xv[p].x : xv[p].z;
        const float x1 = uu == 0 ? xv[p].y : xv[p].w;
        const float2 a01 = fadd2(make_float2(x0, x0), make_float2(l0.x, l0.y));
        const float2 a23 = fadd2(make_float2(x0, x0), make_float2(l0.z, l0.w));
        const float2 b01 = fadd2(make_float2(x1, x1), make_float2(l1.x, l1.y));
        const float2 b23 = fadd2(make_float2(x1, x1), make_float2(l1.z, l1.w));
        m[p][0] = fmax3(m[p][0], a01.x, b01.x);
        m[p][1] = fmax3(m[p][1], a01.y, b01.y);
        m[p][2] = fmax3(m[p][2], a23.x, b23.x);
        m[p][3] = fmax3(m[p][3], a23.y, b23.y);
      }
    }
  }
}

// W warps per block, P pairs per warp. All-models items without model sets
// are (group of W * P sequences, model): every pair of the block has the
// model whose matrix the block staged. Labelled pairs and model sets: one
// pair per block (W = P = 1).
template <int W, int P, bool ALL>
__global__ void __launch_bounds__(W * 32) hmm_viterbi_scores_wide(VitLaunch a) {
  extern __shared__ __align__(16) float vsm[];
  float* lA = vsm;                                  // [128][128]
  float* xs = vsm + kVW * kVW;                      // [W][P][2][128]
  __shared__ int item_s;
  __shared__ int last_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, j0 = 4 * lane;
  const int M = a.seq.M, S = a.seq.S;
  const int span = a.seq.span;
  const bool param_bad = (__ldcg(a.status) & HMM_STATUS_PARAM) != 0;
  float* xw = xs + warp * P * 2 * kVW;

  for (;;) {
    __syncthreads();  // the previous item's readers of lA are done
    if (threadIdx.x == 0) item_s = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = item_s;
    if (item >= a.n_items_score) break;
    const int g = ALL ? item / span : item;
    const int kr = ALL ? item % span : 0;
    int s[P], Tn[P];
    bool has[P], bad[P], dead[P];
    long long Q[P];
    float x[P][4];
    float4 bn[P];
    int on[P], o2[P], err[P];
    const int32_t* o[P];
    int k = kr;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int pos = (g * W + warp) * P + p;
      has[p] = pos < S;
      s[p] = has[p] ? a.seq.order[pos] : 0;
      const int T = has[p] ? a.seq.seqlen[s[p]] : 0;
      if (P == 1) {  // one pair: its own model
        if (!ALL && has[p] && T >= 0) k = a.seq.model_of_seq[s[p]];
        if (ALL && has[p] && T >= 0 && a.seq.model_base) k += a.seq.model_base[s[p]];
      }
      bad[p] = T < 0 || param_bad;
      Tn[p] = T < 0 ? 0 : T;
      dead[p] = false;
      Q[p] = 0;
      err[p] = 0;
    }
    stage_la(lA, a.mod.Ap, k, W * 32);
    __syncthreads();

    const float* Bk = a.mod.Btp + (size_t)k * M * kVW + j0;
    int Tmax = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      Tmax = max(Tmax, Tn[p]);
      o[p] = a.seq.symbols + (has[p] && Tn[p] > 0 ? a.seq.offsets[s[p]] : 0);
      int o0 = Tn[p] > 0 ? __ldg(o[p]) : 0;
      if ((unsigned)o0 >= (unsigned)M) { bad[p] = true; err[p] |= HMM_STATUS_SYMBOL; o0 = 0; }
      const float4 b = __ldg(reinterpret_cast<const float4*>(Bk + (size_t)o0 * kVW));
      const float4 pv = __ldg(reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * kVW + j0));
      x[p][0] = pv.x + b.x; x[p][1] = pv.y + b.y; x[p][2] = pv.z + b.z; x[p][3] = pv.w + b.w;
      if (!shift_max(x[p], Q[p], Tn[p] > 0 && !bad[p])) dead[p] = true;
      on[p] = 0;
      if (1 < Tn[p]) {
        on[p] = __ldg(o[p] + 1);
        if ((unsigned)on[p] >= (unsigned)M) { bad[p] = true; err[p] |= HMM_STATUS_SYMBOL; on[p] = 0; }
      }
      bn[p] = __ldg(reinterpret_cast<const float4*>(Bk + (size_t)on[p] * kVW));
      o2[p] = (2 < Tn[p]) ? __ldg(o[p] + 2) : 0;
    }

    for (int t = 1; t < Tmax; ++t) {  // warp-uniform: the longest of the warp's pairs
#pragma unroll
      for (int p = 0; p < P; ++p)
        *reinterpret_cast<float4*>(xw + (p * 2 + (t & 1)) * kVW + j0) =
            make_float4(x[p][0], x[p][1], x[p][2], x[p][3]);
      __syncwarp();
      float m[P][4];
      maxplus_smem_multi<P>(xw + (t & 1) * kVW, lA, j0, m);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const bool act = t < Tn[p] && !dead[p] && !bad[p];
        const float4 b = bn[p];
        if (t + 1 < Tn[p]) {
          on[p] = o2[p];
          if ((unsigned)on[p] >= (unsigned)M) { bad[p] = true; err[p] |= HMM_STATUS_SYMBOL; on[p] = 0; }
          bn[p] = __ldg(reinterpret_cast<const float4*>(Bk + (size_t)on[p] * kVW));
          if (t + 2 < Tn[p]) o2[p] = __ldg(o[p] + t + 2);
        }
        m[p][0] += b.x; m[p][1] += b.y; m[p][2] += b.z; m[p][3] += b.w;
        const long long Qold = Q[p];
        if (!shift_max(m[p], Q[p], act)) dead[p] = true;
        if (act && !dead[p]) {
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) x[p][jj] = m[p][jj];
        } else {
          Q[p] = Qold;
        }
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float fm = group_max<32>(fmaxf(fmaxf(x[p][0], x[p][1]), fmaxf(x[p][2], x[p][3])));
      if (has[p] && lane == 0) {
        float out;
        if (bad[p]) {
          out = nan_w();
          if (err[p]) set_status(a.status, err[p]);
        } else if (Tn[p] == 0) {
          out = 0.f;
        } else if (dead[p]) {
          out = -INFINITY;
        } else {
          out = (float)((double)fm + (double)Q[p] * (1.0 / kViterbiQuant));
        }
        a.score[ALL ? (size_t)s[p] * span + kr : (size_t)s[p]] = out;
        if (!ALL && a.best) a.best[s[p]] = bad[p] ? -1 : k;
      }
    }

    if (ALL && a.best) {
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        last_s = atomicAdd(a.done + g, 1) == span - 1;
      }
      __syncthreads();
      if (last_s) {
        __threadfence();
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (has[p] && lane == 0) {
            const float* row = a.score + (size_t)s[p] * span;
            float best = __ldcg(row);
            int barg = isnan(best) ? -1 : 0;
            for (int kk = 1; kk < span; ++kk) {
              const float v = __ldcg(row + kk);
              if (isnan(v)) barg = -1;
              else if (barg >= 0 && v > best) { best = v; barg = kk; }
            }
            a.best[s[p]] = barg;
          }
        }
      }
    }
  }
}

// Groups the sequences by decoded (or labelled) model for the path kernel:
// gorder holds each model's sequences (visited in length order) in a segment
// padded with -1 to a multiple of kPathGroup, segments in model order, and
// the rejected or undecoded ones in a last segment; gcount = the number of
// kPathGroup-entry items. One block; nk = K + 1 buckets in shared memory.
constexpr int kPathGroup = 4;

__device__ __forceinline__ int path_bucket(const VitLaunch& a, int s, int nk) {
  const int T = a.seq.seqlen[s];
  if (T < 0) return nk - 1;
  if (a.seq.model_of_seq) return a.seq.model_of_seq[s];  // validated by the setup
  const int b = __ldcg(a.best + s);
  if (b < 0 || b >= a.seq.span) return nk - 1;
  return b + (a.seq.model_base ? a.seq.model_base[s] : 0);
}

__global__ void __launch_bounds__(1024) vw_group_kernel(VitLaunch a, int nk) {
  extern __shared__ int gsm[];
  int* hist = gsm;       // [nk]
  int* cur = gsm + nk;   // [nk]
  __shared__ int wsum[32];
  const int tid = threadIdx.x, S = a.seq.S;
  for (int k = tid; k < nk; k += 1024) hist[k] = 0;
  __syncthreads();
  for (int pos = tid; pos < S; pos += 1024) atomicAdd(&hist[path_bucket(a, a.seq.order[pos], nk)], 1);
  __syncthreads();
  // exclusive prefix of the padded segment sizes: thread t owns buckets
  // [t per, t per + per)
  const int per = (nk + 1023) / 1024;
  const int k0 = tid * per, k1 = min(nk, k0 + per);
  int local = 0;
  for (int k = k0; k < k1; ++k) local += (hist[k] + kPathGroup - 1) / kPathGroup * kPathGroup;
  int x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(HMM_FULL_MASK, x, o);
    if ((tid & 31) >= o) x += y;
  }
  if ((tid & 31) == 31) wsum[tid >> 5] = x;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < (tid >> 5); ++w) wbase += wsum[w];
  int run = wbase + x - local;
  for (int k = k0; k < k1; ++k) {
    const int padded = (hist[k] + kPathGroup - 1) / kPathGroup * kPathGroup;
    cur[k] = run;
    for (int j = run + hist[k]; j < run + padded; ++j) a.gorder[j] = -1;
    run += padded;
  }
  if (tid == 1023) *a.gcount = run / kPathGroup;  // the last thread's run is the total
  __syncthreads();
  for (int pos = tid; pos < S; pos += 1024) {
    const int s = a.seq.order[pos];
    a.gorder[atomicAdd(&cur[path_bucket(a, s, nk)], 1)] = s;
  }
}

// W = 1: one pair per block, items in length order. W = kPathGroup: the
// items of vw_group_kernel, whose W sequences share one decoded model, so the
// block stages one matrix for W warps (one pair each).
template <int W>
__global__ void __launch_bounds__(W * 32) hmm_viterbi_paths_wide(VitLaunch a) {
  constexpr int CH = 32;  // backtrack rows fetched per chunk
  extern __shared__ __align__(16) float vsm[];
  __shared__ int item_s, kblk_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, j0 = 4 * lane;
  float* lA = vsm;
  float* xs = vsm + kVW * kVW + warp * 2 * kVW;  // [2][128] per warp
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;
  const int span = a.seq.span;
  const bool labelled = a.seq.model_of_seq != nullptr;
  const bool param_bad = (__ldcg(a.status) & HMM_STATUS_PARAM) != 0;
  const int n_items = W == 1 ? a.n_items_path : __ldcg(a.gcount);

  for (;;) {
    __syncthreads();  // the previous item's readers of lA are done
    if (threadIdx.x == 0) {
      item_s = atomicAdd(a.queue + 1, 1);
      kblk_s = INT_MAX;
    }
    __syncthreads();
    const int item = item_s;
    if (item >= n_items) break;
    bool has;
    int s;
    if (W == 1) {
      has = item < S;
      s = has ? a.seq.order[item] : 0;
    } else {
      const int e = __ldcg(a.gorder + item * W + warp);
      has = e >= 0;
      s = has ? e : 0;
    }
    const int T = has ? a.seq.seqlen[s] : 0;
    int k = 0;
    bool bad = T < 0 || param_bad;
    if (has && T >= 0) {
      if (labelled) {
        k = a.seq.model_of_seq[s];
        if (k < 0 || k >= K) { bad = true; k = 0; }
      } else {
        k = __ldcg(a.best + s);
        if (k < 0 || k >= span) { bad = true; k = 0; }
        else if (a.seq.model_base) k += a.seq.model_base[s];
      }
    }
    int kb = k;
    if (W > 1) {  // the block's model (one per item by construction)
      if (lane == 0 && has && !bad) atomicMin(&kblk_s, k);
      __syncthreads();
      kb = kblk_s == INT_MAX ? 0 : kblk_s;
      if (has && !bad && k != kb) bad = true;
      k = kb;
    }
    const int Tn = (T < 0) ? 0 : T;
    stage_la(lA, a.mod.Ap, kb, W * 32);
    __syncthreads();

    const float* Bk = a.mod.Btp + (size_t)k * M * kVW + j0;
    const long long off = (has && T >= 0) ? a.seq.offsets[s] : 0;
    const int32_t* o = a.seq.symbols + off;
    uint8_t* bp = a.bp + ((has && T >= 0) ? a.bpoff[s] : 0) * (long long)kVW + j0;

    float x[4];
    long long Q = 0;
    bool dead = false;
    int err = 0;
    {
      int o0 = Tn > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; o0 = 0; }
      const float4 b = __ldg(reinterpret_cast<const float4*>(Bk + (size_t)o0 * kVW));
      const float4 pv = __ldg(reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * kVW + j0));
      x[0] = pv.x + b.x; x[1] = pv.y + b.y; x[2] = pv.z + b.z; x[3] = pv.w + b.w;
      if (!shift_max(x, Q, Tn > 0 && !bad)) dead = true;
    }
    int on = 0;
    if (1 < Tn) {
      on = __ldg(o + 1);
      if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
    }
    float4 bn = __ldg(reinterpret_cast<const float4*>(Bk + (size_t)on * kVW));
    int o2 = (2 < Tn) ? __ldg(o + 2) : 0;

    for (int t = 1; t < Tn; ++t) {
      const bool act = !dead && !bad;
      float* xb = xs + (t & 1) * kVW;
      *reinterpret_cast<float4*>(xb + j0) = make_float4(x[0], x[1], x[2], x[3]);
      __syncwarp();
      float m[4];
      int arg[4];
      maxplus_smem<true>(xb, lA, j0, m, arg);
      const float4 b = bn;
      if (t + 1 < Tn) {
        on = o2;
        if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
        bn = __ldg(reinterpret_cast<const float4*>(Bk + (size_t)on * kVW));
        if (t + 2 < Tn) o2 = __ldg(o + t + 2);
      }
      m[0] += b.x; m[1] += b.y; m[2] += b.z; m[3] += b.w;
      const long long Qold = Q;
      if (!shift_max(m, Q, act)) dead = true;
      if (act && !dead) {
        const uint32_t w = (uint32_t)(arg[0] & 0xff) | ((uint32_t)(arg[1] & 0xff) << 8) |
                           ((uint32_t)(arg[2] & 0xff) << 16) | ((uint32_t)(arg[3] & 0xff) << 24);
        *reinterpret_cast<uint32_t*>(bp + (long long)t * kVW) = w;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) x[jj] = m[jj];
      } else {
        Q = Qold;
      }
    }

    // final state: smallest argmax of delta_T
    float fv = x[0];
    int fj = j0;
#pragma unroll
    for (int jj = 1; jj < 4; ++jj)
      if (x[jj] > fv) { fv = x[jj]; fj = j0 + jj; }
#pragma unroll
    for (int o5 = 16; o5 > 0; o5 >>= 1) {
      const float v2 = __shfl_xor_sync(HMM_FULL_MASK, fv, o5);
      const int j2 = __shfl_xor_sync(HMM_FULL_MASK, fj, o5);
      if (v2 > fv || (v2 == fv && j2 < fj)) { fv = v2; fj = j2; }
    }
    if (has && lane == 0) {
      float out;
      if (bad) {
        out = nan_w();
        if (err) set_status(a.status, err);
      } else if (Tn == 0) {
        out = 0.f;
      } else if (dead) {
        out = -INFINITY;
      } else {
        out = (float)((double)fv + (double)Q * (1.0 / kViterbiQuant));
      }
      if (labelled) {
        a.score[s] = out;
        if (a.best) a.best[s] = bad ? -1 : k;
      }
    }
    if (!a.path) continue;

    // backtrack: 32 rows of this lane's four bytes at a time
    const bool walk = has && !bad && !dead && Tn > 0;
    int q = walk ? fj : 0;
    if (has && Tn > 0 && lane == 0) a.path[off + Tn - 1] = bad ? -1 : q;
    for (int tc = Tn - 1; tc >= 1; tc -= CH) {
      uint32_t rows[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = tc - u;
        rows[u] = (walk && t >= 1) ? __ldcg(reinterpret_cast<const unsigned int*>(
                                         bp + (long long)t * kVW)) : 0u;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = tc - u;
        const int owner = q >> 2;
        const uint32_t byte = (rows[u] >> (8 * (q & 3))) & 0xffu;
        const int nq = __shfl_sync(HMM_FULL_MASK, (int)byte, owner);
        if (has && t >= 1) {
          if (walk) q = nq;
          if (lane == (t - 1) % 32) a.path[off + t - 1] = bad ? -1 : (dead ? 0 : q);
        }
      }
    }
  }
}

size_t viterbi_group_smem(int nk) { return (size_t)2 * nk * 4; }

size_t viterbi_wide_smem(int warps, int pairs) {
  return ((size_t)kVW * kVW + (size_t)warps * pairs * 2 * kVW) * 4;
}

template <typename Kern>
static cudaError_t launch_vw(Kern kern, int warps, int pairs, int n_items, const VitLaunch& a,
                             cudaStream_t st) {
  const size_t smem = viterbi_wide_smem(warps, pairs);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int blocks = num_sms() * per_sm;
  if (blocks > n_items) blocks = n_items > 0 ? n_items : 1;
  kern<<<blocks, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_viterbi_scores_wide(const VitLaunch& a, cudaStream_t st) {
  if (a.seq.model_of_seq != nullptr)
    return launch_vw(hmm_viterbi_scores_wide<1, 1, false>, 1, 1, a.n_items_score, a, st);
  if (a.seq.model_base == nullptr)
    return launch_vw(hmm_viterbi_scores_wide<4, 4, true>, 4, 4, a.n_items_score, a, st);
  return launch_vw(hmm_viterbi_scores_wide<1, 1, true>, 1, 1, a.n_items_score, a, st);
}

cudaError_t launch_viterbi_paths_wide(const VitLaunch& a, cudaStream_t st) {
  const int nk = a.seq.K + 1;
  if (!a.gorder || !a.gcount || viterbi_group_smem(nk) > 200 * 1024)
    return launch_vw(hmm_viterbi_paths_wide<1>, 1, 1, a.n_items_path, a, st);
  const size_t gs = viterbi_group_smem(nk);
  cudaError_t e = cudaFuncSetAttribute(vw_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gs);
  if (e != cudaSuccess) return e;
  vw_group_kernel<<<1, 1024, gs, st>>>(a, nk);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // at most (S + nk (kPathGroup - 1)) / kPathGroup items; the kernel reads the count
  const int max_items = (a.seq.S + nk * (kPathGroup - 1) + kPathGroup - 1) / kPathGroup;
  return launch_vw(hmm_viterbi_paths_wide<kPathGroup>, kPathGroup, 1, max_items, a, st);
}

}  // namespace hmmgb
