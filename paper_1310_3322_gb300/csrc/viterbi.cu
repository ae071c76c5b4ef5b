// viterbi.cu -- Viterbi decoding, FP32 SIMT (Sec. 2.7 "Viterbi"; Rabiner 1989
// eqs. 32-35), in two kernels:
//
//  * scores: the max-plus recursion delta_t(j) = max_i(delta_{t-1}(i) + log a_ij)
//    + log b_j(o_t) for every scored pair, with the work decomposition of the
//    forward kernel (G lanes per pair, P pairs per warp, length-sorted atomic
//    queue). The inner step is one packed FP32x2 add and one three-input max
//    per two (i, j) terms. Every step the vector is shifted by its maximum
//    rounded to a multiple of 2^-15 (exactly representable), whose integer
//    count is summed exactly, so |delta| stays small and FP32 keeps its
//    relative precision over long sequences. The last warp of a group takes
//    the argmax over models (decoded model, smallest k on ties).
//  * paths: for the decoded model of each sequence only, the same recursion
//    with the smallest maximising predecessor tracked and stored as one byte
//    per (t, j) in the workspace, then the backtrack: each lane of the pair
//    fetches its own bytes of 32 rows at a time into registers and the chain
//    q_{t-1} = psi_t(q_t) walks them with one shuffle per step.
// Both kernels compute the same FP32 values in the same order, so the path
// kernel's score equals the score kernel's bit for bit.
#include "hmm_internal.cuh"

namespace hmmgb {

__device__ __forceinline__ float nan_f() { return __int_as_float(0x7fc00000); }

// Group argmax of (value, state) with the smallest state on ties.
template <int G>
__device__ __forceinline__ void group_argmax(float& v, int& j) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(HMM_FULL_MASK, v, o);
    const int j2 = __shfl_xor_sync(HMM_FULL_MASK, j, o);
    if (v2 > v || (v2 == v && j2 < j)) { v = v2; j = j2; }
  }
}

// Shift x by the group maximum rounded to a multiple of 2^-15; returns false
// when every entry is -inf (impossible so far).
template <int J, int G>
__device__ __forceinline__ bool normalise_max(float (&x)[J], long long& Q, bool apply) {
  float m = group_max<G>(tree_max<J>(x));
  if (!apply) return true;
  if (m == -INFINITY) return false;
  const int q = __float2int_rn(m * kViterbiQuant);
  const float qf = (float)q * (1.f / kViterbiQuant);
#pragma unroll
  for (int jj = 0; jj < J; ++jj) x[jj] -= qf;
  Q += q;
  return true;
}

template <int NP, int G, bool ALL, int NV = NP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
hmm_viterbi_scores(VitLaunch a) {
  constexpr int J = NP / G;
  constexpr int PP = 32 / G;
  constexpr int XS = NP + 4;
  __shared__ __align__(16) float xs[kWarpsPerBlock][2][PP][XS];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / G, r = lane % G, j0 = r * J;
  const int M = a.seq.M, S = a.seq.S;
  const int span = a.seq.span;  // models per sequence in all-models mode
  const bool param_bad = (__ldcg(a.status) & HMM_STATUS_PARAM) != 0;

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_items_score) break;
    const int g = ALL ? item / span : item;
    const int kr = ALL ? item % span : 0;  // model index within the sequence's set
    int k = kr;
    const int pos = g * PP + p;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    if (!ALL && has && T >= 0) k = a.seq.model_of_seq[s];
    if (ALL && has && T >= 0 && a.seq.model_base) k += a.seq.model_base[s];
    const bool bad_seq = T < 0;
    const int Tn = bad_seq ? 0 : T;
    const int Tmax = __reduce_max_sync(HMM_FULL_MASK, Tn);

    float2 a2[NP / 2][J];
    {
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP + j0;
#pragma unroll
      for (int i2 = 0; i2 < NP / 2; ++i2)
#pragma unroll
        for (int jj = 0; jj < J; ++jj)
          a2[i2][jj] = make_float2(__ldg(Ak + (2 * i2) * NP + jj), __ldg(Ak + (2 * i2 + 1) * NP + jj));
    }
    const float* Bk = a.mod.Btp + (size_t)k * M * NP + j0;
    const int32_t* o = a.seq.symbols + (has && !bad_seq ? a.seq.offsets[s] : 0);

    float x[J];
    long long Q = 0;
    bool dead = false, bad = bad_seq || param_bad;
    int err = 0;
    {
      int o0 = Tn > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; o0 = 0; }
      float b[J], pv[J];
      load_vec<J>(b, Bk + (size_t)o0 * NP);
      load_vec<J>(pv, a.mod.pip + (size_t)k * NP + j0);
#pragma unroll
      for (int jj = 0; jj < J; ++jj) x[jj] = pv[jj] + b[jj];
      if (!normalise_max<J, G>(x, Q, Tn > 0 && !bad)) dead = true;
    }
    float bn[J];
    int on = 0;
    if (1 < Tn) {
      on = __ldg(o + 1);
      if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
    }
    load_vec<J>(bn, Bk + (size_t)on * NP);
    int o2 = (2 < Tn) ? __ldg(o + 2) : 0;

    for (int t = 1; t < Tmax; ++t) {
      const bool act = t < Tn && !dead && !bad;
      float* xb = &xs[warp][t & 1][p][0];
      store_vec<J>(xb + j0, x);
      __syncwarp();
      float m[J];
      maxplus_cols<NP, J, NV>(xb, a2, m);
      float b[J];
#pragma unroll
      for (int jj = 0; jj < J; ++jj) b[jj] = bn[jj];
      if (t + 1 < Tn) {
        on = o2;
        if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
        load_vec<J>(bn, Bk + (size_t)on * NP);
        if (t + 2 < Tn) o2 = __ldg(o + t + 2);
      }
#pragma unroll
      for (int jj = 0; jj < J; ++jj) m[jj] += b[jj];
      const long long Qold = Q;
      if (!normalise_max<J, G>(m, Q, act)) dead = true;
      if (act && !dead) {
#pragma unroll
        for (int jj = 0; jj < J; ++jj) x[jj] = m[jj];
      } else {
        Q = Qold;
      }
    }
    float fm = x[0];
#pragma unroll
    for (int jj = 1; jj < J; ++jj) fm = fmaxf(fm, x[jj]);
    fm = group_max<G>(fm);
    if (has && r == 0) {
      float out;
      if (bad) {
        out = nan_f();
        if (err) set_status(a.status, err);
      } else if (Tn == 0) {
        out = 0.f;
      } else if (dead) {
        out = -INFINITY;
      } else {
        out = (float)((double)fm + (double)Q * (1.0 / kViterbiQuant));
      }
      a.score[ALL ? (size_t)s * span + kr : (size_t)s] = out;
      if (!ALL && a.best) a.best[s] = bad ? -1 : k;
    }

    if (ALL && a.best) {
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence();
        last = atomicAdd(a.done + g, 1) == span - 1;
      }
      last = __shfl_sync(HMM_FULL_MASK, last, 0);
      if (last) {
        __threadfence();
        if (has && r == 0) {
          const float* row = a.score + (size_t)s * span;
          float best = __ldcg(row);
          int arg = isnan(best) ? -1 : 0;
          for (int kk = 1; kk < span; ++kk) {
            const float v = __ldcg(row + kk);
            if (isnan(v)) arg = -1;
            else if (arg >= 0 && v > best) { best = v; arg = kk; }
          }
          a.best[s] = arg;
        }
      }
    }
  }
}

template <int J>
__device__ __forceinline__ uint32_t pack_bytes(const int (&arg)[J]) {
  uint32_t w = 0;
#pragma unroll
  for (int jj = 0; jj < J; ++jj) w |= (uint32_t)(arg[jj] & 0xff) << (8 * jj);
  return w;
}

template <int J>
__device__ __forceinline__ void store_bp(uint8_t* p, uint32_t w) {
  if constexpr (J == 1) *p = (uint8_t)w;
  else if constexpr (J == 2) *reinterpret_cast<uint16_t*>(p) = (uint16_t)w;
  else *reinterpret_cast<uint32_t*>(p) = w;
}

template <int J>
__device__ __forceinline__ uint32_t load_bp(const uint8_t* p) {
  if constexpr (J == 1) return __ldcg(p);
  else if constexpr (J == 2) return __ldcg(reinterpret_cast<const unsigned short*>(p));
  else return __ldcg(reinterpret_cast<const unsigned int*>(p));
}

template <int NP, int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
hmm_viterbi_paths(VitLaunch a) {
  constexpr int J = NP / G;
  static_assert(J <= 4, "backpointer words hold at most 4 states per lane");
  constexpr int PP = 32 / G;
  constexpr int XS = NP + 4;
  constexpr int CH = 32;  // backtrack rows fetched per chunk
  __shared__ __align__(16) float xs[kWarpsPerBlock][2][PP][XS];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / G, r = lane % G, j0 = r * J;
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;
  const int span = a.seq.span;
  const bool labelled = a.seq.model_of_seq != nullptr;
  const bool param_bad = (__ldcg(a.status) & HMM_STATUS_PARAM) != 0;

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue + 1, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_items_path) break;
    const int pos = item * PP + p;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    int k = 0;
    bool bad = T < 0 || param_bad;
    if (has && T >= 0) {
      if (labelled) {
        k = a.seq.model_of_seq[s];
        if (k < 0 || k >= K) { bad = true; k = 0; }
      } else {  // best model within the sequence's set
        k = __ldcg(a.best + s);
        if (k < 0 || k >= span) { bad = true; k = 0; }
        else if (a.seq.model_base) k += a.seq.model_base[s];
      }
    }
    const int Tn = (T < 0) ? 0 : T;
    const int Tmax = __reduce_max_sync(HMM_FULL_MASK, Tn);

    float2 a2[NP / 2][J];
    {
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP + j0;
#pragma unroll
      for (int i2 = 0; i2 < NP / 2; ++i2)
#pragma unroll
        for (int jj = 0; jj < J; ++jj)
          a2[i2][jj] = make_float2(__ldg(Ak + (2 * i2) * NP + jj), __ldg(Ak + (2 * i2 + 1) * NP + jj));
    }
    const float* Bk = a.mod.Btp + (size_t)k * M * NP + j0;
    const long long off = (has && T >= 0) ? a.seq.offsets[s] : 0;
    const int32_t* o = a.seq.symbols + off;
    uint8_t* bp = a.bp + ((has && T >= 0) ? a.bpoff[s] : 0) * (long long)NP + j0;

    float x[J];
    long long Q = 0;
    bool dead = false;
    int err = 0;
    {
      int o0 = Tn > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; o0 = 0; }
      float b[J], pv[J];
      load_vec<J>(b, Bk + (size_t)o0 * NP);
      load_vec<J>(pv, a.mod.pip + (size_t)k * NP + j0);
#pragma unroll
      for (int jj = 0; jj < J; ++jj) x[jj] = pv[jj] + b[jj];
      if (!normalise_max<J, G>(x, Q, Tn > 0 && !bad)) dead = true;
    }
    float bn[J];
    int on = 0;
    if (1 < Tn) {
      on = __ldg(o + 1);
      if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
    }
    load_vec<J>(bn, Bk + (size_t)on * NP);
    int o2 = (2 < Tn) ? __ldg(o + 2) : 0;

    for (int t = 1; t < Tmax; ++t) {
      const bool act = t < Tn && !dead && !bad;
      float* xb = &xs[warp][t & 1][p][0];
      store_vec<J>(xb + j0, x);
      __syncwarp();
      float m[J];
      int arg[J];
      maxarg_cols<NP, J>(xb, a2, m, arg);
      float b[J];
#pragma unroll
      for (int jj = 0; jj < J; ++jj) b[jj] = bn[jj];
      if (t + 1 < Tn) {
        on = o2;
        if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
        load_vec<J>(bn, Bk + (size_t)on * NP);
        if (t + 2 < Tn) o2 = __ldg(o + t + 2);
      }
#pragma unroll
      for (int jj = 0; jj < J; ++jj) m[jj] += b[jj];
      const long long Qold = Q;
      if (!normalise_max<J, G>(m, Q, act)) dead = true;
      if (act && !dead) {
        store_bp<J>(bp + (long long)t * NP, pack_bytes<J>(arg));
#pragma unroll
        for (int jj = 0; jj < J; ++jj) x[jj] = m[jj];
      } else {
        Q = Qold;
      }
    }

    // final state: smallest argmax of delta_T
    float fv = x[0];
    int fj = j0;
#pragma unroll
    for (int jj = 1; jj < J; ++jj)
      if (x[jj] > fv) { fv = x[jj]; fj = j0 + jj; }
    group_argmax<G>(fv, fj);

    if (has && r == 0) {
      float out;
      if (bad) {
        out = nan_f();
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

    // backtrack (warp-uniform loop over the longest pair of the warp)
    const bool walk = has && !bad && !dead && Tn > 0;
    int q = walk ? fj : 0;
    if (has && Tn > 0 && r == 0) a.path[off + Tn - 1] = bad ? -1 : q;
    for (int tc = Tmax - 1; tc >= 1; tc -= CH) {
      uint32_t rows[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = tc - u;
        rows[u] = (walk && t >= 1 && t <= Tn - 1) ? load_bp<J>(bp + (long long)t * NP) : 0u;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = tc - u;
        const int owner = q / J;
        const uint32_t byte = (rows[u] >> (8 * (q - owner * J))) & 0xffu;
        const int nq = __shfl_sync(HMM_FULL_MASK, (int)byte, p * G + owner);
        if (has && t >= 1 && t <= Tn - 1) {
          if (walk) q = nq;
          if (r == (t - 1) % G) a.path[off + t - 1] = bad ? -1 : (dead ? 0 : q);
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------
template <typename Kern>
static cudaError_t launch_persistent(Kern kern, int n_items, const VitLaunch& a, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int blocks = num_sms() * per_sm;
  const int need = (n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<blocks, kWarpsPerBlock * 32, 0, st>>>(a);
  return cudaGetLastError();
}

template <int NP, int G>
static cudaError_t launch_vs_t(const VitLaunch& a, cudaStream_t st) {
  const bool all = a.seq.model_of_seq == nullptr;
  if (all) return launch_persistent(hmm_viterbi_scores<NP, G, true>, a.n_items_score, a, st);
  return launch_persistent(hmm_viterbi_scores<NP, G, false>, a.n_items_score, a, st);
}

template <int NP, int G>
static cudaError_t launch_vp_t(const VitLaunch& a, cudaStream_t st) {
  return launch_persistent(hmm_viterbi_paths<NP, G>, a.n_items_path, a, st);
}

#define HMM_VS_CASE(NPV, GV) \
  if (NP == NPV && G == GV) return launch_vs_t<NPV, GV>(a, st);
#define HMM_VP_CASE(NPV, GV) \
  if (NP == NPV && G == GV) return launch_vp_t<NPV, GV>(a, st);

cudaError_t launch_viterbi_scores(int NP, int G, const VitLaunch& a, cudaStream_t st) {
  HMM_VS_CASE(4, 1) HMM_VS_CASE(4, 2) HMM_VS_CASE(4, 4)
  HMM_VS_CASE(8, 1) HMM_VS_CASE(8, 2) HMM_VS_CASE(8, 4) HMM_VS_CASE(8, 8)
  HMM_VS_CASE(16, 2) HMM_VS_CASE(16, 4) HMM_VS_CASE(16, 8) HMM_VS_CASE(16, 16)
  HMM_VS_CASE(32, 8) HMM_VS_CASE(32, 16) HMM_VS_CASE(32, 32)
  HMM_VS_CASE(64, 32)
  return cudaErrorInvalidValue;
}

cudaError_t launch_viterbi_paths(int NP, int G, const VitLaunch& a, cudaStream_t st) {
  HMM_VP_CASE(4, 1) HMM_VP_CASE(4, 2) HMM_VP_CASE(4, 4)
  HMM_VP_CASE(8, 2) HMM_VP_CASE(8, 4) HMM_VP_CASE(8, 8)
  HMM_VP_CASE(16, 4) HMM_VP_CASE(16, 8) HMM_VP_CASE(16, 16)
  HMM_VP_CASE(32, 8) HMM_VP_CASE(32, 16) HMM_VP_CASE(32, 32)
  HMM_VP_CASE(64, 32)
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
