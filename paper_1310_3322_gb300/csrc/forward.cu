// forward.cu -- scaled forward algorithm, FP32 SIMT (Sec. 2.7 "Forward";
// Rabiner 1989 eqs. 19-21 with per-step rescaling, Sec. V-A).
//
// Work decomposition (persistent kernel):
//   * a "pair" is one (sequence, model); G lanes of a warp cooperate on it,
//     lane r owning the J = NP/G states [rJ, rJ+J);
//   * a warp holds P = 32/G pairs: P consecutive sequences of the
//     length-sorted order, all against one model (all-models mode: work item
//     = (group of P sequences, model k), K items per group) or each against its
//     own model (labelled mode);
//   * warps take items from an atomic queue in order of decreasing length, so
//     the long sequences start first and the tail is short.
//
// Per step t (all arithmetic FP32, packed FP32x2 where it pairs up):
//   1. each lane publishes its J values of alpha_{t-1} to a per-pair
//      shared-memory row (double-buffered, one __syncwarp);
//   2. abar(j) = sum_i alpha_{t-1}(i) a_ij for its J columns: NP/4 broadcast
//      float4 loads of alpha, 2 packed FMAs each, with column j of A held in
//      registers as (a_{2i,j}, a_{2i+1,j}) pairs;
//   3. abar(j) *= b_j(o_t) (row o_t of the symbol-major emission table, one
//      vector load, prefetched a step ahead);
//   4. the group sums abar (log2 G shuffles) and rescales by an exact power of
//      two so the sum lies in [1,2); the removed exponent is added to an
//      integer. log P = ln(sum_j alpha_T(j)) + E ln 2 is formed in FP64 once.
// Recognition (Sec. 3 item 3): the last warp to finish a group's K items
// takes the argmax over models for its sequences.
#include "hmm_internal.cuh"

namespace hmmgb {

template <int NP, int G, bool ALL, int NV = NP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
hmm_forward_simt(FwdLaunch a) {
  constexpr int J = NP / G;
  constexpr int PP = 32 / G;
  constexpr int XS = NP + 4;  // padded row: conflict-free broadcast reads
  __shared__ __align__(16) float xs[kWarpsPerBlock][2][PP][XS];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / G, r = lane % G, j0 = r * J;
  const int M = a.seq.M, S = a.seq.S;
  const int span = a.seq.span;  // models per sequence in all-models mode

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_items) break;
    const int g = ALL ? item / span : item;
    const int kr = ALL ? item % span : 0;  // model index within the sequence's set
    int k = kr;
    const int pos = g * PP + p;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    int T = has ? a.seq.seqlen[s] : 0;
    if (!ALL && has && T >= 0) k = a.seq.model_of_seq[s];
    if (ALL && has && T >= 0 && a.seq.model_base) k += a.seq.model_base[s];
    const bool bad_seq = T < 0;
    const int Tn = bad_seq ? 0 : T;
    const int Tmax = __reduce_max_sync(HMM_FULL_MASK, Tn);

    // column slice of A for this pair's model, packed over pairs of rows
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
    int E = 0;
    bool dead = false, bad = bad_seq;
    int err = 0;  // HMM_STATUS_* bits found by this pair
    if (Tn > 0) {
      int o0 = __ldg(o);
      if ((unsigned)o0 >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; o0 = 0; }
      float b[J], pv[J];
      load_vec<J>(b, Bk + (size_t)o0 * NP);
      load_vec<J>(pv, a.mod.pip + (size_t)k * NP + j0);
#pragma unroll
      for (int jj = 0; jj < J; ++jj) x[jj] = pv[jj] * b[jj];
    } else {
#pragma unroll
      for (int jj = 0; jj < J; ++jj) x[jj] = 0.f;
    }
    {
      const float gs = group_sum<G>(tree_sum<J>(x));
      if (Tn > 0 && !bad) {
        if (gs == 0.f) dead = true;
        else if (!(gs > 0.f) || isinf(gs)) { bad = true; err |= HMM_STATUS_PARAM; }
        else E += rescale_pow2<J>(x, gs);
      }
    }

    // emission row for step 1 and the symbol of step 2, prefetched: the
    // symbol load of step t+2 and the emission-row load of step t+1 are both
    // issued a full step before their values are needed
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
      float nx[J];
      matvec_cols<NP, J, NV>(xb, a2, nx);
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
      for (int jj = 0; jj < J; ++jj) nx[jj] *= b[jj];
      const float gs = group_sum<G>(tree_sum<J>(nx));
      if (act) {
        if (gs == 0.f) {
          dead = true;
        } else if (!(gs > 0.f) || isinf(gs)) {
          bad = true;
          err |= HMM_STATUS_PARAM;
        } else {
          E += rescale_pow2<J>(nx, gs);
#pragma unroll
          for (int jj = 0; jj < J; ++jj) x[jj] = nx[jj];
        }
      }
    }
    // (bad, dead and E are uniform across the lanes of a pair: every lane
    // reads the same symbols and the butterfly sums agree bitwise)
    const float fs = group_sum<G>(tree_sum<J>(x));
    if (has && r == 0) {
      float out;
      if (bad) {
        out = __int_as_float(0x7fc00000);
        if (err) set_status(a.status, err);
      } else if (Tn == 0) {
        out = 0.f;
      } else if (dead) {
        out = -INFINITY;
      } else {
        out = (float)(log((double)fs) + (double)E * 0.69314718055994530942);
      }
      a.loglik[ALL ? (size_t)s * span + kr : (size_t)s] = out;
    }

    if (ALL && a.argmax) {
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
          const float* row = a.loglik + (size_t)s * span;
          float best = __ldcg(row);
          int arg = isnan(best) ? -1 : 0;
          for (int kk = 1; kk < span; ++kk) {
            const float v = __ldcg(row + kk);
            if (isnan(v)) arg = -1;
            else if (arg >= 0 && v > best) { best = v; arg = kk; }
          }
          a.argmax[s] = arg;
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------
template <int NP, int G>
static cudaError_t launch_fwd_t(const FwdLaunch& a, cudaStream_t st) {
  const bool all = a.seq.model_of_seq == nullptr;
  auto kern = all ? hmm_forward_simt<NP, G, true> : hmm_forward_simt<NP, G, false>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  const int items_per_block = kWarpsPerBlock;
  int blocks = num_sms() * per_sm;
  const int need = (a.n_items + items_per_block - 1) / items_per_block;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<blocks, kWarpsPerBlock * 32, 0, st>>>(a);
  return cudaGetLastError();
}

#define HMM_FWD_CASE(NPV, GV) \
  if (NP == NPV && G == GV) return launch_fwd_t<NPV, GV>(a, st);

cudaError_t launch_forward(int NP, int G, const FwdLaunch& a, cudaStream_t st) {
  HMM_FWD_CASE(4, 1) HMM_FWD_CASE(4, 2) HMM_FWD_CASE(4, 4)
  HMM_FWD_CASE(8, 1) HMM_FWD_CASE(8, 2) HMM_FWD_CASE(8, 4) HMM_FWD_CASE(8, 8)
  HMM_FWD_CASE(16, 2) HMM_FWD_CASE(16, 4) HMM_FWD_CASE(16, 8) HMM_FWD_CASE(16, 16)
  HMM_FWD_CASE(32, 8) HMM_FWD_CASE(32, 16) HMM_FWD_CASE(32, 32)
  HMM_FWD_CASE(64, 32)
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
