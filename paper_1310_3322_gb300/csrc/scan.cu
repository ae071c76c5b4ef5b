// scan.cu -- parallel-in-time forward for few, very long sequences (FP32 SIMT).
//
// The forward recursion alpha_t = (alpha_{t-1} A) o b(o_t) (Rabiner eqs.
// 19-20) is a product of per-step matrices M_t = A diag(b(o_t)):
//   alpha_{T-1} = alpha_0 M_1 M_2 ... M_{T-1},  alpha_0 = pi o b(o_0),
// and log P(O | lambda) = log sum_j alpha_{T-1}(j) (eq. 21). Matrix products
// associate, so the steps of one sequence split into chunks of L steps whose
// products P_c = M_{t0} ... M_{t0+L-1} are independent work items:
//
//   * hmm_scan_chunks: one work item per (pair, chunk). Row i of P_c is the
//     forward recursion started from the unit vector e_i, so NP lanes hold
//     the NP rows (lane i <-> start state i) and step together, reading A from
//     shared memory and the emission row b(o_t) from the L1-cached table.
//     Each row keeps its own power-of-two exponent (max entry in [1, 2)), so
//     rows of very different magnitude keep full precision.
//   * hmm_scan_combine: one sub-warp per pair walks its chunks in order,
//     v <- v P_c, with the next chunk's product loaded while the current one
//     is applied: sum_i v_i 2^{E_c[i]} Phat_c[i][:] is evaluated against the
//     largest term's exponent, the result renormalised by a power of two.
//
// Work: NP^3 FMAs per step in the chunk products (the sequential recursion
// does NP^2), so this pays only when a batch has too few pairs to fill the
// GPU and the sequential chain of T steps sets the time. The chain becomes
// L steps + T / L chunk combines.
#include "hmm_internal.cuh"

namespace hmmgb {

// v = m * 2^e with m in [1, 2), for finite v > 0 (subnormals included).
__device__ __forceinline__ float split_pow2(float v, int& e) {
  int shift = 0;
  if (v < 0x1p-120f) {
    v *= 0x1p64f;
    shift = -64;
  }
  const int f = frexp2(v);
  e = f + shift;
  return v * exp2i(-f);
}

// y * 2^-e, exact for the e that split_pow2 returns on the largest |y| of a
// vector (e in [-149, 127]).
__device__ __forceinline__ float pow2_scale(float y, int e) {
  if (e > 120) return (y * 0x1p-64f) * exp2i(64 - e);
  if (e >= -120) return y * exp2i(-e);
  return (y * 0x1p64f) * exp2i(-e - 64);
}

// m * 2^d for m in [1, 2) and d <= 0 (0 once the value is below the
// subnormal range).
__device__ __forceinline__ float scale_down(float m, int d) {
  if (d >= -126) return m * exp2i(d);
  if (d >= -190) return (m * exp2i(d + 64)) * 0x1p-64f;
  return 0.f;
}

template <int NP>
__device__ __forceinline__ int group_max_int(int v) {
#pragma unroll
  for (int o = NP / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(HMM_FULL_MASK, v, o));
  return v;
}

template <int NP>
__device__ __forceinline__ int group_or(int v) {
#pragma unroll
  for (int o = NP / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(HMM_FULL_MASK, v, o);
  return v;
}

// Largest s in [0, S) with coff[s] <= g (coff non-decreasing, coff[0] = 0).
__device__ __forceinline__ int seq_of_chunk(const int64_t* coff, int S, int64_t g) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(coff + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// --------------------------------------------------------------------------
// chunk products
// --------------------------------------------------------------------------
// R rows of one chunk item per lane (lanes li and rows li, li + NP / R, ...):
// every A value read from shared memory feeds R * 4 FMAs, and the warp's
// 32 / (NP / R) items read distinct, bank-disjoint copies of A.
template <int NP, int R>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
hmm_scan_chunks(ScanLaunch a) {
  constexpr int LPI = NP / R;        // lanes per chunk item
  constexpr int RPW = 32 / LPI;      // chunk items per warp
  constexpr int AS = NP * NP + 4;    // per-item A stride (floats): items on different banks
  __shared__ __align__(16) float As[kWarpsPerBlock][RPW][AS];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LPI, li = lane % LPI;
  const int S = a.seq.S, M = a.seq.M;
  const bool all = a.seq.model_of_seq == nullptr;
  const int64_t CT = __ldcg(a.coff + S);  // chunks of all sequences (written by setup)
  const int64_t n_chunks = CT * (all ? a.seq.span : 1);
  float* Asub = &As[warp][sub][0];

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if ((int64_t)item * RPW >= n_chunks) break;
    const int64_t f = (int64_t)item * RPW + sub;
    const bool has = f < n_chunks;

    int kk = 0, s = 0, T = 0, k = 0;
    int64_t g = 0;
    if (has) {
      kk = all ? (int)(f / CT) : 0;
      g = all ? f % CT : f;
      s = seq_of_chunk(a.coff, S, g);
      T = a.seq.seqlen[s];
      if (T >= 0) {  // a rejected sequence (T = -1) keeps k = 0 and runs no step
        if (all) k = kk + (a.seq.model_base ? a.seq.model_base[s] : 0);
        else k = a.seq.model_of_seq[s];
      }
    }
    const int c = has ? (int)(g - __ldg(a.coff + s)) : 0;
    const int t0 = 1 + c * a.L;
    const int t1 = has ? min(T, t0 + a.L) : t0;
    const int nT = t1 - t0;  // >= 1 for every real chunk
    const int nTmax = __reduce_max_sync(HMM_FULL_MASK, nT);

    // A of this item's model, rows li + r LPI loaded by lane li
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = li + r * LPI;
      float row[NP];
      load_vec<NP>(row, a.mod.Ap + ((size_t)k * NP + i) * NP);
#pragma unroll
      for (int q = 0; q < NP / 4; ++q)
        *reinterpret_cast<float4*>(Asub + i * NP + 4 * q) =
            make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
    }
    __syncwarp();

    const float* Bk = a.mod.Btp + (size_t)k * M * NP;
    const int32_t* o = a.seq.symbols + (has ? a.seq.offsets[s] : 0);
    float x[R][NP];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < NP; ++j) x[r][j] = (j == li + r * LPI) ? 1.f : 0.f;
    int E[R];
    bool dead[R], perr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { E[r] = 0; dead[r] = false; perr[r] = false; }
    bool bad = false;  // an invalid symbol (the same for every row of the item)

    // emission row of the first step, symbol of the second
    int on = nT > 0 ? __ldg(o + t0) : 0;
    bool serr = false;
    if ((unsigned)on >= (unsigned)M) { bad = serr = true; on = 0; }
    float bn[NP];
    load_vec<NP>(bn, Bk + (size_t)on * NP);
    int o2 = nT > 1 ? __ldg(o + t0 + 1) : 0;

    for (int u = 0; u < nTmax; ++u) {
      const bool act = u < nT && !bad;
      float b[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) b[j] = bn[j];
      if (u + 1 < nT) {
        on = o2;
        if ((unsigned)on >= (unsigned)M) { bad = serr = true; on = 0; }
        load_vec<NP>(bn, Bk + (size_t)on * NP);
        if (u + 2 < nT) o2 = __ldg(o + t0 + u + 2);
      }
      // y = x A: packed FMAs over pairs of columns, each A row of shared
      // memory applied to the R rows
      float2 acc[R][NP / 2];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) acc[r][q] = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < NP; ++l) {
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) {
          const float4 av = *reinterpret_cast<const float4*>(Asub + l * NP + 4 * q);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 xl = make_float2(x[r][l], x[r][l]);
            acc[r][2 * q] = ffma2(xl, make_float2(av.x, av.y), acc[r][2 * q]);
            acc[r][2 * q + 1] = ffma2(xl, make_float2(av.z, av.w), acc[r][2 * q + 1]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float y[NP];
#pragma unroll
        for (int q = 0; q < NP / 2; ++q) {
          y[2 * q] = acc[r][q].x * b[2 * q];
          y[2 * q + 1] = acc[r][q].y * b[2 * q + 1];
        }
        const float m = tree_max<NP>(y);
        if (act && !dead[r] && !perr[r]) {
          if (!(m < INFINITY)) {  // finite parameters whose product overflows
            perr[r] = true;
          } else if (m > 0.f) {
            int e;
            split_pow2(m, e);
#pragma unroll
            for (int j = 0; j < NP; ++j) x[r][j] = pow2_scale(y[j], e);
            E[r] += e;
          } else {
            dead[r] = true;  // this start state cannot produce the chunk
#pragma unroll
            for (int j = 0; j < NP; ++j) x[r][j] = 0.f;
          }
        }
      }
    }

    if (has) {
      const int64_t slot = (int64_t)kk * a.cap + g;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = li + r * LPI;
        store_vec<NP>(a.P + (slot * NP + i) * NP, x[r]);
        a.E[slot * NP + i] = (bad || perr[r]) ? kScanBad : (dead[r] ? kScanDead : E[r]);
        if (perr[r]) set_status(a.status, HMM_STATUS_PARAM);
      }
      if (serr && li == 0) set_status(a.status, HMM_STATUS_SYMBOL);
    }
  }
}

// --------------------------------------------------------------------------
// combine along each pair's chunks
// --------------------------------------------------------------------------
template <int NP, bool ALL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
hmm_scan_combine(ScanLaunch a) {
  constexpr int RPW = 32 / NP;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NP, j = lane % NP;
  const int S = a.seq.S, M = a.seq.M;
  const int span = ALL ? a.seq.span : 1;
  const bool param_bad = (__ldcg(a.status) & HMM_STATUS_PARAM) != 0;

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue + 1, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_pair_items) break;
    const int q = item * RPW + sub;
    const bool has = q < S * span;
    const int pos = has ? q / span : 0;
    const int kk = has ? q % span : 0;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    const bool bad_seq = T < 0;
    const int Tn = bad_seq ? 0 : T;
    int k = kk;
    if (has && !bad_seq) {
      if (!ALL) k = a.seq.model_of_seq[s];
      else if (a.seq.model_base) k += a.seq.model_base[s];
    }
    const int64_t c0 = (has && !bad_seq) ? __ldg(a.coff + s) : 0;
    const int nC = (has && !bad_seq) ? (int)(__ldg(a.coff + s + 1) - c0) : 0;
    const int nCmax = __reduce_max_sync(HMM_FULL_MASK, nC);
    const int64_t slot0 = (int64_t)kk * a.cap + c0;

    // alpha_0 = pi o b(o_0), normalised so that its largest entry is in [1, 2)
    int bad = bad_seq ? 1 : 0;
    int o0 = Tn > 0 ? __ldg(a.seq.symbols + a.seq.offsets[s]) : 0;
    const bool serr = (unsigned)o0 >= (unsigned)M;
    if (serr) { bad = 1; o0 = 0; }
    float v = __ldg(a.mod.pip + (size_t)k * NP + j) * __ldg(a.mod.Btp + ((size_t)k * M + o0) * NP + j);
    long long Ev = 0;
    bool dead = false;
    {
      const float m = group_max<NP>(v);
      if (!(m < INFINITY)) {
        bad = 1;
      } else if (m > 0.f) {
        int e;
        split_pow2(m, e);
        v = pow2_scale(v, e);
        Ev = e;
      } else {
        dead = true;
      }
    }

    // chunk c's column j (rows i) and row j's exponent, one chunk ahead
    float pn[NP];
    int en = 0;
    if (nC > 0) {
      const float* P = a.P + slot0 * NP * NP + j;
#pragma unroll
      for (int r = 0; r < NP; ++r) pn[r] = __ldg(P + r * NP);
      en = __ldg(a.E + slot0 * NP + j);
    }
    for (int c = 0; c < nCmax; ++c) {
      const bool act = c < nC;
      float p[NP];
#pragma unroll
      for (int r = 0; r < NP; ++r) p[r] = pn[r];
      const int ec = en;
      if (c + 1 < nC) {
        const float* P = a.P + (slot0 + c + 1) * NP * NP + j;
#pragma unroll
        for (int r = 0; r < NP; ++r) pn[r] = __ldg(P + r * NP);
        en = __ldg(a.E + (slot0 + c + 1) * NP + j);
      }
      if (act && ec == kScanBad) bad = 1;
      // lane j holds v_j and row j's exponent: weights against the largest term
      const bool live = act && !dead && v > 0.f && ec != kScanDead && ec != kScanBad;
      int ev = 0;
      const float mv = live ? split_pow2(v, ev) : 0.f;
      const int key = live ? ec + ev : INT_MIN;
      const int kmax = group_max_int<NP>(key);
      const float w = live ? scale_down(mv, key - kmax) : 0.f;
      float y = 0.f;
#pragma unroll
      for (int r = 0; r < NP; ++r) y = fmaf(__shfl_sync(HMM_FULL_MASK, w, sub * NP + r), p[r], y);
      // every lane takes part in the shuffles; only the branch below diverges
      const float m = group_max<NP>(y);
      if (act && !dead) {
        if (kmax == INT_MIN) {
          dead = true;
        } else if (!(m < INFINITY)) {
          bad = 1;
        } else if (m > 0.f) {
          int e;
          split_pow2(m, e);
          v = pow2_scale(y, e);
          Ev += (long long)kmax + e;
        } else {
          dead = true;
        }
      }
    }
    bad = group_or<NP>(bad);
    const float sum = group_sum<NP>(dead ? 0.f : v);

    if (has && j == 0) {
      float out;
      if (serr) set_status(a.status, HMM_STATUS_SYMBOL);
      if (bad || param_bad) {
        out = __int_as_float(0x7fc00000);
      } else if (Tn == 0) {
        out = 0.f;
      } else if (dead) {
        out = -INFINITY;
      } else {
        out = (float)(log((double)sum) + (double)Ev * 0.69314718055994530942);
      }
      a.loglik[ALL ? (size_t)s * span + kk : (size_t)s] = out;
      if (ALL && a.argmax) {
        __threadfence();
        if (atomicAdd(a.done + pos, 1) == span - 1) {
          __threadfence();
          const float* row = a.loglik + (size_t)s * span;
          float best = __ldcg(row);
          int arg = isnan(best) ? -1 : 0;
          for (int m2 = 1; m2 < span; ++m2) {
            const float vv = __ldcg(row + m2);
            if (isnan(vv)) arg = -1;
            else if (arg >= 0 && vv > best) { best = vv; arg = m2; }
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
template <typename Kern>
static cudaError_t launch_fill(Kern kern, int64_t need_warps, cudaStream_t st, const ScanLaunch& a) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)num_sms() * per_sm;
  const int64_t need = (need_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<(int)blocks, kWarpsPerBlock * 32, 0, st>>>(a);
  return cudaGetLastError();
}

// rows per lane of the chunk products: two from 8 states up (fewer shared
// loads per FMA; at 4 states eight items already share each warp)
template <int NP>
constexpr int scan_rows() { return NP >= 8 ? 2 : 1; }

template <int NP>
static cudaError_t launch_scan_t(const ScanLaunch& a, int64_t max_chunks, cudaStream_t st,
                                 int phase) {
  constexpr int R = scan_rows<NP>();
  constexpr int RPW = 32 / (NP / R);
  if (phase == 0)
    return launch_fill(hmm_scan_chunks<NP, R>, (max_chunks + RPW - 1) / RPW, st, a);
  if (a.seq.model_of_seq == nullptr)
    return launch_fill(hmm_scan_combine<NP, true>, a.n_pair_items, st, a);
  return launch_fill(hmm_scan_combine<NP, false>, a.n_pair_items, st, a);
}

cudaError_t launch_scan(int NP, const ScanLaunch& a, int64_t max_chunks, int phase,
                        cudaStream_t st) {
  switch (NP) {
    case 4: return launch_scan_t<4>(a, max_chunks, st, phase);
    case 8: return launch_scan_t<8>(a, max_chunks, st, phase);
    case 16: return launch_scan_t<16>(a, max_chunks, st, phase);
    case 32: return launch_scan_t<32>(a, max_chunks, st, phase);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hmmgb
