// mma_forward.cu -- scaled forward algorithm on the tensor cores for N = 64 or
// 128 states (Sec. 2.7 "Forward"; Rabiner 1989 eqs. 19-21, per-step scaling).
//
// At these state counts the step  abar_t = alpha_{t-1} A  is a real dense
// contraction when 128 (sequence, model) pairs of one model are stacked:
//   D[128 x N] = X[128 x N] . A[N x N]
// tcgen05.mma (cta_group::1, kind::f16, M = 128, N = NP, K = 16 per
// instruction) with
//   * X, the BF16 rescaled alpha rows, in tensor memory (A operand: lane =
//     row, two BF16 per 32-bit column), written by the epilogue with
//     tcgen05.st -- no shared-memory traffic for X at all;
//   * A^T in BF16 in shared memory (B operand, K-major, no swizzle);
//   * D in FP32 in tensor memory.
// The epilogue gives every row TPR threads (warps w, w+4, ... of a tile's
// group see the same 32 tensor-memory lanes); each streams its share of the
// row's D columns through registers 32 at a time: multiply by the emission
// row b(o_t) in FP32, scale by an exact power of two, accumulate a partial row
// sum, pack to BF16 and store its share of the next X row.
//
// Emission rows: when the model's whole emission table (M rows of NP FP32
// values, rows padded by 16 bytes) fits in shared memory next to A^T, it is
// loaded there once per model and each row reads b(o_t) straight from it, with
// the symbols themselves loaded two steps ahead -- no global-memory round trip
// remains on a step's critical path. Otherwise each row's b(o_{t+1}) is
// brought into that row's slot of a shared-memory staging tile by one bulk
// (TMA-engine) copy, issued as soon as the row has read b(o_t) and completing
// on an mbarrier while the next MMA runs.
//
// Scaling is one step late so no thread waits for a full row sum inside a
// step: step t scales by 2^-f_t with f_t the exponent of the previous row sum
// sigma_{t-1} (clamped to the float range; a clamped step is caught up by the
// next one), the two partial sums meet in shared memory behind the barrier
// that precedes the next MMA, sums stay near the per-step likelihood ratio,
// and
//   log P = ln sigma_{T-1} + (sum_t f_t) ln 2
// with the exponents summed exactly in an integer.
//
// A CTA of 512 threads owns NT 128-row tiles of the same model (NT = 2 with two
// threads per row at N = 128, where tensor memory holds two tiles; NT = 4 with
// one thread per row at N = 64): while one tile's MMA runs, the others run
// their epilogues. Work items are (group of NT tiles, model), taken
// longest-first from an atomic queue over the length-sorted sequence order.
// Every mbarrier wait is bounded; on timeout the kernel records
// HMM_STATUS_TIMEOUT and leaves.
#include "hmm_internal.cuh"
#include "mma_rows.cuh"
#include "tc.cuh"

namespace hmmgb {

constexpr uint32_t kWaitLimit = 1u << 24;  // polls of the teardown's drain waits
constexpr uint32_t kTmemCols = 512;  // per tile: D (NP cols) then X (NP/2 cols) at (512/NT) * tile
constexpr int kMmaThreads = 512;

template <int NP, int NT, int TPR, int AB, bool EMIS>
__global__ void __launch_bounds__(kMmaThreads, 1) hmm_forward_mma(MmaFwdLaunch a) {
  using L = MmaFwdSmem<NP, NT, TPR, AB, EMIS>;
  constexpr int XC = AB == 1 ? NP / 2 : NP;   // tensor-memory columns of X
  constexpr int KI = AB == 1 ? 16 : 8;        // K per instruction
  constexpr int WGT = 128 * TPR;     // threads per tile
  static_assert(NT * WGT == kMmaThreads, "512 threads per CTA");
  constexpr int HALF = NP / TPR;     // columns per thread
  constexpr int CH = HALF / 32;      // 32-column chunks per thread
  constexpr int TS = 512 / NT;       // tensor-memory columns per tile
  static_assert(NP + XC <= TS, "tile does not fit its tensor-memory share");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem + L::OFF_B;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);

  const int tid = threadIdx.x, wg = tid / WGT, wtid = tid % WGT;
  const int warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = (wtid >> 7);   // lane quarter, column share
  const int row = wq * 32 + lane;
  // staging slot of this row (EMIS: the table's base)
  const uint8_t* erow = smem + L::OFF_E + (EMIS ? 0 : wg * L::kE + row * L::kES);
  const uint32_t eslot = tc::smem_u32(erow);
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS) + wg * TPR * 128;  // [TPR][128]
  uint64_t* mbar = &bars[wg];
  uint64_t* ebar = &bars[NT + wg];
  uint64_t* fbar = &bars[2 * NT + wg];  // teardown: every MMA of this warpgroup done
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;

  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), kTmemCols);
  if (tid == 0) {
    for (int i = 0; i < NT; ++i) {
      tc::mbar_init(&bars[i], 1);
      tc::mbar_init(&bars[NT + i], 128);
      tc::mbar_init(&bars[2 * NT + i], 1);
    }
    misc[2] = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t d_tmem = tmem + (uint32_t)(wg * TS);           // D: NP FP32 columns
  const uint32_t x_tmem = d_tmem + (uint32_t)NP;                // X: XC columns
  const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
  const uint32_t d_mine = d_tmem + lane_off + (uint32_t)(h * HALF);
  const uint32_t x_mine = x_tmem + lane_off + (uint32_t)(h * HALF * XC / NP);
  constexpr uint32_t idesc = tc::instr_desc(AB, 128, NP);
  const uint32_t b_base = tc::smem_u32(sB);
  constexpr uint32_t SBO = AB == 1 ? NP * 16 : NP * 32;  // next 8 rows of the B image
  uint32_t mphase = 0, ephase = 0;
  int cur_model = -1;

  for (;;) {
    __syncthreads();
    if (tid == 0) misc[1] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = misc[1];
    if (item >= a.n_items || misc[2]) break;
    const int tp = item / K, k = item % K;

    if (k != cur_model) {
      // B operand: element (n = j, k = i) = a_ij, K-major core matrices of 8
      // rows x 16 bytes (8 BF16 or 4 TF32 values of i)
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
      if constexpr (AB == 1) {
        for (int idx = tid; idx < NP * NP / 2; idx += kMmaThreads) {
          const int j = idx / (NP / 2), i = (idx % (NP / 2)) * 2;
          const uint32_t w = tc::pack_bf16(__ldg(Ak + i * NP + j), __ldg(Ak + (i + 1) * NP + j));
          const uint32_t off = (j / 8) * SBO + (i / 8) * 128 + (j % 8) * 16 + (i % 8) * 2;
          *reinterpret_cast<uint32_t*>(sB + off) = w;
        }
      } else {
        for (int idx = tid; idx < NP * NP; idx += kMmaThreads) {
          const int j = idx / NP, i = idx % NP;
          const uint32_t off = (j / 8) * SBO + (i / 4) * 128 + (j % 8) * 16 + (i % 4) * 4;
          *reinterpret_cast<uint32_t*>(sB + off) = tc::to_tf32(__ldg(Ak + i * NP + j));
        }
      }
      if constexpr (EMIS)  // the model's emission table, rows padded to kET bytes
        fill_emission_table<NP, AB, L::kET>(smem + L::OFF_E, a.mod.Btp + (size_t)k * M * NP, M, tid,
                                            kMmaThreads);
      cur_model = k;
      tc::fence_proxy_async();
      __syncthreads();
    }

    const int tile = NT * tp + wg;
    const int pos = tile * 128 + row;
    const bool has = tile < a.n_tiles && pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    const bool bad_seq = T < 0;
    const int Tn = bad_seq ? 0 : T;
    {
      const int wm = __reduce_max_sync(HMM_FULL_MASK, Tn);
      if (lane == 0) misc[4 + warp] = wm;
    }
    tc::bar_sync(1 + wg, WGT);
    int Tmax = 0;
#pragma unroll
    for (int w8 = 0; w8 < WGT / 32; ++w8) Tmax = max(Tmax, (int)misc[4 + (WGT / 32) * wg + w8]);

    const float* Bk = a.mod.Btp + (size_t)k * M * NP;
    const int32_t* o = a.seq.symbols + (has && !bad_seq ? a.seq.offsets[s] : 0);
    RowState st;
    st.F = 0; st.f = 0; st.dead = false; st.bad = bad_seq; st.written = (Tn == 0);
    st.err = 0; st.ll = 0.f;

    // t = 0: x_0 = pi . b(o_0), no scaling
    {
      int o0 = Tn > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; o0 = 0; }
      const bool live = Tn > 0 && !st.bad;
      const float4* b4 = reinterpret_cast<const float4*>(Bk + (size_t)o0 * NP + h * HALF);
      const float4* p4 = reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * NP + h * HALF);
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        float y[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 bb = __ldg(b4 + 8 * c + q), pp = __ldg(p4 + 8 * c + q);
          y[4 * q] = live ? pp.x * bb.x : 0.f; y[4 * q + 1] = live ? pp.y * bb.y : 0.f;
          y[4 * q + 2] = live ? pp.z * bb.z : 0.f; y[4 * q + 3] = live ? pp.w * bb.w : 0.f;
        }
        part += tree_sum<32>(y);
        store_x<AB>(x_mine, c, y);
      }
      tc::tmem_st_wait();
      psum[h * 128 + row] = part;
    }
    int o_next = (1 < Tn) ? __ldg(o + 1) : 0;
    int o_next2 = (EMIS && 2 < Tn) ? __ldg(o + 2) : 0;  // EMIS: symbols two steps ahead
    if constexpr (!EMIS) {
      if (Tmax > 1 && h == 0)
        stage_emission<NP>(eslot, Bk, (1 < Tn && (unsigned)o_next < (unsigned)M) ? o_next : 0, ebar);
    }

    bool aborted = false;
    for (int t = 1; t < Tmax; ++t) {
      tc::fence_before_sync();
      tc::bar_sync(1 + wg, WGT);
      if (wtid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < NP / KI; ++ks) {  // 8 tensor-memory columns of X per instruction
          if constexpr (AB == 1)
            tc::mma_bf16_ts(d_tmem, x_tmem + (uint32_t)(ks * 8),
                            tc::smem_desc(b_base + ks * 256, 128, SBO), idesc, ks > 0 ? 1u : 0u);
          else
            tc::mma_tf32_ts(d_tmem, x_tmem + (uint32_t)(ks * 8),
                            tc::smem_desc(b_base + ks * 256, 128, SBO), idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(mbar);
      }
      close_step(st, TPR == 2 ? psum[row] + psum[128 + row] : psum[row], t - 1, Tn);
      const int ot = o_next;
      if constexpr (EMIS) {
        o_next = o_next2;
        if (t + 2 < Tn) o_next2 = __ldg(o + t + 2);
      } else {
        if (t + 1 < Tn) o_next = __ldg(o + t + 1);
      }
      if (t < Tn && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
      const uint8_t* eb = EMIS ? erow + ((unsigned)ot < (unsigned)M ? ot : 0) * L::kET : erow;
      const bool live = t < Tn && !st.dead && !st.bad;
      if (live) st.F += st.f;
      const float2 fac2 = make_float2(exp2i(-st.f), exp2i(-st.f));
      // one warp polls both mbarriers; the rest of the warpgroup waits in the
      // hardware barrier (no issue slots spent spinning)
      bool ok = true;
      if (wtid < 32) {
        if constexpr (!EMIS) ok = tc::mbar_wait_bounded(ebar, ephase, a.wait_limit);
        ok = tc::mbar_wait_bounded(mbar, mphase, a.wait_limit) && ok;
      }
      if constexpr (!EMIS) ephase ^= 1;
      mphase ^= 1;
      // the whole warpgroup agrees before anyone leaves the loop (and every
      // thread has read the partial sums before they are overwritten)
      if (!tc::bar_and(1 + wg, WGT, ok)) {
        aborted = true;
        break;
      }
      tc::fence_after_sync();
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        float y[32];
        tc::tmem_ld32(d_mine + (uint32_t)(c * 32), y);
        tc::tmem_ld_wait();
        float2 acc = make_float2(0.f, 0.f);
        float be[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 b;
          if constexpr (EMIS) {
            if ((q & 1) == 0) emission8<AB>(eb, h * HALF + 32 * c + 4 * q, be);
            b = make_float4(be[4 * (q & 1)], be[4 * (q & 1) + 1], be[4 * (q & 1) + 2],
                            be[4 * (q & 1) + 3]);
          } else {
            b = *reinterpret_cast<const float4*>(eb + (h * HALF + 32 * c + 4 * q) * 4);
          }
          float2 lo = __fmul2_rn(__fmul2_rn(make_float2(y[4 * q], y[4 * q + 1]),
                                            make_float2(b.x, b.y)), fac2);
          float2 hi = __fmul2_rn(__fmul2_rn(make_float2(y[4 * q + 2], y[4 * q + 3]),
                                            make_float2(b.z, b.w)), fac2);
          if (!live) { lo = make_float2(0.f, 0.f); hi = lo; }
          acc = __fadd2_rn(acc, __fadd2_rn(lo, hi));
          y[4 * q] = lo.x; y[4 * q + 1] = lo.y; y[4 * q + 2] = hi.x; y[4 * q + 3] = hi.y;
        }
        part += acc.x + acc.y;
        store_x<AB>(x_mine, c, y);
      }
      tc::tmem_st_wait();
      psum[h * 128 + row] = part;
      if constexpr (!EMIS) {
        if (t + 1 < Tmax && h == 0) {
          const int on = (t + 1 < Tn && (unsigned)o_next < (unsigned)M) ? o_next : 0;
          stage_emission<NP>(eslot, Bk, on, ebar);
        }
      }
    }
    tc::bar_sync(1 + wg, WGT);
    if (!aborted && Tmax > 0)
      close_step(st, TPR == 2 ? psum[row] + psum[128 + row] : psum[row], Tmax - 1, Tn);
    if (aborted && lane == 0 && h == 0) {
      misc[2] = 1;
      set_status(a.status, HMM_STATUS_TIMEOUT);
    }
    if (has && h == 0) {
      float out = st.ll;
      if (st.bad || aborted) out = __int_as_float(0x7fc00000);
      else if (st.dead) out = -INFINITY;
      else if (!st.written) out = __int_as_float(0x7fc00000);
      if (st.bad && st.err) set_status(a.status, st.err);
      a.loglik[(size_t)s * K + k] = out;
    }

    // recognition: the last item of a tile pair takes the argmax over models
    if (a.argmax) {
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        misc[3] = (atomicAdd(a.done + tp, 1) == K - 1) ? 1 : 0;
      }
      __syncthreads();
      if (misc[3]) {
        __threadfence();
        if (has && h == 0) {
          const float* rp = a.loglik + (size_t)s * K;
          float best = __ldcg(rp);
          int arg = isnan(best) ? -1 : 0;
          for (int kk = 1; kk < K; ++kk) {
            const float vv = __ldcg(rp + kk);
            if (isnan(vv)) arg = -1;
            else if (arg >= 0 && vv > best) { best = vv; arg = kk; }
          }
          a.argmax[s] = arg;
        }
      }
    }
  }

  // teardown: no MMA or copy of ours may still be in flight. After a wait
  // gave up, the MMAs this warpgroup's issuing thread started are awaited
  // through a fresh commit, and the emission copies through the phase that
  // was being waited for (its parity is the flipped one's complement: a
  // completed phase returns at once).
  tc::fence_before_sync();
  __syncthreads();
  if (misc[2] && wtid == 0) {
    tc::mma_commit(fbar);
    tc::mbar_wait_bounded(fbar, 0, kWaitLimit);
    if constexpr (!EMIS) tc::mbar_wait_bounded(ebar, ephase ^ 1u, kWaitLimit);
  }
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int NP, int NT, int TPR, int AB, bool EMIS>
static cudaError_t launch_mma_t(const MmaFwdLaunch& a, cudaStream_t st) {
  auto kern = hmm_forward_mma<NP, NT, TPR, AB, EMIS>;
  using L = MmaFwdSmem<NP, NT, TPR, AB, EMIS>;
  // one CTA per SM (it holds all 512 tensor-memory columns): ask for more
  // than half of the shared memory even when the tiles need less
  const int need = L::total(a.seq.M);
  const int smem = need > 120 * 1024 ? need : 120 * 1024;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  int blocks = num_sms();
  if (blocks > a.n_items) blocks = a.n_items > 0 ? a.n_items : 1;
  kern<<<blocks, kMmaThreads, smem, st>>>(a);
  return cudaGetLastError();
}

int mma_tiles_per_cta(int NP) { return NP == 64 ? 4 : 2; }

// The emission table goes to shared memory when it fits next to A^T.
template <int NP, int NT, int TPR, int AB>
static cudaError_t launch_mma_e(const MmaFwdLaunch& a, cudaStream_t st) {
  if (MmaFwdSmem<NP, NT, TPR, AB, true>::total(a.seq.M) <= kFwdSmemMax)
    return launch_mma_t<NP, NT, TPR, AB, true>(a, st);
  return launch_mma_t<NP, NT, TPR, AB, false>(a, st);
}

cudaError_t launch_forward_mma(int NP, bool tf32, const MmaFwdLaunch& a, cudaStream_t st) {
  if (NP == 64) return tf32 ? launch_mma_e<64, 4, 1, 2>(a, st) : launch_mma_e<64, 4, 1, 1>(a, st);
  if (NP == 128) return tf32 ? launch_mma_e<128, 2, 2, 2>(a, st) : launch_mma_e<128, 2, 2, 1>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
