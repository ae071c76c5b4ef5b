// mma_pass.cu -- the first kernel of the tensor-core adjoint for N = 64 or 128
// states (Sec. 2.7 "Baum-Welch", its E-step; Rabiner 1989 eqs. 19-21 forward
// and 24-25 backward variables): the forward and the backward recursion of
// every tile as independent chains, each leaving checkpoints, so that the
// second kernel (mma_fb.cu) can process the checkpoint segments of one tile
// as independent work items instead of one chain of 3 T dependent steps.
//
// A work item is one group of up to NT tiles of one model (the plan's pass
// groups) in one direction; a CTA runs the NT tiles side by side (one
// warpgroup each, as the tensor-core forward of mma_forward.cu: the BF16
// operand rows in tensor memory, the B operand image in shared memory, D in
// tensor memory, the model's emission table in shared memory when it fits).
//
//  direction 0 (forward): X_t = bf16(D_t . b(o_t) . 2^-f_t), D_t = X_{t-1} A,
//    with the exponent f_t of the previous step's row sum (one step late,
//    clamped). Kept for the second kernel: X_t at t = c C (checkpoint images,
//    C = the tile's segment length), every row's f_t (one byte per step), the
//    row sum at the row's last step, and log P = ln sigma_{T-1} + (sum f) ln 2
//    (the call's log-likelihood output).
//  direction 1 (backward): with Y_t = b(o_t) . beta_t (up to scale), the
//    backward recursion reads Y_t = (Y_{t+1} A^T) . b(o_t): the forward
//    recursion with the image of A in place of A^T, in reversed time. Each row
//    starts at its own last step T - 1 from Y = b(o_{T-1}) (rows of a tile end
//    at different steps; the tile's steps run from its longest row's end),
//    scaled by exact powers of two from the previous row sum like the forward.
//    Kept: Y_t at t = c C for c >= 1, the operand from which the second kernel
//    restarts the backward recursion of the segment that ends at c C - 1.
// Both directions use the same operand rounding as the second kernel's
// recursion, so a segment restarted from these checkpoints continues the
// same recursion. Every mbarrier wait is bounded; on timeout the kernel
// records HMM_STATUS_TIMEOUT, waits (bounded) for its own MMAs and copies and
// leaves.
#include "hmm_internal.cuh"
#include "mma_rows.cuh"
#include "tc.cuh"

namespace hmmgb {

constexpr int kPassThreads = 512;
constexpr uint32_t kPassTmemCols = 512;  // per tile: D (NP cols) then X (NP/2 cols)

// One 32-column chunk of this thread's share of a row: packed BF16 into the
// tensor-memory operand and, when `img` is set, into the row image in memory.
template <int NP>
__device__ __forceinline__ void put_chunk(uint32_t x_mine, int c, const float (&y)[32],
                                          uint8_t* img, int row, int col) {
  uint32_t w[16];
  pack32(y, w);
  tc::tmem_st16(x_mine + (uint32_t)(16 * c), w);
  if (img) {
#pragma unroll
    for (int g = 0; g < 4; ++g)
      __stcg(reinterpret_cast<uint4*>(img + img_off<NP>(row, col / 8 + g)),
             make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]));
  }
}

template <int NP, int NT, int TPR, bool EMIS>
__global__ void __launch_bounds__(kPassThreads, 1) hmm_fb_pass_mma(MmaPassLaunch a) {
  using L = MmaFwdSmem<NP, NT, TPR, 1, EMIS>;
  constexpr int XC = NP / 2;         // tensor-memory columns of X (BF16 pairs)
  constexpr int WGT = 128 * TPR;     // threads per tile
  static_assert(NT * WGT == kPassThreads, "512 threads per CTA");
  constexpr int HALF = NP / TPR;     // columns per thread
  constexpr int CH = HALF / 32;      // 32-column chunks per thread
  constexpr int TS = 512 / NT;       // tensor-memory columns per tile
  constexpr int IMG = 128 * NP * 2;  // one row image
  static_assert(NP + XC <= TS, "tile does not fit its tensor-memory share");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem + L::OFF_B;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);

  const int tid = threadIdx.x, wg = tid / WGT, wtid = tid % WGT;
  const int warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = (wtid >> 7);   // lane quarter, column share
  const int row = wq * 32 + lane;
  const uint8_t* erow = smem + L::OFF_E + (EMIS ? 0 : wg * L::kE + row * L::kES);
  const uint32_t eslot = tc::smem_u32(erow);
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS) + wg * TPR * 128;  // [TPR][128]
  uint64_t* mbar = &bars[wg];
  uint64_t* ebar = &bars[NT + wg];
  uint64_t* fbar = &bars[2 * NT + wg];
  const int K = a.seq.K, M = a.seq.M;

  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), kPassTmemCols);
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
  const uint32_t d_tmem = tmem + (uint32_t)(wg * TS);
  const uint32_t x_tmem = d_tmem + (uint32_t)NP;
  const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
  const uint32_t d_mine = d_tmem + lane_off + (uint32_t)(h * HALF);
  const uint32_t x_mine = x_tmem + lane_off + (uint32_t)(h * HALF / 2);
  constexpr uint32_t idesc = tc::instr_desc(1, 128, NP);
  const uint32_t b_base = tc::smem_u32(sB);
  constexpr uint32_t SBO = NP * 16;
  uint32_t mphase = 0, ephase = 0;
  int cur_key = -1;
  auto row_total = [&]() {  // the row sum of the last step (its TPR partial sums)
    float sum = psum[row];
#pragma unroll
    for (int q = 1; q < TPR; ++q) sum += psum[q * 128 + row];
    return sum;
  };

  for (;;) {
    __syncthreads();
    if (tid == 0) misc[1] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = misc[1];
    if (item >= 2 * __ldcg(a.n_pass) || misc[2]) break;
    const int grp = item >> 1, dir = item & 1;
    const int k = a.tile_model[a.pass_tiles[grp * NT]];

    if (2 * k + dir != cur_key) {
      // B operand, K-major: forward (n = j, k = i) = a_ij; backward (n = i, k = j) = a_ij
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
      for (int idx = tid; idx < NP * NP / 2; idx += kPassThreads) {
        const int n = idx / (NP / 2), kk = (idx % (NP / 2)) * 2;
        const float v0 = dir ? __ldg(Ak + n * NP + kk) : __ldg(Ak + kk * NP + n);
        const float v1 = dir ? __ldg(Ak + n * NP + kk + 1) : __ldg(Ak + (kk + 1) * NP + n);
        const uint32_t off = (n / 8) * SBO + (kk / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2;
        *reinterpret_cast<uint32_t*>(sB + off) = tc::pack_bf16(v0, v1);
      }
      if constexpr (EMIS) {
        if (cur_key < 0 || (cur_key >> 1) != k)
          fill_emission_table<NP, 1, L::kET>(smem + L::OFF_E, a.mod.Btp + (size_t)k * M * NP, M,
                                             tid, kPassThreads);
      }
      cur_key = 2 * k + dir;
      tc::fence_proxy_async();
      __syncthreads();
    }

    const int tile = a.pass_tiles[grp * NT + wg];
    const int rows = tile >= 0 ? a.tile_rows[tile] : 0;
    const bool has = row < rows;
    const int s = has ? a.sorted[a.tile_start[tile] + row] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;  // >= 1 for every row of a tile
    const int Tmax = tile >= 0 ? a.tile_len[tile] : 0;
    const int C = fb_mma_segment(Tmax > 0 ? Tmax : 1);
    // the row's first step: 0 forward; backward, its last symbol's step from
    // the end of the tile's longest row
    const int u0 = dir ? Tmax - T : 0;
    const float* Bk = a.mod.Btp + (size_t)k * M * NP;
    const int32_t* o = a.seq.symbols + (has ? a.seq.offsets[s] : 0);
    uint8_t* ckx = tile >= 0 ? a.ckx + (size_t)tile * a.ck_stride : nullptr;
    uint8_t* cky = tile >= 0 ? a.cky + (size_t)tile * a.ck_stride : nullptr;
    int8_t* gexp = tile >= 0 ? a.gexp + (size_t)tile * a.gexp_stride : nullptr;
    // symbol of tile step u (0 outside the row)
    auto sym_at = [&](int u) -> int {
      if (!has || u < u0 || u >= u0 + T) return 0;
      return __ldg(o + (dir ? Tmax - 1 - u : u));
    };
    // row image stored at tile step u (nullptr: none)
    auto ck_at = [&](int u) -> uint8_t* {
      if (tile < 0) return nullptr;
      if (!dir) return (u % C == 0) ? ckx + (size_t)(u / C) * IMG : nullptr;
      const int tt = Tmax - 1 - u;
      return (tt % C == 0 && tt >= C) ? cky + (size_t)(tt / C) * IMG : nullptr;
    };
    RowState st;
    st.F = 0; st.f = 0; st.dead = false; st.bad = false; st.written = false;
    st.err = 0; st.ll = 0.f; st.slast = 0.f;

    // step 0: forward x_0 = pi . b(o_0); backward, the rows whose last symbol
    // is the tile's last step: Y = b(o_{T-1}); no scaling
    {
      int o0 = sym_at(0);
      if ((unsigned)o0 >= (unsigned)M) {
        if (!dir) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
        o0 = 0;
      }
      const bool live = has && u0 == 0 && !st.bad;
      const float4* b4 = reinterpret_cast<const float4*>(Bk + (size_t)o0 * NP + h * HALF);
      const float4* p4 = reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * NP + h * HALF);
      uint8_t* img = ck_at(0);
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        float y[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 bb = __ldg(b4 + 8 * c + q);
          const float4 pp = dir ? make_float4(1.f, 1.f, 1.f, 1.f) : __ldg(p4 + 8 * c + q);
          y[4 * q] = live ? pp.x * bb.x : 0.f; y[4 * q + 1] = live ? pp.y * bb.y : 0.f;
          y[4 * q + 2] = live ? pp.z * bb.z : 0.f; y[4 * q + 3] = live ? pp.w * bb.w : 0.f;
        }
        part += tree_sum<32>(y);
        put_chunk<NP>(x_mine, c, y, img, row, h * HALF + 32 * c);
      }
      tc::tmem_st_wait();
      psum[h * 128 + row] = part;
      if (!dir && h == 0 && gexp) __stcg(gexp + row, (int8_t)0);
    }
    int o_next = sym_at(1);
    int o_next2 = EMIS ? sym_at(2) : 0;
    if constexpr (!EMIS) {
      if (Tmax > 1 && h == 0)
        stage_emission<NP>(eslot, Bk, (unsigned)o_next < (unsigned)M ? o_next : 0, ebar);
    }

    bool aborted = false;
    for (int t = 1; t < Tmax; ++t) {
      tc::fence_before_sync();
      tc::bar_sync(1 + wg, WGT);
      if (wtid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < NP / 16; ++ks)
          tc::mma_bf16_ts(d_tmem, x_tmem + (uint32_t)(ks * 8),
                          tc::smem_desc(b_base + ks * 256, 128, SBO), idesc, ks > 0 ? 1u : 0u);
        tc::mma_commit(mbar);
      }
      const float sig = row_total();
      if (!dir) {
        close_step(st, sig, t - 1, T);
      } else if (has && t - 1 >= u0 && !st.dead) {
        // backward: any positive scale will do; a zero row stays zero
        if (!(sig > 0.f) || isinf(sig)) st.dead = true;
        else st.f = min(126, max(-126, exponent_of(sig)));
      }
      const int ot = o_next;
      if constexpr (EMIS) {
        o_next = o_next2;
        o_next2 = sym_at(t + 2);
      } else {
        o_next = sym_at(t + 1);
      }
      const bool inrow = has && t >= u0 && t < u0 + T;
      if (!dir && inrow && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
      const uint8_t* eb = EMIS ? erow + ((unsigned)ot < (unsigned)M ? ot : 0) * L::kET : erow;
      const bool start = dir && t == u0;   // the backward row starts here: beta = 1
      const bool live = inrow && !st.dead && !st.bad;
      const int f = start ? 0 : st.f;
      if (!dir && live) st.F += f;
      const float2 fac2 = make_float2(exp2i(-f), exp2i(-f));
      bool ok = true;
      if (wtid < 32) {
        if constexpr (!EMIS) ok = tc::mbar_wait_bounded(ebar, ephase, a.wait_limit);
        ok = tc::mbar_wait_bounded(mbar, mphase, a.wait_limit) && ok;
      }
      if constexpr (!EMIS) ephase ^= 1;
      mphase ^= 1;
      if (!tc::bar_and(1 + wg, WGT, ok)) {
        aborted = true;
        break;
      }
      tc::fence_after_sync();
      uint8_t* img = ck_at(t);
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
            if ((q & 1) == 0) emission8<1>(eb, h * HALF + 32 * c + 4 * q, be);
            b = make_float4(be[4 * (q & 1)], be[4 * (q & 1) + 1], be[4 * (q & 1) + 2],
                            be[4 * (q & 1) + 3]);
          } else {
            b = *reinterpret_cast<const float4*>(eb + (h * HALF + 32 * c + 4 * q) * 4);
          }
          float2 ylo = make_float2(y[4 * q], y[4 * q + 1]);
          float2 yhi = make_float2(y[4 * q + 2], y[4 * q + 3]);
          if (start) { ylo = make_float2(1.f, 1.f); yhi = ylo; }
          float2 lo = __fmul2_rn(__fmul2_rn(ylo, make_float2(b.x, b.y)), fac2);
          float2 hi = __fmul2_rn(__fmul2_rn(yhi, make_float2(b.z, b.w)), fac2);
          if (!live) { lo = make_float2(0.f, 0.f); hi = lo; }
          acc = __fadd2_rn(acc, __fadd2_rn(lo, hi));
          y[4 * q] = lo.x; y[4 * q + 1] = lo.y; y[4 * q + 2] = hi.x; y[4 * q + 3] = hi.y;
        }
        part += acc.x + acc.y;
        put_chunk<NP>(x_mine, c, y, img, row, h * HALF + 32 * c);
      }
      tc::tmem_st_wait();
      psum[h * 128 + row] = part;
      if (!dir && h == 0) __stcg(gexp + (size_t)t * 128 + row, (int8_t)(live ? f : 0));
      if constexpr (!EMIS) {
        if (t + 1 < Tmax && h == 0)
          stage_emission<NP>(eslot, Bk, (unsigned)o_next < (unsigned)M ? o_next : 0, ebar);
      }
    }
    tc::bar_sync(1 + wg, WGT);
    if (!dir && !aborted && Tmax > 0)
      close_step(st, row_total(), Tmax - 1, T);
    if (aborted && lane == 0 && h == 0) {
      misc[2] = 1;
      set_status(a.status, HMM_STATUS_TIMEOUT);
    }
    if (!dir && tile >= 0 && h == 0) {
      // the second kernel's inputs: NaN = invalid row, 0 = no counts
      float sl = 0.f;
      if (st.bad || aborted) sl = __int_as_float(0x7fc00000);
      else if (has && st.written && !st.dead) sl = st.slast;
      a.s_last[(size_t)tile * 128 + row] = sl;
      if (has) {
        float out = st.ll;
        if (st.bad || aborted) out = __int_as_float(0x7fc00000);
        else if (st.dead) out = -INFINITY;
        else if (!st.written) out = __int_as_float(0x7fc00000);
        if (st.bad && st.err) set_status(a.status, st.err);
        a.loglik[a.labelled ? (size_t)s : (size_t)s * K + k] = out;
      }
    }
  }

  // teardown: no MMA or copy of ours may still be in flight (see mma_forward.cu)
  tc::fence_before_sync();
  __syncthreads();
  if (misc[2] && wtid == 0) {
    tc::mma_commit(fbar);
    tc::mbar_wait_bounded(fbar, 0, kDrainPolls);
    if constexpr (!EMIS) tc::mbar_wait_bounded(ebar, ephase ^ 1u, kDrainPolls);
  }
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kPassTmemCols);
}

template <int NP, int NT, int TPR, bool EMIS>
static cudaError_t launch_pass_t(const MmaPassLaunch& a, cudaStream_t st) {
  auto kern = hmm_fb_pass_mma<NP, NT, TPR, EMIS>;
  using L = MmaFwdSmem<NP, NT, TPR, 1, EMIS>;
  // one CTA per SM (it holds all 512 tensor-memory columns)
  const int need = L::total(a.seq.M);
  const int smem = need > 120 * 1024 ? need : 120 * 1024;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  kern<<<num_sms(), kPassThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NP, int NT, int TPR>
static cudaError_t launch_pass_e(const MmaPassLaunch& a, cudaStream_t st) {
  if (MmaFwdSmem<NP, NT, TPR, 1, true>::total(a.seq.M) <= kFwdSmemMax)
    return launch_pass_t<NP, NT, TPR, true>(a, st);
  return launch_pass_t<NP, NT, TPR, false>(a, st);
}

int fb_pass_tiles_per_cta(int NP, int tiles) {
  // N = 128: one tile per CTA (four threads per row) while the batch's forward
  // and backward chains fit about one per SM -- each chain's steps are then
  // shorter, and the pass is bound by its longest chain; two tiles per CTA
  // otherwise, trading step latency for throughput
  if (NP == 128) return 2 * tiles <= 2 * num_sms() ? 1 : 2;
  return 2;
}

cudaError_t launch_fb_pass(int NP, int tiles_per_cta, const MmaPassLaunch& a, cudaStream_t st) {
  if (NP == 64 && tiles_per_cta == 4) return launch_pass_e<64, 4, 1>(a, st);
  if (NP == 64 && tiles_per_cta == 2) return launch_pass_e<64, 2, 2>(a, st);
  if (NP == 128 && tiles_per_cta == 2) return launch_pass_e<128, 2, 2>(a, st);
  if (NP == 128 && tiles_per_cta == 1) return launch_pass_e<128, 1, 4>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
