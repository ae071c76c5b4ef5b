// mma_fb.cu -- forward-backward adjoint on the tensor cores for N = 64 or 128
// states (Sec. 2.7 "Baum-Welch", its E-step; Rabiner 1989 eqs. 24-25
// backward variable, 37 xi, 38 gamma), the tensor-core twin of fb.cu.
//
// A tile is 128 (sequence, model) pairs of ONE model (the plan kernel groups
// them, rows sorted by decreasing length bucket; the tile runs for its longest
// row). Per time step every product of the
// recursion is a dense contraction over those 128 rows or over the states:
//   forward    D[m][j]  = sum_i X_{t-1}[m][i] a_ij         (M=128, N=NP, K=NP)
//   backward   D[m][i]  = sum_j Y_{t+1}[m][j] a_ij         (M=128, N=NP, K=NP)
//   xi         XI[i][j] += sum_m X_t[m][i] Y_{t+1}[m][j]   (M=128, N=NP, K=128 rows)
//   emissions  CB[k][j] += sum_m [o_t(m) = k] G_t[m][j]    (M=128 symbols, N=NP, K=128)
// all as tcgen05.mma kind::f16 (BF16 operands in shared memory, FP32
// accumulators in tensor memory). X, Y and G are stored once per step as
// 128 x NP BF16 "row images" (row m contiguous in 8-column groups); the same
// bytes are the K-major operand of the per-row products and the MN-major
// operand of the contractions over rows, so no operand is ever transposed.
// XI and CB accumulate over the whole tile in tensor memory and are written
// once per tile to the tile's slot; the slots are summed in a fixed order
// (bitwise reproducible). At N = 64 the xi product uses M = 128 with rows
// 64..127 of the A operand running into the next buffer: those accumulator
// rows are never read.
//
// Scaling. The forward pass is the one of mma_forward.cu: X_t = bf16(D_t .
// b(o_t) . 2^-g_t) with the exponent g_t of the previous step's row sum
// (one step late, clamped), log P = ln sigma_{T-1} + (sum g) ln 2. The
// exponents are stored (one byte per row and step) so the recompute repeats
// phase 1 bit for bit. Backward, with Bt_t = A Y_{t+1} (Bt_{T-1} = 1):
//   G_t = X_t . Bt_t . c_t,    Y_t = b(o_t) . Bt_t . 2^-g_t . c_t,
// with c_{T-1} = w / sigma_{T-1} and c_t = w / (c_{t+1} rho_{t+1}),
// rho_t = sum_i X_t(i) Bt_t(i). In exact arithmetic rho_t = c_{t+1} rho_{t+1},
// so every step's gamma sums to the row weight w; using the previous step's
// measured sum keeps the BF16 rounding of one step from accumulating over T
// (the same one-step-late idea as the forward scaling, and no extra barrier).
//
// Memory (Sec. 2.7, checkpointed adjoint): phase 1 keeps X every C steps,
// C = ceil(sqrt(L)) for the tile's longest row L (at most 16 while L <= 8192,
// so one segment's recomputed images stay in L2); phase 2 walks the
// segments backwards, recomputing a segment's X images into a per-CTA buffer
// and then running the backward recursion over it.
//
// Ordering per backward step (single-buffered operands): the step's MMAs are
// issued as [emissions of step t+1, xi of step t, backward of step t] under
// one commit, so when the epilogue of step t starts every operand buffer is
// free to be rewritten. Every mbarrier wait is bounded; on timeout the kernel
// sets HMM_STATUS_TIMEOUT, waits (bounded) for its own MMAs and copies and
// leaves.
#include "hmm_internal.cuh"
#include "tc.cuh"

namespace hmmgb {

template <int NP, int MB>
struct MmaFbCfg {
  static constexpr int TPR = NP / 32;            // threads per row, 32 columns each
  static constexpr int NTH = 128 * TPR;
  static constexpr int IMG = 128 * NP * 2;       // one 128-row BF16 image
  static constexpr int MAT = NP * NP * 2;        // one BF16 transition image
  static constexpr int OFF_AT = 0;               // forward B operand: (n=j, k=i) = a_ij
  static constexpr int OFF_AM = MAT;             // backward B operand: (n=i, k=j) = a_ij
  static constexpr int OFF_XI = 2 * MAT;         // X_t (xi A operand)
  static constexpr int OFF_Y = OFF_XI + IMG;     // Y_t
  static constexpr int OFF_G = OFF_Y + IMG;      // gamma_t; forward X operand in phase 1 / recompute
  static constexpr int OFF_OH = OFF_G + IMG;     // one-hot [k][m], MB blocks of 128 x 128
  static constexpr int OFF_PS = OFF_OH + MB * 32768;    // row partial sums [TPR][128]
  static constexpr int OFF_BAR = OFF_PS + TPR * 128 * 4;  // mma, xi copy
  static constexpr int OFF_MISC = OFF_BAR + 16;
  static constexpr int TOTAL = OFF_MISC + 64;
  static constexpr int TMEM_USED = (2 + MB) * NP;  // D, XI, CB blocks
  static constexpr int TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
  static constexpr int CTAS = (TOTAL <= 113 * 1024 && TMEM_COLS <= 256) ? 2 : 1;
};
static_assert(MmaFbCfg<128, 2>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<128, 2>::TMEM_USED <= 512, "tensor memory budget");
static_assert(MmaFbCfg<64, 1>::CTAS == 2, "two CTAs per SM at N = 64, M <= 128");

constexpr uint32_t kFbWaitLimit = 1u << 24;

// Byte offset of 8-column group c8 of row m in a 128 x NP row image.
template <int NP>
__device__ __forceinline__ uint32_t img_off(int m, int c8) {
  return (uint32_t)((m & 7) * 16 + c8 * 128 + (m >> 3) * NP * 16);
}

// Row m, columns [32h, 32h + 32) of an image, as 16 packed BF16 pairs.
template <int NP>
__device__ __forceinline__ void img_put(uint8_t* img, int m, int h, const uint32_t (&w)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(img + img_off<NP>(m, 4 * h + q)) =
        make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}
template <int NP>
__device__ __forceinline__ void img_put_global(uint8_t* img, int m, int h, const uint32_t (&w)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    __stcg(reinterpret_cast<uint4*>(img + img_off<NP>(m, 4 * h + q)),
           make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]));
}
template <int NP>
__device__ __forceinline__ void img_get_global(const uint8_t* img, int m, int h, uint32_t (&w)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(img + img_off<NP>(m, 4 * h + q)));
    w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
  }
}

// 32 emission probabilities b_j(sym), j in [32h, 32h + 32).
template <int NP>
__device__ __forceinline__ void load_emis(float (&b)[32], const float* Bk, int sym, int h) {
  const float4* p = reinterpret_cast<const float4*>(Bk + (size_t)sym * NP + 32 * h);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 v = __ldg(p + q);
    b[4 * q] = v.x; b[4 * q + 1] = v.y; b[4 * q + 2] = v.z; b[4 * q + 3] = v.w;
  }
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

__device__ __forceinline__ void pack32w(const float (&y)[32], uint32_t (&w)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = tc::pack_bf16(y[2 * i], y[2 * i + 1]);
}

__device__ __forceinline__ int exponent_of_fb(float s) {
  if (s < 0x1p-120f) return frexp2(s * 0x1p64f) - 64;
  return frexp2(s);
}

// Forward-pass row state (identical in all threads of a row).
struct FbRow {
  int F;          // sum of applied exponents
  int f;          // exponent for the next step
  bool dead, bad, written;
  int err;
  float ll;       // log-likelihood
  float S_last;   // row sum at the last step
};

__device__ __forceinline__ void fb_close(FbRow& st, float sigma, int t, int T) {
  if (t >= T || st.dead || st.bad) return;
  if (sigma == 0.f) { st.dead = true; return; }
  if (!(sigma > 0.f) || isinf(sigma)) { st.bad = true; st.err |= HMM_STATUS_PARAM; return; }
  if (t == T - 1) {
    st.ll = (float)(log((double)sigma) + (double)st.F * 0.69314718055994530942);
    st.S_last = sigma;
    st.written = true;
  }
  st.f = min(126, max(-126, exponent_of_fb(sigma)));
}

template <int NP, int MB>
__global__ void __launch_bounds__(MmaFbCfg<NP, MB>::NTH, MmaFbCfg<NP, MB>::CTAS)
    hmm_fb_mma(MmaFbLaunch a) {
  using L = MmaFbCfg<NP, MB>;
  constexpr int TPR = L::TPR, NTH = L::NTH, IMG = L::IMG;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAT = smem + L::OFF_AT;
  uint8_t* sAM = smem + L::OFF_AM;
  uint8_t* sXI = smem + L::OFF_XI;
  uint8_t* sY = smem + L::OFF_Y;
  uint8_t* sG = smem + L::OFF_G;
  uint8_t* sOH = smem + L::OFF_OH;
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint64_t* xbar = mbar + 1;
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = warp >> 2, row = wq * 32 + lane;
  const int K = a.seq.K, M = a.seq.M;

  for (int i = tid; i < MB * 32768 / 16; i += NTH)
    reinterpret_cast<uint4*>(sOH)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), L::TMEM_COLS);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(xbar, 1);
    misc[2] = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
  const uint32_t d_tm = tmem, xi_tm = tmem + NP, cb_tm = tmem + 2 * NP;
  constexpr uint32_t id_kk = tc::instr_desc(1, 128, NP);               // A, B K-major
  constexpr uint32_t id_mm = id_kk | (1u << 15) | (1u << 16);          // A, B MN-major
  constexpr uint32_t id_km = id_kk | (1u << 16);                       // B MN-major
  const uint32_t aAT = tc::smem_u32(sAT), aAM = tc::smem_u32(sAM), aXI = tc::smem_u32(sXI);
  const uint32_t aY = tc::smem_u32(sY), aG = tc::smem_u32(sG), aOH = tc::smem_u32(sOH);
  constexpr uint32_t SBO = NP * 16;

  uint8_t* ckpt = a.ckpt + (size_t)blockIdx.x * a.ckpt_bytes;
  uint8_t* scr = a.scr + (size_t)blockIdx.x * a.scr_bytes;
  int8_t* gexp = a.gexp + (size_t)blockIdx.x * a.gexp_bytes;
  float* gbuf = a.gbuf + (size_t)blockIdx.x * 128 * NP;

  uint32_t mph = 0, xph = 0;
  bool x_inflight = false;  // thread 0: a copy into sXI not yet waited for
  uint32_t x_par = 0;       // ... and the parity its completion flips
  bool mma_pending = false; // thread 0: MMAs committed but not waited for
  uint32_t m_par = 0;       // ... and the parity their commit completes
  bool aborted = false;
  int cur_model = -1;

  // thread 0 issues; warp 0 polls; everyone agrees on the outcome
  auto commit = [&]() {  // thread 0
    tc::mma_commit(mbar);
    mma_pending = true;
    m_par = mph;
  };
  auto wait_mma = [&]() -> bool {
    bool ok = true;
    if (warp == 0) ok = tc::mbar_wait_bounded(mbar, mph, kFbWaitLimit);
    mph ^= 1;
    if (tid == 0) mma_pending = !ok;
    ok = tc::bar_and(1, NTH, ok);
    tc::fence_after_sync();
    return ok;
  };
  auto copy_x = [&](const uint8_t* src) {  // thread 0: sXI <- one row image
    tc::mbar_arrive_expect_tx(xbar, IMG);
    tc::bulk_g2s(aXI, src, IMG, xbar);
    x_inflight = true;
    x_par = xph;
  };
  auto issue_fwd = [&]() {  // D = X_op . A   (X_op in sG)
#pragma unroll
    for (int ks = 0; ks < NP / 16; ++ks)
      tc::mma_bf16(d_tm, tc::smem_desc(aG + ks * 256, 128, SBO),
                   tc::smem_desc(aAT + ks * 256, 128, SBO), id_kk, ks > 0 ? 1u : 0u);
  };

  for (;;) {
    __syncthreads();
    if (tid == 0) misc[1] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = misc[1];
    if (item >= __ldcg(a.n_tiles) || misc[2]) break;
    const int tile = a.tile_order[item];
    const int k = a.tile_model[tile];
    const int start = a.tile_start[tile];
    const int nrows = a.tile_rows[tile];
    const int Lt = a.tile_len[tile];

    const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
    if (k != cur_model) {
      for (int idx = tid; idx < NP * NP / 2; idx += NTH) {
        // forward image: (n = j, k = i), pairs along i
        {
          const int j = idx / (NP / 2), i = (idx % (NP / 2)) * 2;
          const uint32_t w = tc::pack_bf16(__ldg(Ak + i * NP + j), __ldg(Ak + (i + 1) * NP + j));
          *reinterpret_cast<uint32_t*>(sAT + (j / 8) * SBO + (i / 8) * 128 + (j % 8) * 16 +
                                       (i % 8) * 2) = w;
        }
        // backward image: (n = i, k = j), pairs along j
        {
          const int i = idx / (NP / 2), j = (idx % (NP / 2)) * 2;
          const uint32_t w = tc::pack_bf16(__ldg(Ak + i * NP + j), __ldg(Ak + i * NP + j + 1));
          *reinterpret_cast<uint32_t*>(sAM + (i / 8) * SBO + (j / 8) * 128 + (i % 8) * 16 +
                                       (j % 8) * 2) = w;
        }
      }
      cur_model = k;
      tc::fence_proxy_async();
      __syncthreads();
    }

    const bool has = row < nrows;
    const int s = has ? a.sorted[start + row] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    const size_t oidx = a.labelled ? (size_t)s : (size_t)s * K + k;
    const float w = has ? (a.weight ? a.weight[oidx] : 1.f) : 0.f;
    const int32_t* o = a.seq.symbols + (has ? a.seq.offsets[s] : 0);
    const float* Bk = a.mod.Btp + (size_t)k * M * NP;
    const int C = fb_mma_segment(Lt);
    const int NS = (Lt + C - 1) / C;

    // ---------------- phase 1: forward, checkpoints every C steps ----------------
    FbRow st;
    st.F = 0; st.f = 0; st.dead = false; st.bad = false; st.written = false;
    st.err = 0; st.ll = 0.f; st.S_last = 0.f;
    {
      int o0 = T > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; o0 = 0; }
      const bool live = T > 0 && !st.bad;
      float b[32], y[32];
      load_emis<NP>(b, Bk, o0, h);
      const float4* p4 = reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * NP + 32 * h);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 pp = __ldg(p4 + q);
        y[4 * q] = live ? pp.x * b[4 * q] : 0.f;
        y[4 * q + 1] = live ? pp.y * b[4 * q + 1] : 0.f;
        y[4 * q + 2] = live ? pp.z * b[4 * q + 2] : 0.f;
        y[4 * q + 3] = live ? pp.w * b[4 * q + 3] : 0.f;
      }
      uint32_t wv[16];
      pack32w(y, wv);
      img_put<NP>(sG, row, h, wv);
      img_put_global<NP>(ckpt, row, h, wv);
      psum[h * 128 + row] = tree_sum<32>(y);
      if (h == 0) __stcg(gexp + row, (int8_t)0);
    }
    int o_n1 = (1 < T) ? __ldg(o + 1) : 0;  // symbol of the next step
    int o_n2 = (2 < T) ? __ldg(o + 2) : 0;  // and the one after
    float bcur[32];
    load_emis<NP>(bcur, Bk, (unsigned)o_n1 < (unsigned)M ? o_n1 : 0, h);
    tc::fence_proxy_async();

    for (int t = 1; t < Lt && !aborted; ++t) {
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        issue_fwd();
        commit();
      }
      {
        float sig = 0.f;
#pragma unroll
        for (int q = 0; q < TPR; ++q) sig += psum[q * 128 + row];
        fb_close(st, sig, t - 1, T);
      }
      const int ot = o_n1;
      o_n1 = o_n2;
      o_n2 = (t + 2 < T) ? __ldg(o + t + 2) : 0;
      if (t < T && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
      const bool live = t < T && !st.dead && !st.bad;
      if (live) st.F += st.f;
      if (h == 0) __stcg(gexp + (size_t)t * 128 + row, (int8_t)st.f);
      if (!wait_mma()) { aborted = true; break; }
      float y[32];
      tc::tmem_ld32(d_tm + lane_off + (uint32_t)(32 * h), y);
      tc::tmem_ld_wait();
      const float fac = exp2i(-st.f);
#pragma unroll
      for (int i = 0; i < 32; ++i) y[i] = live ? y[i] * bcur[i] * fac : 0.f;
      uint32_t wv[16];
      pack32w(y, wv);
      img_put<NP>(sG, row, h, wv);
      if (t % C == 0) img_put_global<NP>(ckpt + (size_t)(t / C) * IMG, row, h, wv);
      psum[h * 128 + row] = tree_sum<32>(y);
      load_emis<NP>(bcur, Bk, (t + 1 < T && (unsigned)o_n1 < (unsigned)M) ? o_n1 : 0, h);
      tc::fence_proxy_async();
    }
    // checkpoints (generic-proxy stores) may be read by bulk copies
    asm volatile("fence.proxy.async;" ::: "memory");
    __syncthreads();
    if (!aborted && Lt > 0) {
      float sig = 0.f;
#pragma unroll
      for (int q = 0; q < TPR; ++q) sig += psum[q * 128 + row];
      fb_close(st, sig, Lt - 1, T);
    }
    __syncthreads();  // every row has read its sums before phase 2 rewrites them
    if (has && h == 0) {
      float out = st.ll;
      if (st.bad || aborted) out = __int_as_float(0x7fc00000);
      else if (st.dead) out = -INFINITY;
      else if (!st.written) out = __int_as_float(0x7fc00000);
      if (st.bad && st.err) set_status(a.status, st.err);
      a.loglik[oidx] = out;
    }
    if (aborted) break;

    // ---------------- phase 2: segments backwards ----------------
    const bool act = has && st.written && !st.dead && !st.bad && w != 0.f;
    float c = 0.f;        // this row's current normaliser
    int kprev = -1;       // one-hot entry set by the previous step
    bool xi_on = false;   // thread 0: an xi MMA has been issued for this tile
    bool cb_on = false;   // thread 0: an emission MMA has been issued for this tile
    bool cb_pending = false;
    for (int seg = NS - 1; seg >= 0 && !aborted; --seg) {
      const int t0 = seg * C, t1 = min(t0 + C, Lt);
      const uint8_t* ck = ckpt + (size_t)seg * IMG;
      auto img_of = [&](int t) -> const uint8_t* {
        return t == t0 ? ck : scr + (size_t)(t - t0) * IMG;
      };
      // (R) recompute X over the segment from its checkpoint
      if (t1 - t0 > 1) {
        {
          uint32_t wv[16];
          img_get_global<NP>(ck, row, h, wv);
          img_put<NP>(sG, row, h, wv);
        }
        int fn = (int)__ldcg(gexp + (size_t)(t0 + 1) * 128 + row);
        int on = (t0 + 1 < T) ? __ldg(o + t0 + 1) : 0;
        load_emis<NP>(bcur, Bk, (unsigned)on < (unsigned)M ? on : 0, h);
        on = (t0 + 2 < T && t0 + 2 < t1) ? __ldg(o + t0 + 2) : 0;
        tc::fence_proxy_async();
        for (int t = t0 + 1; t < t1; ++t) {
          tc::fence_before_sync();
          __syncthreads();
          if (tid == 0) {
            tc::fence_after_sync();
            issue_fwd();
            commit();
          }
          const int f = fn;
          if (!wait_mma()) { aborted = true; break; }
          const bool live = act && t < T;
          float y[32];
          tc::tmem_ld32(d_tm + lane_off + (uint32_t)(32 * h), y);
          tc::tmem_ld_wait();
          const float fac = exp2i(-f);
#pragma unroll
          for (int i = 0; i < 32; ++i) y[i] = live ? y[i] * bcur[i] * fac : 0.f;
          uint32_t wv[16];
          pack32w(y, wv);
          img_put<NP>(sG, row, h, wv);
          img_put_global<NP>(scr + (size_t)(t - t0) * IMG, row, h, wv);
          if (t + 1 < t1) {
            fn = (int)__ldcg(gexp + (size_t)(t + 1) * 128 + row);
            load_emis<NP>(bcur, Bk, (unsigned)on < (unsigned)M ? on : 0, h);
            on = (t + 2 < T && t + 2 < t1) ? __ldg(o + t + 2) : 0;
          }
          tc::fence_proxy_async();
        }
        if (aborted) break;
        // the recomputed images (generic-proxy stores) are read by bulk copies
        asm volatile("fence.proxy.async;" ::: "memory");
      }
      __syncthreads();

      // (B) backward over the segment
      uint32_t xcur[16];
      float bb[32];
      int ocur, gcur;
      {
        const int t = t1 - 1;
        img_get_global<NP>(img_of(t), row, h, xcur);
        ocur = (t < T) ? __ldg(o + t) : 0;
        if ((unsigned)ocur >= (unsigned)M) ocur = 0;
        load_emis<NP>(bb, Bk, ocur, h);
        gcur = (int)__ldcg(gexp + (size_t)t * 128 + row);
        if (tid == 0 && t < Lt - 1) copy_x(img_of(t));
      }
      for (int t = t1 - 1; t >= t0; --t) {
        const bool has_mma = t < Lt - 1;
        float rho_prev = 0.f;
        if (has_mma) {
          tc::fence_before_sync();
          __syncthreads();
          bool ok0 = true;
          if (tid == 0) {
            ok0 = tc::mbar_wait_bounded(xbar, xph, kFbWaitLimit);
            xph ^= 1;
            x_inflight = !ok0;
            if (ok0) {
              tc::fence_after_sync();
              if (cb_pending) {
#pragma unroll
                for (int b = 0; b < MB; ++b)
#pragma unroll
                  for (int ks = 0; ks < 8; ++ks)
                    tc::mma_bf16(cb_tm + (uint32_t)(b * NP),
                                 tc::smem_desc(aOH + b * 32768 + ks * 256, 128, 2048),
                                 tc::smem_desc(aG + ks * 32 * NP, NP * 16, 128), id_km,
                                 (ks > 0 || cb_on) ? 1u : 0u);
                cb_on = true;
              }
#pragma unroll
              for (int ks = 0; ks < 8; ++ks)
                tc::mma_bf16(xi_tm, tc::smem_desc(aXI + ks * 32 * NP, NP * 16, 128),
                             tc::smem_desc(aY + ks * 32 * NP, NP * 16, 128), id_mm,
                             (ks > 0 || xi_on) ? 1u : 0u);
              xi_on = true;
#pragma unroll
              for (int ks = 0; ks < NP / 16; ++ks)
                tc::mma_bf16(d_tm, tc::smem_desc(aY + ks * 256, 128, SBO),
                             tc::smem_desc(aAM + ks * 256, 128, SBO), id_kk, ks > 0 ? 1u : 0u);
            }
            commit();  // also when skipped: the phase still completes
          }
#pragma unroll
          for (int q = 0; q < TPR; ++q) rho_prev += psum[q * 128 + row];
          bool ok = true;
          if (warp == 0) ok = tc::mbar_wait_bounded(mbar, mph, kFbWaitLimit);
          mph ^= 1;
          if (tid == 0) mma_pending = !ok;
          ok = tc::bar_and(1, NTH, ok && ok0);
          tc::fence_after_sync();
          if (!ok) { aborted = true; break; }
        }
        cb_pending = false;
        // copy X_{t-1} for the next step's xi product (sXI is free now)
        if (tid == 0 && t > t0) copy_x(img_of(t - 1));
        float bt[32];
        if (has_mma) {
          tc::tmem_ld32(d_tm + lane_off + (uint32_t)(32 * h), bt);
          tc::tmem_ld_wait();
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) bt[i] = 0.f;
        }
        const bool is_init = act && t == T - 1;
        const bool on = act && t < T - 1;
        if (is_init) {
#pragma unroll
          for (int i = 0; i < 32; ++i) bt[i] = 1.f;
          c = w / st.S_last;
        } else if (on) {
          c = w / (c * rho_prev);
        }
        const bool live = (is_init || on) && isfinite(c);
        const float fc = exp2i(-gcur) * c;  // exact: c times a power of two
        float part = 0.f;
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {  // 8 columns = one 16-byte image chunk
          uint32_t gp[4], yp[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = 4 * g8 + u;
            const float2 xv = unpack_bf16(xcur[q]);
            const float g0 = xv.x * bt[2 * q], g1 = xv.y * bt[2 * q + 1];
            part += g0 + g1;
            float ga = g0 * c, gb = g1 * c;
            float ya = bb[2 * q] * bt[2 * q] * fc, yb = bb[2 * q + 1] * bt[2 * q + 1] * fc;
            if (!live) { ga = 0.f; gb = 0.f; ya = 0.f; yb = 0.f; }
            if (t == 0)
              __stcg(reinterpret_cast<float2*>(gbuf + (size_t)row * NP + 32 * h + 2 * q),
                     make_float2(ga, gb));
            gp[u] = tc::pack_bf16(ga, gb);
            yp[u] = tc::pack_bf16(ya, yb);
          }
          *reinterpret_cast<uint4*>(sY + img_off<NP>(row, 4 * h + g8)) =
              make_uint4(yp[0], yp[1], yp[2], yp[3]);
          *reinterpret_cast<uint4*>(sG + img_off<NP>(row, 4 * h + g8)) =
              make_uint4(gp[0], gp[1], gp[2], gp[3]);
        }
        if (h == 0) {
          if (kprev >= 0)
            *reinterpret_cast<uint16_t*>(sOH + (kprev >> 7) * 32768 + img_off<128>(kprev & 127, row >> 3) +
                                         (row & 7) * 2) = 0;
          kprev = -1;
          if (live) {
            *reinterpret_cast<uint16_t*>(sOH + (ocur >> 7) * 32768 + img_off<128>(ocur & 127, row >> 3) +
                                         (row & 7) * 2) = 0x3F80;  // BF16 1.0
            kprev = ocur;
          }
        }
        psum[h * 128 + row] = live ? part : 0.f;
        if (!live) c = 0.f;
        // prefetch step t - 1
        if (t > t0) {
          img_get_global<NP>(img_of(t - 1), row, h, xcur);
          ocur = (t - 1 < T) ? __ldg(o + t - 1) : 0;
          if ((unsigned)ocur >= (unsigned)M) ocur = 0;
          load_emis<NP>(bb, Bk, ocur, h);
          gcur = (int)__ldcg(gexp + (size_t)(t - 1) * 128 + row);
        }
        tc::fence_proxy_async();
        cb_pending = true;
      }
      if (aborted) break;
      // the segment's last emission product, before gamma's buffer is reused
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int b = 0; b < MB; ++b)
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            tc::mma_bf16(cb_tm + (uint32_t)(b * NP),
                         tc::smem_desc(aOH + b * 32768 + ks * 256, 128, 2048),
                         tc::smem_desc(aG + ks * 32 * NP, NP * 16, 128), id_km,
                         (ks > 0 || cb_on) ? 1u : 0u);
        cb_on = true;
        commit();
      }
      cb_pending = false;
      if (!wait_mma()) { aborted = true; break; }
    }
    if (aborted) break;

    // ---------------- tile counts -> slot ----------------
    float* slot = a.slots + (size_t)tile * a.slot_floats;
    if (wq * 32 < NP) {  // xi rows i = row (warp-uniform)
      float v[32];
      if (Lt >= 2) {
        tc::tmem_ld32(xi_tm + lane_off + (uint32_t)(32 * h), v);
        tc::tmem_ld_wait();
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      const float4* a4 = reinterpret_cast<const float4*>(Ak + (size_t)row * NP + 32 * h);
      float4* d4 = reinterpret_cast<float4*>(slot + NP + (size_t)row * NP + 32 * h);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 av = __ldg(a4 + q);
        d4[q] = make_float4(v[4 * q] * av.x, v[4 * q + 1] * av.y, v[4 * q + 2] * av.z,
                            v[4 * q + 3] * av.w);
      }
    }
#pragma unroll
    for (int b = 0; b < MB; ++b) {
      float v[32];
      tc::tmem_ld32(cb_tm + (uint32_t)(b * NP) + lane_off + (uint32_t)(32 * h), v);
      tc::tmem_ld_wait();
      const int sym = b * 128 + row;
      if (sym < M) {
        float* dst = slot + NP + (size_t)NP * NP + sym;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) dst[(size_t)(32 * h + jj) * M] = v[jj];
      }
    }
    __syncthreads();
    if (tid < NP) {
      float sum = 0.f;
      for (int m = 0; m < 128; ++m) sum += __ldcg(gbuf + (size_t)m * NP + tid);
      slot[tid] = sum;
    }
    if (h == 0 && kprev >= 0)
      *reinterpret_cast<uint16_t*>(sOH + (kprev >> 7) * 32768 + img_off<128>(kprev & 127, row >> 3) +
                                   (row & 7) * 2) = 0;
    tc::fence_proxy_async();
    tc::fence_before_sync();
  }

  // teardown: nothing of ours may still be in flight
  if (aborted) {
    if (lane == 0 && h == 0) {
      misc[2] = 1;
      set_status(a.status, HMM_STATUS_TIMEOUT);
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (mma_pending) tc::mbar_wait_bounded(mbar, m_par, kFbWaitLimit);
    if (x_inflight) tc::mbar_wait_bounded(xbar, x_par, kFbWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
}

template <int NP, int MB>
static cudaError_t launch_fb_mma_t(int grid, const MmaFbLaunch& a, cudaStream_t st) {
  using L = MmaFbCfg<NP, MB>;
  auto kern = hmm_fb_mma<NP, MB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
  if (err != cudaSuccess) return err;
  kern<<<grid, L::NTH, L::TOTAL, st>>>(a);
  return cudaGetLastError();
}

static int fb_mma_blocks(int M) { return (M + 127) / 128; }

bool fb_mma_supported(int NP, int M) {
  if (NP == 64) return fb_mma_blocks(M) <= 2;
  if (NP == 128) return fb_mma_blocks(M) <= 2;
  return false;
}

int fb_mma_ctas_per_sm(int NP, int M) {
  const int mb = fb_mma_blocks(M);
  if (NP == 64) return mb == 1 ? MmaFbCfg<64, 1>::CTAS : MmaFbCfg<64, 2>::CTAS;
  return mb == 1 ? MmaFbCfg<128, 1>::CTAS : MmaFbCfg<128, 2>::CTAS;
}

cudaError_t launch_fb_mma(int NP, int M, int grid, const MmaFbLaunch& a, cudaStream_t st) {
  const int mb = fb_mma_blocks(M);
  if (NP == 64 && mb == 1) return launch_fb_mma_t<64, 1>(grid, a, st);
  if (NP == 64 && mb == 2) return launch_fb_mma_t<64, 2>(grid, a, st);
  if (NP == 128 && mb == 1) return launch_fb_mma_t<128, 1>(grid, a, st);
  if (NP == 128 && mb == 2) return launch_fb_mma_t<128, 2>(grid, a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
