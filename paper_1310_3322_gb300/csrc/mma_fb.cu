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
  static constexpr int TPR = 4;                  // threads per row
  static constexpr int NTH = 128 * TPR;
  static constexpr int COLS = NP / TPR;          // columns per thread (16 or 32)
  static constexpr int CH = COLS / 8;            // 16-byte image chunks per thread
  static constexpr int IMG = 128 * NP * 2;       // one 128-row BF16 image
  static constexpr int MAT = NP * NP * 2;        // the BF16 transition image
  static constexpr bool EMIS = (NP == 64 && MB == 1);   // emission table in shared memory
  static constexpr int XIB = (NP == 64 || MB == 1) ? 2 : 1;  // X_t buffers
  static constexpr int ES = NP * 4 + 16;         // padded emission row (bytes)
  static constexpr int OFF_AT = 0;               // (n=j, k=i) = a_ij: forward K-major, backward MN-major
  static constexpr int OFF_XI = MAT;             // X_t images (xi A operand; epilogue rows)
  static constexpr int OFF_Y = OFF_XI + XIB * IMG;   // Y_t
  static constexpr int OFF_G = OFF_Y + IMG;      // gamma_t; the forward X operand in phase 1 / recompute
  static constexpr int OFF_OH = OFF_G + IMG;     // one-hot [k][m], MB blocks of 128 x 128
  static constexpr int OFF_B = OFF_OH + MB * 32768;  // emission rows b(k), k < 128 (EMIS)
  static constexpr int OFF_PS = OFF_B + (EMIS ? 128 * ES : 0);  // row partial sums [2][TPR][128]
  static constexpr int OFF_BAR = OFF_PS + 2 * TPR * 128 * 4;    // mma, gload, xi[2]
  static constexpr int OFF_MISC = OFF_BAR + 64;
  static constexpr int TOTAL = OFF_MISC + 64;
  static constexpr int TMEM_USED = (2 + MB) * NP;  // D, XI, CB blocks
  static constexpr int TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
};
static_assert(MmaFbCfg<128, 2>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<128, 1>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<64, 1>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<64, 2>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<128, 2>::TMEM_USED <= 512, "tensor memory budget");

constexpr uint32_t kFbWaitLimit = 1u << 24;

// Byte offset of 8-column group c8 of row m in a 128 x NP row image.
template <int NP>
__device__ __forceinline__ uint32_t img_off(int m, int c8) {
  return (uint32_t)((m & 7) * 16 + c8 * 128 + (m >> 3) * NP * 16);
}

// COLS consecutive FP32 values from tensor memory (one row = one lane).
template <int COLS>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[COLS]) {
  if constexpr (COLS == 32) tc::tmem_ld32(taddr, v);
  else tc::tmem_ld16(taddr, v);
  tc::tmem_ld_wait();
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
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

// Per-thread view of one tile row: the row, its column range and where its
// emission rows come from.
template <int NP, int MB>
struct FbThread {
  using L = MmaFbCfg<NP, MB>;
  int row, col0;
  const uint8_t* sB;   // shared emission table (EMIS)
  const float* Bk;     // global emission table of the model [M][NP]

  // b_j(sym) for this thread's columns
  __device__ __forceinline__ void emis(float (&b)[L::COLS], int sym) const {
    if constexpr (L::EMIS) {
      const float4* p = reinterpret_cast<const float4*>(sB + sym * L::ES + col0 * 4);
#pragma unroll
      for (int q = 0; q < L::COLS / 4; ++q) {
        const float4 v = p[q];
        b[4 * q] = v.x; b[4 * q + 1] = v.y; b[4 * q + 2] = v.z; b[4 * q + 3] = v.w;
      }
    } else {
      const float4* p = reinterpret_cast<const float4*>(Bk + (size_t)sym * NP + col0);
#pragma unroll
      for (int q = 0; q < L::COLS / 4; ++q) {
        const float4 v = __ldg(p + q);
        b[4 * q] = v.x; b[4 * q + 1] = v.y; b[4 * q + 2] = v.z; b[4 * q + 3] = v.w;
      }
    }
  }
  // this thread's columns of the row image: write (BF16 pairs) / read
  __device__ __forceinline__ void put(uint8_t* img, const uint32_t (&w)[L::COLS / 2]) const {
#pragma unroll
    for (int c = 0; c < L::CH; ++c)
      *reinterpret_cast<uint4*>(img + img_off<NP>(row, col0 / 8 + c)) =
          make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
  }
  __device__ __forceinline__ void get(const uint8_t* img, uint32_t (&w)[L::COLS / 2]) const {
#pragma unroll
    for (int c = 0; c < L::CH; ++c) {
      const uint4 v = *reinterpret_cast<const uint4*>(img + img_off<NP>(row, col0 / 8 + c));
      w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
    }
  }
  __device__ __forceinline__ void get_global(const uint8_t* img, uint32_t (&w)[L::COLS / 2]) const {
#pragma unroll
    for (int c = 0; c < L::CH; ++c) {
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(img + img_off<NP>(row, col0 / 8 + c)));
      w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
    }
  }
};

// Forward step epilogue: y = D . b . 2^-f (zero when not live), packed into
// the operand image; returns the partial row sum.
template <int COLS>
__device__ __forceinline__ float fwd_epilogue(float (&y)[COLS], const float (&b)[COLS], int f,
                                              bool live, uint32_t (&w)[COLS / 2]) {
  const float fac = exp2i(-f);
  const float2 f2 = make_float2(fac, fac);
#pragma unroll
  for (int i = 0; i < COLS / 2; ++i) {
    float2 v = __fmul2_rn(__fmul2_rn(make_float2(y[2 * i], y[2 * i + 1]),
                                     make_float2(b[2 * i], b[2 * i + 1])), f2);
    if (!live) v = make_float2(0.f, 0.f);
    y[2 * i] = v.x; y[2 * i + 1] = v.y;
    w[i] = tc::pack_bf16(v.x, v.y);
  }
  return tree_sum<COLS>(y);
}

template <int NP, int MB>
__global__ void __launch_bounds__(MmaFbCfg<NP, MB>::NTH, 1) hmm_fb_mma(MmaFbLaunch a) {
  using L = MmaFbCfg<NP, MB>;
  constexpr int TPR = L::TPR, NTH = L::NTH, IMG = L::IMG, COLS = L::COLS, XIB = L::XIB;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAT = smem + L::OFF_AT;
  uint8_t* sXI = smem + L::OFF_XI;
  uint8_t* sY = smem + L::OFF_Y;
  uint8_t* sG = smem + L::OFF_G;
  uint8_t* sOH = smem + L::OFF_OH;
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS);  // [2][TPR][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint64_t* mbar = bars;       // MMA commits
  uint64_t* gbar = bars + 1;   // checkpoint -> forward operand loads
  uint64_t* xbar = bars + 2;   // [XIB] X_t image loads
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);
  enum { M_TMEM = 0, M_ITEM = 1, M_ABORT = 2 };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = warp >> 2;
  const int K = a.seq.K, M = a.seq.M;
  FbThread<NP, MB> me;
  me.row = wq * 32 + lane;
  me.col0 = h * COLS;
  me.sB = smem + L::OFF_B;
  const int row = me.row;

  for (int i = tid; i < MB * 32768 / 16; i += NTH)
    reinterpret_cast<uint4*>(sOH)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), L::TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < 2 + XIB; ++i) tc::mbar_init(&bars[i], 1);
    misc[M_ABORT] = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = (uint32_t)misc[M_TMEM];
  const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
  const uint32_t d_tm = tmem, xi_tm = tmem + NP, cb_tm = tmem + 2 * NP;
  const uint32_t my_cols = lane_off + (uint32_t)me.col0;
  constexpr uint32_t id_kk = tc::instr_desc(1, 128, NP);               // A, B K-major
  constexpr uint32_t id_mm = id_kk | (1u << 15) | (1u << 16);          // A, B MN-major
  constexpr uint32_t id_km = id_kk | (1u << 16);                       // B MN-major
  const uint32_t aAT = tc::smem_u32(sAT), aXI = tc::smem_u32(sXI);
  const uint32_t aY = tc::smem_u32(sY), aG = tc::smem_u32(sG), aOH = tc::smem_u32(sOH);
  constexpr uint32_t SBO = NP * 16;

  uint8_t* ckpt = a.ckpt + (size_t)blockIdx.x * a.ckpt_bytes;
  uint8_t* scr = a.scr + (size_t)blockIdx.x * a.scr_bytes;
  int8_t* gexp = a.gexp + (size_t)blockIdx.x * a.gexp_bytes;
  float* gbuf = a.gbuf + (size_t)blockIdx.x * 128 * NP;

  // barrier phases (every thread tracks them; thread 0 also remembers what
  // it has in flight for the teardown)
  uint32_t mph = 0, gph = 0, xph[2] = {0, 0};
  bool m_pend = false, g_pend = false, x_pend[2] = {false, false};
  uint32_t m_par = 0, g_par = 0, x_par[2] = {0, 0};
  int cur_model = -1;

  auto fail = [&]() { misc[M_ABORT] = 1; };
  auto commit = [&]() {  // thread 0
    tc::mma_commit(mbar);
    m_pend = true;
    m_par = mph;
  };
  auto wait_mma = [&]() {  // every thread; a timeout is acted on at the next barrier
    if (!tc::mbar_wait_bounded(mbar, mph, kFbWaitLimit)) fail();
    else if (tid == 0) m_pend = false;
    mph ^= 1;
    tc::fence_after_sync();
  };
  auto load_x = [&](int b, const uint8_t* src) {  // thread 0: sXI[b] <- one row image
    tc::mbar_arrive_expect_tx(&xbar[b], IMG);
    tc::bulk_g2s(aXI + b * IMG, src, IMG, &xbar[b]);
    x_pend[b] = true;
    x_par[b] = xph[b];
  };
  auto wait_x = [&](int b) {  // every thread
    if (!tc::mbar_wait_bounded(&xbar[b], xph[b], kFbWaitLimit)) fail();
    else if (tid == 0) x_pend[b] = false;
    xph[b] ^= 1;
  };
  auto issue_fwd = [&]() {  // D = X_op . A   (X_op in sG)
#pragma unroll
    for (int ks = 0; ks < NP / 16; ++ks)
      tc::mma_bf16(d_tm, tc::smem_desc(aG + ks * 256, 128, SBO),
                   tc::smem_desc(aAT + ks * 256, 128, SBO), id_kk, ks > 0 ? 1u : 0u);
  };
  auto store_img = [&](uint8_t* dst) {  // thread 0: sG -> global image
    tc::bulk_s2g(dst, aG, IMG);
    tc::bulk_commit();
  };
  auto row_sum = [&](int par) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < TPR; ++q) s += psum[(par * TPR + q) * 128 + row];
    return s;
  };

  for (;;) {
    __syncthreads();
    if (tid == 0) misc[M_ITEM] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = misc[M_ITEM];
    if (item >= __ldcg(a.n_tiles) || misc[M_ABORT]) break;
    const int tile = a.tile_order[item];
    const int k = a.tile_model[tile];
    const int start = a.tile_start[tile];
    const int nrows = a.tile_rows[tile];
    const int Lt = a.tile_len[tile];

    const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
    me.Bk = a.mod.Btp + (size_t)k * M * NP;
    if (k != cur_model) {
      // transition image: (n = j, k = i) = a_ij, pairs along i
      for (int idx = tid; idx < NP * NP / 2; idx += NTH) {
        const int j = idx / (NP / 2), i = (idx % (NP / 2)) * 2;
        const uint32_t w = tc::pack_bf16(__ldg(Ak + i * NP + j), __ldg(Ak + (i + 1) * NP + j));
        *reinterpret_cast<uint32_t*>(sAT + (j / 8) * SBO + (i / 8) * 128 + (j % 8) * 16 +
                                     (i % 8) * 2) = w;
      }
      if constexpr (L::EMIS) {  // emission rows of the model, padded
        for (int idx = tid; idx < M * (NP / 4); idx += NTH) {
          const int sym = idx / (NP / 4), q = idx % (NP / 4);
          *reinterpret_cast<float4*>(smem + L::OFF_B + sym * L::ES + q * 16) =
              __ldg(reinterpret_cast<const float4*>(me.Bk + (size_t)sym * NP) + q);
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
    const int C = fb_mma_segment(Lt);
    const int NS = (Lt + C - 1) / C;
    auto sym_at = [&](int t) -> int {  // symbol at step t (0 past the row's end)
      if (t >= T) return 0;
      const int v = __ldg(o + t);
      return (unsigned)v < (unsigned)M ? v : 0;
    };

    // ---------------- phase 1: forward, checkpoints every C steps ----------------
    FbRow st;
    st.F = 0; st.f = 0; st.dead = false; st.bad = false; st.written = false;
    st.err = 0; st.ll = 0.f; st.S_last = 0.f;
    {
      int o0 = T > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; o0 = 0; }
      const bool live = T > 0 && !st.bad;
      float b[COLS], y[COLS];
      me.emis(b, o0);
      const float* pik = a.mod.pip + (size_t)k * NP + me.col0;
#pragma unroll
      for (int i = 0; i < COLS; ++i) y[i] = __ldg(pik + i);
      uint32_t wv[COLS / 2];
      const float sum = fwd_epilogue<COLS>(y, b, 0, live, wv);
      me.put(sG, wv);
      psum[(0 * TPR + h) * 128 + row] = sum;
      if (h == 0) __stcg(gexp + row, (int8_t)0);
    }
    int o_n1 = (1 < T) ? __ldg(o + 1) : 0;  // symbol of the next step
    int o_n2 = (2 < T) ? __ldg(o + 2) : 0;  // and the one after
    float bcur[COLS];
    if constexpr (!L::EMIS) me.emis(bcur, (unsigned)o_n1 < (unsigned)M ? o_n1 : 0);
    tc::fence_proxy_async();

    for (int t = 1; t < Lt; ++t) {
      tc::fence_before_sync();
      __syncthreads();
      if (misc[M_ABORT]) break;
      if (tid == 0) {
        tc::fence_after_sync();
        issue_fwd();
        if ((t - 1) % C == 0) {  // checkpoint X_{t-1} while the MMA reads it too
          store_img(ckpt + (size_t)((t - 1) / C) * IMG);
          tc::bulk_wait_read();
        }
        commit();
      }
      fb_close(st, row_sum((t - 1) & 1), t - 1, T);
      const int ot = o_n1;
      o_n1 = o_n2;
      o_n2 = (t + 2 < T) ? __ldg(o + t + 2) : 0;
      if (t < T && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
      const bool live = t < T && !st.dead && !st.bad;
      if (live) st.F += st.f;
      if (h == 0) __stcg(gexp + (size_t)t * 128 + row, (int8_t)st.f);
      if constexpr (L::EMIS) me.emis(bcur, live ? ot : 0);
      wait_mma();
      float y[COLS];
      tmem_ld_cols<COLS>(d_tm + my_cols, y);
      uint32_t wv[COLS / 2];
      const float sum = fwd_epilogue<COLS>(y, bcur, st.f, live, wv);
      me.put(sG, wv);
      psum[((t & 1) * TPR + h) * 128 + row] = sum;
      if constexpr (!L::EMIS)
        me.emis(bcur, (t + 1 < T && (unsigned)o_n1 < (unsigned)M) ? o_n1 : 0);
      tc::fence_proxy_async();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (misc[M_ABORT]) break;
    if (tid == 0) {
      if ((Lt - 1) % C == 0) store_img(ckpt + (size_t)((Lt - 1) / C) * IMG);
      tc::bulk_wait_all();  // every checkpoint written before phase 2 reads them
    }
    if (Lt > 0) fb_close(st, row_sum((Lt - 1) & 1), Lt - 1, T);
    if (has && h == 0) {
      float out = st.ll;
      if (st.bad) out = __int_as_float(0x7fc00000);
      else if (st.dead) out = -INFINITY;
      else if (!st.written) out = __int_as_float(0x7fc00000);
      if (st.bad && st.err) set_status(a.status, st.err);
      a.loglik[oidx] = out;
    }
    __syncthreads();  // every row has read its sums (and thread 0 waited for the checkpoints)

    // ---------------- phase 2: segments backwards ----------------
    const bool act = has && st.written && !st.dead && !st.bad && w != 0.f;
    float c = 0.f;        // this row's current normaliser
    int kprev = -1;       // one-hot entry set by the previous step
    bool xi_on = false;   // thread 0: an xi MMA has been issued for this tile
    bool cb_on = false;   // thread 0: an emission MMA has been issued for this tile
    bool cb_pending = false;
    bool stop = false;
    for (int seg = NS - 1; seg >= 0 && !stop; --seg) {
      const int t0 = seg * C, t1 = min(t0 + C, Lt);
      const uint8_t* ck = ckpt + (size_t)seg * IMG;
      auto img_of = [&](int t) -> const uint8_t* {
        return t == t0 ? ck : scr + (size_t)(t - t0) * IMG;
      };
      // (R) recompute X over the segment from its checkpoint
      if (t1 - t0 > 1) {
        if (tid == 0) {
          tc::mbar_arrive_expect_tx(gbar, IMG);
          tc::bulk_g2s(aG, ck, IMG, gbar);
          g_pend = true;
          g_par = gph;
        }
        int fn = (int)__ldcg(gexp + (size_t)(t0 + 1) * 128 + row);
        int on = sym_at(t0 + 1);
        if constexpr (!L::EMIS) me.emis(bcur, on);
        for (int t = t0 + 1; t < t1; ++t) {
          tc::fence_before_sync();
          __syncthreads();
          if (misc[M_ABORT]) { stop = true; break; }
          if (tid == 0) {
            if (t == t0 + 1) {
              if (!tc::mbar_wait_bounded(gbar, gph, kFbWaitLimit)) fail();
              else g_pend = false;
            }
            tc::fence_after_sync();
            issue_fwd();
            if (t - 1 > t0) {
              store_img(scr + (size_t)(t - 1 - t0) * IMG);
              tc::bulk_wait_read();
            }
            commit();
          }
          if (t == t0 + 1) gph ^= 1;
          const int f = fn;
          const int ot = on;
          if (t + 1 < t1) {
            fn = (int)__ldcg(gexp + (size_t)(t + 1) * 128 + row);
            on = sym_at(t + 1);
          }
          if constexpr (L::EMIS) me.emis(bcur, ot);
          wait_mma();
          float y[COLS];
          tmem_ld_cols<COLS>(d_tm + my_cols, y);
          uint32_t wv[COLS / 2];
          fwd_epilogue<COLS>(y, bcur, f, act && t < T, wv);
          me.put(sG, wv);
          if constexpr (!L::EMIS)
            if (t + 1 < t1) me.emis(bcur, on);
          tc::fence_proxy_async();
        }
        if (stop) break;
        tc::fence_before_sync();
        __syncthreads();
        if (misc[M_ABORT]) break;
        if (tid == 0) {
          store_img(scr + (size_t)(t1 - 1 - t0) * IMG);
          tc::bulk_wait_all();  // the segment's images are in memory (and sG is free)
        }
      }

      // (B) backward over the segment
      uint32_t xcur[COLS / 2];   // X_t of this row (XIB == 1: from memory)
      float bb[COLS];
      int ocur = sym_at(t1 - 1), gcur = (int)__ldcg(gexp + (size_t)(t1 - 1) * 128 + row);
      if constexpr (XIB == 1) me.get_global(img_of(t1 - 1), xcur);
      if constexpr (!L::EMIS) me.emis(bb, ocur);
      if (tid == 0 && (XIB == 2 || t1 - 1 < Lt - 1)) load_x((t1 - 1) % XIB, img_of(t1 - 1));
      for (int t = t1 - 1; t >= t0; --t) {
        const bool has_mma = t < Lt - 1;
        const int xb = t % XIB;
        tc::fence_before_sync();
        __syncthreads();
        if (misc[M_ABORT]) { stop = true; break; }
        if (tid == 0) {
          tc::fence_after_sync();
          if (has_mma) {
            if (XIB == 1) wait_x(0);
            else if (tc::mbar_wait_bounded(&xbar[xb], xph[xb], kFbWaitLimit)) x_pend[xb] = false;
            else fail();
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
              tc::mma_bf16(xi_tm, tc::smem_desc(aXI + xb * IMG + ks * 32 * NP, NP * 16, 128),
                           tc::smem_desc(aY + ks * 32 * NP, NP * 16, 128), id_mm,
                           (ks > 0 || xi_on) ? 1u : 0u);
            xi_on = true;
            // beta: D = Y . A^T, the transition image read MN-major
#pragma unroll
            for (int ks = 0; ks < NP / 16; ++ks)
              tc::mma_bf16(d_tm, tc::smem_desc(aY + ks * 256, 128, SBO),
                           tc::smem_desc(aAT + ks * 32 * NP, NP * 16, 128), id_km,
                           ks > 0 ? 1u : 0u);
            commit();
          }
          // the next step's X image (its buffer was last read before this
          // step's barrier; with one buffer, after this step's xi product)
          if (XIB == 2 && t > t0) load_x((t - 1) % 2, img_of(t - 1));
        }
        if (XIB == 1 && has_mma && tid != 0) xph[0] ^= 1;  // thread 0 flipped it in wait_x
        const float rho_prev = row_sum((t + 1) & 1);
        if constexpr (XIB == 2) {
          if (tid != 0 || !has_mma) wait_x(xb);
          else xph[xb] ^= 1;
        }
        if (has_mma) wait_mma();
        if (XIB == 1 && tid == 0 && t > t0) load_x(0, img_of(t - 1));
        float bt[COLS];
        if (has_mma) {
          tmem_ld_cols<COLS>(d_tm + my_cols, bt);
        } else {
#pragma unroll
          for (int i = 0; i < COLS; ++i) bt[i] = 0.f;
        }
        if constexpr (XIB == 2) me.get(sXI + xb * IMG, xcur);
        if constexpr (L::EMIS) me.emis(bb, ocur);
        const bool is_init = act && t == T - 1;
        const bool on = act && t < T - 1;
        if (is_init) {
#pragma unroll
          for (int i = 0; i < COLS; ++i) bt[i] = 1.f;
          c = w / st.S_last;
        } else if (on) {
          c = w / (c * rho_prev);
        }
        const bool live = (is_init || on) && isfinite(c);
        const float fc = exp2i(-gcur) * c;  // exact: c times a power of two
        const float2 c2 = make_float2(c, c), fc2 = make_float2(fc, fc);
        float2 part2 = make_float2(0.f, 0.f);
        uint32_t gp[COLS / 2], yp[COLS / 2];
#pragma unroll
        for (int q = 0; q < COLS / 2; ++q) {
          const float2 bt2 = make_float2(bt[2 * q], bt[2 * q + 1]);
          const float2 g = __fmul2_rn(unpack_bf16(xcur[q]), bt2);
          part2 = __fadd2_rn(part2, g);
          float2 ga = __fmul2_rn(g, c2);
          float2 ya = __fmul2_rn(__fmul2_rn(make_float2(bb[2 * q], bb[2 * q + 1]), bt2), fc2);
          if (!live) { ga = make_float2(0.f, 0.f); ya = ga; }
          if (t == 0) __stcg(reinterpret_cast<float2*>(gbuf + (size_t)row * NP + me.col0 + 2 * q), ga);
          gp[q] = tc::pack_bf16(ga.x, ga.y);
          yp[q] = tc::pack_bf16(ya.x, ya.y);
        }
        me.put(sY, yp);
        me.put(sG, gp);
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
        psum[((t & 1) * TPR + h) * 128 + row] = live ? part2.x + part2.y : 0.f;
        if (!live) c = 0.f;
        // next step's inputs
        if (t > t0) {
          ocur = sym_at(t - 1);
          gcur = (int)__ldcg(gexp + (size_t)(t - 1) * 128 + row);
          if constexpr (XIB == 1) me.get_global(img_of(t - 1), xcur);
          if constexpr (!L::EMIS) me.emis(bb, ocur);
        }
        tc::fence_proxy_async();
        cb_pending = true;
      }
      if (stop) break;
      // the segment's last emission product, before gamma's buffer is reused
      tc::fence_before_sync();
      __syncthreads();
      if (misc[M_ABORT]) { stop = true; break; }
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
      wait_mma();
    }
    if (stop) break;
    tc::fence_before_sync();
    __syncthreads();
    if (misc[M_ABORT]) break;
    tc::fence_after_sync();

    // ---------------- tile counts -> slot ----------------
    float* slot = a.slots + (size_t)tile * a.slot_floats;
    if (wq * 32 < NP) {  // xi rows i = row (warp-uniform)
      float v[COLS];
      if (Lt >= 2) {
        tmem_ld_cols<COLS>(xi_tm + my_cols, v);
      } else {
#pragma unroll
        for (int i = 0; i < COLS; ++i) v[i] = 0.f;
      }
      const float4* a4 = reinterpret_cast<const float4*>(Ak + (size_t)row * NP + me.col0);
      float4* d4 = reinterpret_cast<float4*>(slot + NP + (size_t)row * NP + me.col0);
#pragma unroll
      for (int q = 0; q < COLS / 4; ++q) {
        const float4 av = __ldg(a4 + q);
        d4[q] = make_float4(v[4 * q] * av.x, v[4 * q + 1] * av.y, v[4 * q + 2] * av.z,
                            v[4 * q + 3] * av.w);
      }
    }
#pragma unroll
    for (int b = 0; b < MB; ++b) {
      float v[COLS];
      tmem_ld_cols<COLS>(cb_tm + (uint32_t)(b * NP) + my_cols, v);
      const int sym = b * 128 + row;
      if (sym < M) {
        float* dst = slot + NP + (size_t)NP * NP + sym;
#pragma unroll
        for (int jj = 0; jj < COLS; ++jj) dst[(size_t)(me.col0 + jj) * M] = v[jj];
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
  __syncthreads();
  if (tid == 0) {
    if (misc[M_ABORT]) set_status(a.status, HMM_STATUS_TIMEOUT);
    if (m_pend) tc::mbar_wait_bounded(mbar, m_par, kFbWaitLimit);
    if (g_pend) tc::mbar_wait_bounded(gbar, g_par, kFbWaitLimit);
    for (int b = 0; b < XIB; ++b)
      if (x_pend[b]) tc::mbar_wait_bounded(&xbar[b], x_par[b], kFbWaitLimit);
    tc::bulk_wait_all();
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
  return (NP == 64 || NP == 128) && fb_mma_blocks(M) <= 2;
}

int fb_mma_ctas_per_sm(int, int) { return 1; }

cudaError_t launch_fb_mma(int NP, int M, int grid, const MmaFbLaunch& a, cudaStream_t st) {
  const int mb = fb_mma_blocks(M);
  if (NP == 64 && mb == 1) return launch_fb_mma_t<64, 1>(grid, a, st);
  if (NP == 64 && mb == 2) return launch_fb_mma_t<64, 2>(grid, a, st);
  if (NP == 128 && mb == 1) return launch_fb_mma_t<128, 1>(grid, a, st);
  if (NP == 128 && mb == 2) return launch_fb_mma_t<128, 2>(grid, a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
