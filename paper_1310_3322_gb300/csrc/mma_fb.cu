// mma_fb.cu -- the second kernel of the forward-backward adjoint on the tensor
// cores for N = 64 or 128 states (Sec. 2.7 "Baum-Welch", its E-step; Rabiner
// 1989 eqs. 24-25 backward variable, 37 xi, 38 gamma), the tensor-core twin
// of fb_seg.cu's segment kernel.
//
// A tile is 128 (sequence, model) pairs of ONE model (the plan kernel groups
// them, rows sorted by decreasing length bucket; the tile runs for its longest
// row Lt), cut into NS checkpoint segments of C steps. The pass kernel
// (mma_pass.cu) has run the tile's forward recursion, keeping alpha at every
// segment start and every step's scale exponent, and its backward recursion,
// keeping the backward operand Y at every segment start. A work item here is
// one RANGE of consecutive segments of one tile (the plan's range items), so
// the segments of a long tile are processed side by side on many SMs instead
// of as one chain. Per time step every product is a dense contraction over the
// tile's 128 rows or over the states:
//   forward    D[m][j]  = sum_i X_{t-1}[m][i] a_ij         (M=128, N=NP, K=NP)
//   backward   D[m][i]  = sum_j Y_{t+1}[m][j] a_ij         (M=128, N=NP, K=NP)
//   xi         XI[i][j] += sum_m X_t[m][i] Y_{t+1}[m][j]   (M=128, N=NP, K=128 rows)
//   emissions  CB[k][j] += sum_m [o_t(m) = k] G_t[m][j]    (M=128 symbols, N=NP, K=128)
// all as tcgen05.mma kind::f16 (BF16 operands in shared memory, FP32
// accumulators in tensor memory). X, Y and G are stored once per step as
// 128 x NP BF16 "row images" (row m contiguous in 8-column groups); the same
// bytes are the K-major operand of the per-row products and the MN-major
// operand of the contractions over rows, so no operand is ever transposed.
// XI and CB accumulate over the whole item in tensor memory and are written
// once per item to the item's slot; the slots are summed in a fixed order
// (bitwise reproducible). At N = 64 the xi product uses M = 128 with rows
// 64..127 of the A operand running into the next buffer: those accumulator
// rows are never read.
//
// Per segment (from the range's last to its first): the X images of the
// segment are recomputed from its checkpoint with the pass kernel's exponents
// (the same rounding as the pass: X_t = bf16(D_t . b(o_t) . 2^-f_t)), then the
// backward recursion runs over it. With Bt_t = A Y_{t+1} (Bt_{T-1} = 1):
//   G_t = X_t . Bt_t . c_t,    Y_t = b(o_t) . Bt_t . 2^-f_t . c_t,
// with c_{T-1} = w / sigma_{T-1} (sigma from the pass) and
// c_t = w / (c_{t+1} rho_{t+1}), rho_t = sum_i X_t(i) Bt_t(i). In exact
// arithmetic rho_t = c_{t+1} rho_{t+1}, so every step's gamma sums to the row
// weight w; using the previous step's measured sum keeps the BF16 rounding of
// one step from accumulating over T (no extra barrier per step).
// A range that ends before its tile's last segment starts from the pass
// kernel's Y at its end, t1 = (last segment + 1) C, which carries an arbitrary
// scale per row: one extra product D = Y_{t1} A^T gives
// rho = sum_i X_{t1-1}(i) D(i), Y_{t1} is rescaled in place by w / rho, and
// the recursion continues with c = 1 -- step t1 - 1 then looks exactly as if
// the recursion had come from the sequence's end. (Rows whose last step lies
// inside the range start there from Bt = 1, as in any range.)
//
// Ordering per backward step (single-buffered operands): the step's MMAs are
// issued as [emissions of step t+1, xi of step t, backward of step t] under
// one commit, so when the epilogue of step t starts every operand buffer is
// free to be rewritten (N = 64: beta first on double-buffered operand sets).
// Every mbarrier wait is bounded; on timeout the kernel sets
// HMM_STATUS_TIMEOUT, waits (bounded) for its own MMAs and copies and leaves.
#include "hmm_internal.cuh"
#include "mma_rows.cuh"
#include "tc.cuh"

namespace hmmgb {

template <int NP, int MB>
struct MmaFbCfg {
  // four epilogue threads per row (16 warps, at most 120 registers a thread)
  static constexpr int TPR = 4;
  static constexpr int NEP = 128 * TPR;          // epilogue threads
  static constexpr int NTH = NEP + 32;           // + the control warp (MMAs and copies)
  static constexpr int COLS = NP / TPR;          // columns per epilogue thread (16 or 32)
  static constexpr int SUB = 16;                 // columns per tensor-memory load
  static constexpr int NSUB = COLS / SUB;
  static constexpr int IMG = 128 * NP * 2;       // one 128-row BF16 image
  static constexpr int MAT = NP * NP * 2;        // the BF16 transition image
  static constexpr bool EMIS = (NP == 64 && MB == 1);  // emission table in shared memory
  static constexpr bool DB = (NP == 64 && MB == 1);    // two operand sets: beta issued first
  static constexpr int NB = DB ? 2 : 1;                // Y / gamma / one-hot sets
  static constexpr int XIB = DB ? 3 : 2;         // X_t buffers (DB: loaded two steps ahead)
  static constexpr int ES = NP * 2 + 16;         // padded BF16 emission row (bytes)
  static constexpr int OFF_AT = 0;               // (n=j, k=i) = a_ij: forward K-major, backward MN-major
  static constexpr int OFF_XI = MAT;             // X_t images (xi A operand; epilogue rows)
  static constexpr int OFF_Y = OFF_XI + XIB * IMG;     // Y_t sets
  static constexpr int OFF_G = OFF_Y + NB * IMG;       // gamma_t sets
  static constexpr int OFF_OH = OFF_G + NB * IMG;      // one-hot [k][m] sets, MB blocks of 128 x 128
  static constexpr int OFF_XOP = OFF_OH + NB * MB * 32768;  // forward X operand (else aliases gamma)
  static constexpr int OFF_B = OFF_XOP + (DB ? IMG : 0);    // emission rows b(k), k < 128 (EMIS)
  static constexpr int NBAR = 11;                // mbarriers (see the kernel)
  static constexpr int OFF_BAR = OFF_B + (EMIS ? 128 * ES : 0);
  static constexpr int OFF_MISC = OFF_BAR + 128;
  static_assert(NBAR * 8 <= OFF_MISC - OFF_BAR, "mbarrier area");
  static constexpr int TOTAL = OFF_MISC + 64;
  static constexpr int XOP = DB ? OFF_XOP : OFF_G;
  static constexpr int TMEM_USED = (2 + MB) * NP;  // D, XI, CB blocks
  static constexpr int TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
};
static_assert(MmaFbCfg<128, 2>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<128, 1>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<64, 1>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<64, 2>::TOTAL <= 227 * 1024, "shared memory budget");
static_assert(MmaFbCfg<128, 2>::TMEM_USED <= 512, "tensor memory budget");

constexpr uint32_t kFbWaitLimit = 1u << 24;  // polls of the drain waits after an abort


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

// Per-thread view of one tile row: the row, its column range (in sub-chunks
// of SUB columns) and where its emission rows come from.
template <int NP, int MB>
struct FbThread {
  using L = MmaFbCfg<NP, MB>;
  static constexpr int SUB = L::SUB;
  int row, col0;
  const uint8_t* sB;   // shared emission table (EMIS)
  const float* Bk;     // global emission table of the model [M][NP]
  const uint16_t* Bk16;  // the same as BF16 bits

  // b_j(sym) for this thread's columns: sub-chunk `sub` from the shared BF16
  // table, or all of them from memory (prefetched a step ahead)
  __device__ __forceinline__ void emis_sub(float (&b)[SUB], int sym, int sub) const {
    const uint4* p = reinterpret_cast<const uint4*>(sB + sym * L::ES + (col0 + sub * SUB) * 2);
#pragma unroll
    for (int q = 0; q < SUB / 8; ++q) {
      const uint4 v = p[q];
      const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        b[8 * q + 2 * i] = __uint_as_float(u[i] << 16);
        b[8 * q + 2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
      }
    }
  }
  // This thread's COLS columns of emission row `sym` from the BF16 table in
  // memory (the emission values of the BF16 path are BF16 numbers), in two
  // halves so the loads' latency hides behind the next MMA wait: emis_load
  // at the end of a step, emis_ready after the next step's wait. The 32
  // lanes of a warp are 32 rows with unrelated symbols, so a per-lane load
  // would touch 32 cache lines per warp instruction. Instead the Q = COLS / 16
  // lanes of a group load the Q rows of the group in turn, 32 contiguous
  // bytes (16 values) per lane, and a Q x Q butterfly transpose within the
  // group (element = 8 words) hands every lane its own row. Every lane of the
  // warp must call both (full-warp shuffles).
  static constexpr int QE = L::COLS / 16;
  __device__ __forceinline__ void emis_load(uint32_t (&w)[L::COLS / 2], int sym) const {
    const int lane = threadIdx.x & 31, j = lane & (QE - 1);
#pragma unroll
    for (int i = 0; i < QE; ++i) {
      const int si = QE > 1 ? __shfl_sync(HMM_FULL_MASK, sym, (lane & ~(QE - 1)) | i) : sym;
      const uint16_t* p = Bk16 + (size_t)si * NP + col0 + 16 * j;  // 32-byte aligned
      asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(w[8 * i]), "=r"(w[8 * i + 1]), "=r"(w[8 * i + 2]), "=r"(w[8 * i + 3]),
                     "=r"(w[8 * i + 4]), "=r"(w[8 * i + 5]), "=r"(w[8 * i + 6]), "=r"(w[8 * i + 7])
                   : "l"(p));
    }
  }
  __device__ __forceinline__ void emis_ready(uint32_t (&w)[L::COLS / 2], float (&b)[L::COLS]) const {
    const int j = threadIdx.x & (QE - 1);
    // lane j holds piece j of rows 0..Q-1 of the group; swap the lane bit and
    // the row bit, one bit at a time, so that lane j holds row j's pieces
#pragma unroll
    for (int bit = 1; bit < QE; bit <<= 1) {
      const bool hi = (j & bit) != 0;
#pragma unroll
      for (int i0 = 0; i0 < QE; ++i0) {
        if (i0 & bit) continue;
        const int i1 = i0 | bit;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t y =
              __shfl_xor_sync(HMM_FULL_MASK, hi ? w[8 * i0 + e] : w[8 * i1 + e], bit);
          if (hi) w[8 * i0 + e] = y;
          else w[8 * i1 + e] = y;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < L::COLS / 2; ++k) {
      b[2 * k] = __uint_as_float(w[k] << 16);
      b[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
  // sub-chunk `sub` of this thread's columns of a row image (BF16 pairs)
  __device__ __forceinline__ uint32_t off(int sub, int c) const {
    return img_off<NP>(row, (col0 + sub * SUB) / 8 + c);
  }
  __device__ __forceinline__ void put(uint8_t* img, int sub, const uint32_t (&w)[SUB / 2]) const {
#pragma unroll
    for (int c = 0; c < SUB / 8; ++c)
      *reinterpret_cast<uint4*>(img + off(sub, c)) =
          make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
  }
  __device__ __forceinline__ void put_global(uint8_t* img, int sub, const uint32_t (&w)[SUB / 2]) const {
#pragma unroll
    for (int c = 0; c < SUB / 8; ++c)
      __stcg(reinterpret_cast<uint4*>(img + off(sub, c)),
             make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]));
  }
  __device__ __forceinline__ void get(const uint8_t* img, int sub, uint32_t (&w)[SUB / 2]) const {
#pragma unroll
    for (int c = 0; c < SUB / 8; ++c) {
      const uint4 v = *reinterpret_cast<const uint4*>(img + off(sub, c));
      w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
    }
  }
};

// Forward step epilogue: y = D . b . 2^-f (zero when not live), packed into
// the operand image; returns the partial row sum.
template <int COLS>
__device__ __forceinline__ float fwd_epilogue(float (&y)[COLS], const float* b, int f, bool live,
                                              uint32_t (&w)[COLS / 2]) {
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

// Bounded mbarrier wait (`limit` polls, the first one never suspending the
// thread; 0: none) that also gives up once another thread has recorded an
// abort; a timeout records one.
__device__ __forceinline__ bool fb_wait(uint64_t* bar, uint32_t parity,
                                        volatile int32_t* abort_flag, uint32_t limit) {
  if (limit > 0 && tc::mbar_probe(bar, parity)) return true;
  for (uint32_t i = 1; i < limit; ++i) {
    if (tc::mbar_test(bar, parity)) return true;
    if ((i & 31) == 31 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// One-hot entry (symbol k, row m) of a 128-column block set.
__device__ __forceinline__ uint16_t* onehot_at(uint8_t* set, int k, int m) {
  return reinterpret_cast<uint16_t*>(set + (k >> 7) * 32768 + img_off<128>(k & 127, m >> 3) +
                                     (m & 7) * 2);
}

template <int NP, int MB>
__global__ void __launch_bounds__(MmaFbCfg<NP, MB>::NTH, 1) hmm_fb_mma(MmaFbLaunch a) {
  using L = MmaFbCfg<NP, MB>;
  constexpr int TPR = L::TPR, NEP = L::NEP, IMG = L::IMG, COLS = L::COLS, XIB = L::XIB;
  constexpr int NB = L::NB;
  constexpr bool DB = L::DB;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAT = smem + L::OFF_AT;
  uint8_t* sXI = smem + L::OFF_XI;
  uint8_t* sY = smem + L::OFF_Y;
  uint8_t* sG = smem + L::OFF_G;
  uint8_t* sOH = smem + L::OFF_OH;
  uint8_t* sXO = smem + L::XOP;
  // row partial sums [2][TPR][128], per CTA in memory (L2): written at a
  // step's end, read at the next step's start and needed only after its MMA
  // wait, so the loads' latency hides behind that wait
  float* psum = a.psum + (size_t)blockIdx.x * 2 * TPR * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint64_t* b_rdy = bars + 0;    // epilogue -> control: operands written
  uint64_t* b_done = bars + 1;   // the products the epilogue waits for
  uint64_t* b_aux = bars + 2;    // [2] xi (+ emission) products of even / odd steps: control only
  uint64_t* b_seg = bars + 4;    // segment-end emission product: control only
  uint64_t* b_g = bars + 5;      // checkpoint -> forward operand
  uint64_t* b_x = bars + 6;      // [XIB] X_t images
  uint64_t* b_fin = bars + 9;    // teardown after an abort
  uint64_t* b_y = bars + 10;     // Y checkpoint -> backward operand (a range's start)
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);
  enum { M_TMEM = 0, M_ITEM = 1, M_ABORT = 2 };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ctrl = warp == NEP / 32;
  const int wq = warp & 3, h = (warp >> 2) & 3;
  const int K = a.seq.K, M = a.seq.M;
  FbThread<NP, MB> me;
  me.row = wq * 32 + lane;
  me.col0 = h * COLS;
  me.sB = smem + L::OFF_B;
  const int row = me.row;

  for (int i = tid; i < NB * MB * 32768 / 16; i += L::NTH)
    reinterpret_cast<uint4*>(sOH)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), L::TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < L::NBAR; ++i) tc::mbar_init(&bars[i], 1);
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
  const uint32_t aAT = tc::smem_u32(sAT), aXI = tc::smem_u32(sXI), aXO = tc::smem_u32(sXO);
  const uint32_t aY = tc::smem_u32(sY), aG = tc::smem_u32(sG), aOH = tc::smem_u32(sOH);
  constexpr uint32_t SBO = NP * 16;

  uint8_t* scr = a.scr + (size_t)blockIdx.x * a.scr_bytes;
  float* gbuf = a.gbuf + (size_t)blockIdx.x * 128 * NP;

  // barrier phases: the epilogue threads track b_done and b_x, the control
  // lane every barrier it waits on (each waiter waits every phase, in order)
  uint32_t ph_done = 0, ph_xb = 0;  // ph_xb bit b: the phase of X buffer b
  uint32_t c_rdy = 0, c_aux[2] = {0, 0}, c_seg = 0, c_g = 0, c_y = 0;
  // per X buffer b (bit b): the parity the next load into it completes, that
  // of the last one issued, and whether that one is still unwaited
  uint32_t c_xb = 0, c_xparb = 0, c_xpendb = 0;
  bool c_gpend = false, c_ypend = false;
  uint32_t c_gpar = 0, c_ypar = 0;
  int cur_model = -1;
  volatile int32_t* abortp = misc + M_ABORT;

  for (;;) {
    __syncthreads();
    if (tid == 0) misc[M_ITEM] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = misc[M_ITEM];
    if (item >= __ldcg(a.n_rng) || misc[M_ABORT]) break;
    const int tile = a.rng_tile[item];
    const int seg_lo = a.rng_seg[item] & 0xffff, seg_hi = a.rng_seg[item] >> 16;
    const int k = a.tile_model[tile];
    const int start = a.tile_start[tile];
    const int nrows = a.tile_rows[tile];
    const int Lt = a.tile_len[tile];
    const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
    me.Bk = a.mod.Btp + (size_t)k * M * NP;
    me.Bk16 = a.mod.Btp16 + (size_t)k * M * NP;
    if (k != cur_model) {
      // transition image: (n = j, k = i) = a_ij, pairs along i
      for (int idx = tid; idx < NP * NP / 2; idx += L::NTH) {
        const int j = idx / (NP / 2), i = (idx % (NP / 2)) * 2;
        const uint32_t w = tc::pack_bf16(__ldg(Ak + i * NP + j), __ldg(Ak + (i + 1) * NP + j));
        *reinterpret_cast<uint32_t*>(sAT + (j / 8) * SBO + (i / 8) * 128 + (j % 8) * 16 +
                                     (i % 8) * 2) = w;
      }
      if constexpr (L::EMIS) {  // the model's BF16 emission rows, padded
        for (int idx = tid; idx < M * (NP / 8); idx += L::NTH) {
          const int sym = idx / (NP / 8), q = idx % (NP / 8);
          *reinterpret_cast<uint4*>(smem + L::OFF_B + sym * L::ES + q * 16) =
              __ldg(reinterpret_cast<const uint4*>(me.Bk16 + (size_t)sym * NP) + q);
        }
      }
      cur_model = k;
      tc::fence_proxy_async();
      __syncthreads();
    }
    const int C = fb_mma_segment(Lt);
    const int NS = (Lt + C - 1) / C;
    // a range that stops short of the tile's last segment restarts the
    // backward recursion from the pass kernel's Y checkpoint at its end
    const bool cont = seg_hi < NS - 1;
    const uint8_t* ckx = a.ckx + (size_t)tile * a.ck_stride;
    const uint8_t* cky = a.cky + (size_t)tile * a.ck_stride;
    const int8_t* gexp = a.gexp + (size_t)tile * a.gexp_stride;

    if (ctrl) {
      // ======================= control lane: every MMA and copy =======================
      if (lane == 0) {
        bool ok = true;
        auto wait_c = [&](uint64_t* bar, uint32_t& ph) {
          ok = ok && fb_wait(bar, ph, abortp, a.wait_limit);
          ph ^= 1;
          return ok;
        };
        auto issue_fwd = [&]() {  // D = X_op . A
          tc::fence_after_sync();
#pragma unroll
          for (int ks = 0; ks < NP / 16; ++ks)
            tc::mma_bf16(d_tm, tc::smem_desc(aXO + ks * 256, 128, SBO),
                         tc::smem_desc(aAT + ks * 256, 128, SBO), id_kk, ks > 0 ? 1u : 0u);
          tc::mma_commit(b_done);
        };
        auto load_x = [&](int t, const uint8_t* src) {
          const int b = t % XIB;
          tc::mbar_arrive_expect_tx(&b_x[b], IMG);
          tc::bulk_g2s(aXI + b * IMG, src, IMG, &b_x[b]);
          // the epilogue waits for it too; the last step's load is waited
          // for by the epilogue alone
          c_xpendb |= 1u << b;
          c_xparb = (c_xparb & ~(1u << b)) | (c_xb & (1u << b));
          c_xb ^= 1u << b;
        };
        bool xi_on = false, cb_on = false;
        // the xi / emission products of step t are committed to b_aux[t % 2]:
        // one outstanding phase per barrier at most
        bool aux_pend[2] = {false, false};
        auto wait_aux = [&](int b) {
          if (aux_pend[b] && ok) { wait_c(&b_aux[b], c_aux[b]); aux_pend[b] = false; }
        };
        for (int seg = seg_hi; seg >= seg_lo && ok; --seg) {
          const int t0 = seg * C, t1 = min(t0 + C, Lt);
          const uint8_t* ck = ckx + (size_t)seg * IMG;
          auto img_of = [&](int t) -> const uint8_t* {
            return t == t0 ? ck : scr + (size_t)(t - t0) * IMG;
          };
          const bool restart = seg == seg_hi && cont;
          if (restart) {  // Y_{t1} of the pass kernel into the operand set of step t1
            tc::mbar_arrive_expect_tx(b_y, IMG);
            tc::bulk_g2s(aY + (t1 % NB) * IMG, cky + (size_t)(seg + 1) * IMG, IMG, b_y);
            c_ypend = true;
            c_ypar = c_y;
          }
          if (t1 - t0 > 1) {  // recompute from the checkpoint
            tc::mbar_arrive_expect_tx(b_g, IMG);
            tc::bulk_g2s(aXO, ck, IMG, b_g);
            c_gpend = true;
            c_gpar = c_g;
            if (!wait_c(b_g, c_g)) break;
            c_gpend = false;
            for (int t = t0 + 1; t < t1 && ok; ++t) {
              if (t > t0 + 1 && !wait_c(b_rdy, c_rdy)) break;
              issue_fwd();
            }
            if (!ok || !wait_c(b_rdy, c_rdy)) break;  // images of the segment in memory
          }
          // backward: X images XIB - 1 steps ahead
          load_x(t1 - 1, img_of(t1 - 1));
          if (XIB == 3 && t1 - 2 >= t0) load_x(t1 - 2, img_of(t1 - 2));
          if (restart) {
            // D = Y_{t1} . A^T once, for the epilogue's renormalisation of Y_{t1}
            if (!wait_c(b_y, c_y)) break;
            c_ypend = false;
            tc::fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < NP / 16; ++ks)
              tc::mma_bf16(d_tm, tc::smem_desc(aY + (t1 % NB) * IMG + ks * 256, 128, SBO),
                           tc::smem_desc(aAT + ks * 32 * NP, NP * 16, 128), id_km,
                           ks > 0 ? 1u : 0u);
            tc::mma_commit(b_done);
            if (!wait_c(b_rdy, c_rdy)) break;  // Y_{t1} rescaled in place
          }
          bool cb_pending = false;
          for (int t = t1 - 1; t >= t0 && ok; --t) {
            const int S1 = (t + 1) % NB;  // operand set written by the previous step
            if (t < Lt - 1) {
              if (t < t1 - 1 && !wait_c(b_rdy, c_rdy)) break;
              tc::fence_after_sync();
              auto issue_beta = [&]() {  // D = Y_{t+1} . A^T (transition image MN-major)
#pragma unroll
                for (int ks = 0; ks < NP / 16; ++ks)
                  tc::mma_bf16(d_tm, tc::smem_desc(aY + S1 * IMG + ks * 256, 128, SBO),
                               tc::smem_desc(aAT + ks * 32 * NP, NP * 16, 128), id_km,
                               ks > 0 ? 1u : 0u);
              };
              auto issue_xi_cb = [&]() {
                const int xb = t % XIB;
                uint32_t par = (c_xparb >> xb) & 1u;
                if (!wait_c(&b_x[xb], par)) return;
                c_xpendb &= ~(1u << xb);
                tc::fence_after_sync();
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                  tc::mma_bf16(xi_tm,
                               tc::smem_desc(aXI + (t % XIB) * IMG + ks * 32 * NP, NP * 16, 128),
                               tc::smem_desc(aY + S1 * IMG + ks * 32 * NP, NP * 16, 128), id_mm,
                               (ks > 0 || xi_on) ? 1u : 0u);
                xi_on = true;
                if (cb_pending) {
#pragma unroll
                  for (int b = 0; b < MB; ++b)
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks)
                      tc::mma_bf16(cb_tm + (uint32_t)(b * NP),
                                   tc::smem_desc(aOH + (S1 * MB + b) * 32768 + ks * 256, 128, 2048),
                                   tc::smem_desc(aG + S1 * IMG + ks * 32 * NP, NP * 16, 128),
                                   id_km, (ks > 0 || cb_on) ? 1u : 0u);
                  cb_on = true;
                }
                tc::mma_commit(&b_aux[t & 1]);
                aux_pend[t & 1] = true;
              };
              if (DB) {  // beta first: the epilogue waits for it alone
                issue_beta();
                tc::mma_commit(b_done);
                // the xi batch of step t+1 is waited for at every step (so that
                // b_aux[t & 1], which takes this step's batch, never holds two
                // unwaited phases), then the X image XIB - 1 steps ahead goes
                // into the buffer that batch read, then this step's xi /
                // emission batch
                wait_aux((t + 1) & 1);
                if (!ok) break;
                if (t - (XIB - 1) >= t0) load_x(t - (XIB - 1), img_of(t - (XIB - 1)));
                issue_xi_cb();
              } else {
                issue_xi_cb();
                issue_beta();
                tc::mma_commit(b_done);
              }
              if (!ok) break;
            }
            // the X image XIB - 1 steps ahead: its buffer was last read by
            // the xi product of step t+1
            if (t - (XIB - 1) >= t0 && !(DB && t < Lt - 1)) {
              wait_aux((t + 1) & 1);
              if (!ok) break;
              load_x(t - (XIB - 1), img_of(t - (XIB - 1)));
            }
            cb_pending = true;
          }
          if (!ok) break;
          // the segment's last emission product, before its buffers are reused
          if (!wait_c(b_rdy, c_rdy)) break;
          tc::fence_after_sync();
          const int S0 = t0 % NB;
#pragma unroll
          for (int b = 0; b < MB; ++b)
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
              tc::mma_bf16(cb_tm + (uint32_t)(b * NP),
                           tc::smem_desc(aOH + (S0 * MB + b) * 32768 + ks * 256, 128, 2048),
                           tc::smem_desc(aG + S0 * IMG + ks * 32 * NP, NP * 16, 128), id_km,
                           (ks > 0 || cb_on) ? 1u : 0u);
          cb_on = true;
          tc::mma_commit(b_seg);
          tc::mma_commit(b_done);
          wait_aux(0);
          wait_aux(1);
          wait_c(b_seg, c_seg);
          // the epilogue has consumed that phase too: a waiter on an mbarrier
          // must never fall two phases behind
          wait_c(b_rdy, c_rdy);
        }
        if (!ok) {  // nothing of ours may stay in flight
          tc::mma_commit(b_fin);  // arrives once every MMA issued so far is done
          tc::mbar_wait_bounded(b_fin, 0, kFbWaitLimit);
          if (c_gpend) tc::mbar_wait_bounded(b_g, c_gpar, kFbWaitLimit);
          if (c_ypend) tc::mbar_wait_bounded(b_y, c_ypar, kFbWaitLimit);
          for (int b = 0; b < XIB; ++b)
            if ((c_xpendb >> b) & 1u)
              tc::mbar_wait_bounded(&b_x[b], (c_xparb >> b) & 1u, kFbWaitLimit);
        }
      }
      __syncwarp();
    } else {
      // ======================= epilogue warps =======================
      constexpr int SUB = L::SUB, NSUB = L::NSUB;
      const bool has = row < nrows;
      const int s = has ? a.sorted[start + row] : 0;
      const int T = has ? a.seq.seqlen[s] : 0;
      const size_t oidx = a.labelled ? (size_t)s : (size_t)s * K + k;
      const float w = has ? (a.weight ? a.weight[oidx] : 1.f) : 0.f;
      const int32_t* o = a.seq.symbols + (has ? a.seq.offsets[s] : 0);
      // the pass kernel's row sum at the row's last step: 0 = no counts
      // (impossible sequence), NaN = invalid row
      const float s_last = a.s_last[(size_t)tile * 128 + row];
      // symbols: the load of step t (0 past the row's end) is issued a step or
      // two before its use and range-checked only at the use, so that no
      // instruction waits for it in between
      auto sym_raw = [&](int t) -> int { return t < T ? __ldg(o + t) : 0; };
      auto sym_ok = [&](int v) -> int { return (unsigned)v < (unsigned)M ? v : 0; };
      auto wait_e = [&](uint64_t* bar, uint32_t& ph) {
        fb_wait(bar, ph, abortp, a.wait_limit);
        ph ^= 1;
        tc::fence_after_sync();
      };
      // all epilogue threads: operands written -> tell the control lane;
      // returns false (in every thread) once anyone has recorded an abort
      auto handoff = [&]() -> bool {
        tc::fence_before_sync();
        const bool go = tc::bar_and(1, NEP, *abortp == 0);
        if (go && tid == 0) tc::mbar_arrive(b_rdy);
        return go;
      };
      auto row_sum = [&](int par) {
        float sum = 0.f;
#pragma unroll
        for (int q = 0; q < TPR; ++q) sum += __ldcg(psum + (par * TPR + q) * 128 + row);
        return sum;
      };
      // one forward step's epilogue over this thread's columns: D (tensor
      // memory) -> X_t (operand image, and `gimg` in memory when not null)
      float pf[L::EMIS ? 1 : COLS];  // emission values prefetched from memory
      uint32_t pw[L::EMIS ? 1 : COLS / 2];  // their BF16 words in flight
      float bsm[SUB];                // emission values from the shared table (EMIS)
      auto fwd_step = [&](int f, bool live, uint8_t* gimg) -> float {
        float sum = 0.f;
#pragma unroll
        for (int sub = 0; sub < NSUB; ++sub) {
          float y[SUB];
          tmem_ld_cols<SUB>(d_tm + my_cols + (uint32_t)(sub * SUB), y);
          uint32_t wv[SUB / 2];
          sum += fwd_epilogue<SUB>(y, L::EMIS ? bsm : pf + sub * SUB, f, live, wv);
          me.put(sXO, sub, wv);
          if (gimg) me.put_global(gimg, sub, wv);
        }
        return sum;
      };
      bool run = true;
      const bool act = has && w != 0.f && s_last > 0.f && !isinf(s_last);
      float c = 0.f;               // this row's current normaliser
      // one-hot entries set in each operand set (two registers: an array
      // indexed by the step's parity would live in local memory)
      int kprev0 = -1, kprev1 = -1;
      for (int seg = seg_hi; seg >= seg_lo && run; --seg) {
        const int t0 = seg * C, t1 = min(t0 + C, Lt);
        // (R) recompute X over the segment from its checkpoint
        if (t1 - t0 > 1) {
          // symbol and exponent of steps t + 1 and t + 2 in flight
          int fn = (int)__ldcg(gexp + (size_t)(t0 + 1) * 128 + row);
          int on = sym_ok(sym_raw(t0 + 1));
          int fn2 = t0 + 2 < t1 ? (int)__ldcg(gexp + (size_t)(t0 + 2) * 128 + row) : 0;
          int on2 = t0 + 2 < t1 ? sym_raw(t0 + 2) : 0;
          if constexpr (!L::EMIS) me.emis_load(pw, on);
          for (int t = t0 + 1; t < t1 && run; ++t) {
            const int f = fn;
            const int ot = on;
            fn = fn2;
            on = sym_ok(on2);
            if (t + 2 < t1) {
              fn2 = (int)__ldcg(gexp + (size_t)(t + 2) * 128 + row);
              on2 = sym_raw(t + 2);
            }
            if constexpr (L::EMIS) me.emis_sub(bsm, ot, 0);
            wait_e(b_done, ph_done);
            if constexpr (!L::EMIS) {
              me.emis_ready(pw, pf);
              // the next step's rows, in flight during this epilogue
              if (t + 1 < t1) me.emis_load(pw, on);
            }
            fwd_step(f, act && t < T, scr + (size_t)(t - t0) * IMG);
            tc::fence_proxy_async();
            if (t == t1 - 1) tc::fence_proxy_async_all();  // images read by bulk copies
            run = handoff();
          }
          if (!run) break;
        }

        // (P) a range's restart: D = Y_{t1} A^T from the pass kernel's
        // checkpoint of Y_{t1} (any positive scale per row). With
        // rho = sum_i X_{t1-1}(i) D(i), Y_{t1} <- Y_{t1} w / rho makes step
        // t1 - 1 normalised as if the recursion had come from the sequence's
        // end (its gamma and xi then sum to w, and c = 1); rows whose last
        // step lies in this range start there instead and take no Y_{t1}.
        if (seg == seg_hi && cont) {
          const int SX = (t1 - 1) % XIB, S1 = t1 % NB;
          // the first backward step waits for the same X image phase again
          fb_wait(&b_x[SX], (ph_xb >> SX) & 1u, abortp, a.wait_limit);
          wait_e(b_done, ph_done);
          float part = 0.f;
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            float dv[SUB];
            tmem_ld_cols<SUB>(d_tm + my_cols + (uint32_t)(sub * SUB), dv);
            uint32_t xw[SUB / 2];
            me.get(sXI + SX * IMG, sub, xw);
#pragma unroll
            for (int q = 0; q < SUB / 2; ++q) {
              const float2 xv = unpack_bf16(xw[q]);
              part = fmaf(xv.x, dv[2 * q], fmaf(xv.y, dv[2 * q + 1], part));
            }
          }
          // partial sums in the slot of step t1 - 1 (the first backward step
          // then writes and reads the slot of step t1)
          const int PS = (t1 - 1) & 1;
          psum[(PS * TPR + h) * 128 + row] = part;
          tc::bar_sync(1, NEP);
          const float rho = row_sum(PS);
          const bool controw = act && T > t1;
          float kappa = controw ? w / rho : 0.f;
          if (!(rho > 0.f) || !isfinite(kappa)) kappa = 0.f;
          const float2 k2 = make_float2(kappa, kappa);
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            uint32_t yw[SUB / 2];
            me.get(sY + S1 * IMG, sub, yw);
#pragma unroll
            for (int q = 0; q < SUB / 2; ++q) {
              const float2 v = __fmul2_rn(unpack_bf16(yw[q]), k2);
              yw[q] = tc::pack_bf16(v.x, v.y);
            }
            me.put(sY + S1 * IMG, sub, yw);
          }
          // the first backward step reads c_{t1} rho_{t1} = w (c = 1)
          psum[(((t1 & 1) * TPR) + h) * 128 + row] = (h == 0 && kappa != 0.f) ? w : 0.f;
          c = kappa != 0.f ? 1.f : 0.f;
          tc::fence_proxy_async();
          run = handoff();
          if (!run) break;
        }

        // (B) backward over the segment
        int ocur = sym_ok(sym_raw(t1 - 1)), gcur = (int)__ldcg(gexp + (size_t)(t1 - 1) * 128 + row);
        int onx = t1 - 2 >= t0 ? sym_raw(t1 - 2) : 0;  // step t - 1, in flight
        int gnx = t1 - 2 >= t0 ? (int)__ldcg(gexp + (size_t)(t1 - 2) * 128 + row) : 0;
        if constexpr (!L::EMIS) me.emis_load(pw, ocur);
        for (int t = t1 - 1; t >= t0 && run; --t) {
          const bool has_mma = t < Lt - 1;
          const int S = t % NB;
          const float rho_prev = row_sum((t + 1) & 1);
          if constexpr (L::EMIS) me.emis_sub(bsm, ocur, 0);
          {
            const int xb = t % XIB;
            uint32_t px = (ph_xb >> xb) & 1u;
            wait_e(&b_x[xb], px);
            ph_xb ^= 1u << xb;
          }
          // this step's X image is in shared memory now and its copy in memory
          // (checkpoint or recomputed image) is never read again: drop its
          // L2 lines instead of letting them be written back
          if (tid < IMG / 128)
            tc::discard_l2((t == t0 ? ckx + (size_t)seg * IMG : scr + (size_t)(t - t0) * IMG) +
                           (size_t)tid * 128);
          if (has_mma) wait_e(b_done, ph_done);
          if constexpr (!L::EMIS) {
            me.emis_ready(pw, pf);
            // the next step's rows, in flight during this epilogue
            if (t > t0) me.emis_load(pw, sym_ok(onx));
          }
          const bool is_init = act && t == T - 1;
          const bool on = act && t < T - 1;
          if (is_init) c = w / s_last;
          else if (on) c = w / (c * rho_prev);
          const bool live = (is_init || on) && isfinite(c);
          const float fc = exp2i(-gcur) * c;  // exact: c times a power of two
          const float2 c2 = make_float2(c, c), fc2 = make_float2(fc, fc);
          float2 part2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            float bt[SUB];
            if (has_mma) {
              tmem_ld_cols<SUB>(d_tm + my_cols + (uint32_t)(sub * SUB), bt);
            } else {
#pragma unroll
              for (int i = 0; i < SUB; ++i) bt[i] = 0.f;
            }
            if (is_init) {
#pragma unroll
              for (int i = 0; i < SUB; ++i) bt[i] = 1.f;
            }
            uint32_t xw[SUB / 2];
            me.get(sXI + (t % XIB) * IMG, sub, xw);
            const float* bb = L::EMIS ? bsm : pf + sub * SUB;
            uint32_t gp[SUB / 2], yp[SUB / 2];
#pragma unroll
            for (int q = 0; q < SUB / 2; ++q) {
              const float2 bt2 = make_float2(bt[2 * q], bt[2 * q + 1]);
              const float2 g = __fmul2_rn(unpack_bf16(xw[q]), bt2);
              part2 = __fadd2_rn(part2, g);
              float2 ga = __fmul2_rn(g, c2);
              float2 ya = __fmul2_rn(__fmul2_rn(make_float2(bb[2 * q], bb[2 * q + 1]), bt2), fc2);
              if (!live) { ga = make_float2(0.f, 0.f); ya = ga; }
              if (t == 0)
                __stcg(reinterpret_cast<float2*>(gbuf + (size_t)row * NP + me.col0 + sub * SUB +
                                                 2 * q), ga);
              gp[q] = tc::pack_bf16(ga.x, ga.y);
              yp[q] = tc::pack_bf16(ya.x, ya.y);
            }
            me.put(sY + S * IMG, sub, yp);
            me.put(sG + S * IMG, sub, gp);
          }
          if (h == 0) {
            uint8_t* oh = sOH + S * MB * 32768;
            const int kp = S ? kprev1 : kprev0;
            if (kp >= 0) *onehot_at(oh, kp, row) = 0;
            if (live) *onehot_at(oh, ocur, row) = 0x3F80;  // BF16 1.0
            const int kn = live ? ocur : -1;
            if (S) kprev1 = kn;
            else kprev0 = kn;
          }
          psum[((t & 1) * TPR + h) * 128 + row] = live ? part2.x + part2.y : 0.f;
          if (!live) c = 0.f;
          // next step's inputs
          if (t > t0) {
            ocur = sym_ok(onx);
            gcur = gnx;
            if (t - 2 >= t0) {
              onx = sym_raw(t - 2);
              gnx = (int)__ldcg(gexp + (size_t)(t - 2) * 128 + row);
            }
          }
          tc::fence_proxy_async();
          run = handoff();
        }
        if (!run) break;
        wait_e(b_done, ph_done);  // the segment's last emission product
        run = handoff();
      }
      if (run) {
        // ---------------- item counts -> slot ----------------
        float* slot = a.slots + (size_t)item * a.slot_floats;
        const bool xi_any = seg_lo * C < Lt - 1;  // some xi product was issued
        if (wq * 32 < NP) {  // xi rows i = row (warp-uniform)
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            float v[SUB];
            if (xi_any) {
              tmem_ld_cols<SUB>(xi_tm + my_cols + (uint32_t)(sub * SUB), v);
            } else {
#pragma unroll
              for (int i = 0; i < SUB; ++i) v[i] = 0.f;
            }
            const int j0 = me.col0 + sub * SUB;
            const float4* a4 = reinterpret_cast<const float4*>(Ak + (size_t)row * NP + j0);
            float4* d4 = reinterpret_cast<float4*>(slot + NP + (size_t)row * NP + j0);
#pragma unroll
            for (int q = 0; q < SUB / 4; ++q) {
              const float4 av = __ldg(a4 + q);
              d4[q] = make_float4(v[4 * q] * av.x, v[4 * q + 1] * av.y, v[4 * q + 2] * av.z,
                                  v[4 * q + 3] * av.w);
            }
          }
        }
#pragma unroll
        for (int b = 0; b < MB; ++b) {
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            float v[SUB];
            tmem_ld_cols<SUB>(cb_tm + (uint32_t)(b * NP + sub * SUB) + my_cols, v);
            const int sym = b * 128 + row;
            if (sym < M) {
              float* dst = slot + NP + (size_t)NP * NP + sym;
#pragma unroll
              for (int jj = 0; jj < SUB; ++jj) dst[(size_t)(me.col0 + sub * SUB + jj) * M] = v[jj];
            }
          }
        }
        tc::bar_sync(1, NEP);
        if (tid < NP) {  // gamma_1 rows: only the range holding step 0 has them
          float sum = 0.f;
          if (seg_lo == 0)
            for (int m = 0; m < 128; ++m) sum += __ldcg(gbuf + (size_t)m * NP + tid);
          slot[tid] = sum;
        }
      }
      if (h == 0)
        for (int q = 0; q < NB; ++q) {
          const int kp = q ? kprev1 : kprev0;
          if (kp >= 0) *onehot_at(sOH + q * MB * 32768, kp, row) = 0;
        }
      tc::fence_proxy_async();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (misc[M_ABORT]) break;
    tc::fence_after_sync();
  }

  // teardown
  __syncthreads();
  if (tid == 0 && misc[M_ABORT]) set_status(a.status, HMM_STATUS_TIMEOUT);
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
