// mma_wide.cu -- scaled forward algorithm on the tensor cores for 128 < N <= 512
// states (Sec. 2.7 "Forward"; Sec. 5.6 quotes the cited forward kernel at
// 512 states x 512 sequences; Rabiner 1989 eqs. 19-21, per-step scaling).
//
// Same recursion as mma_forward.cu -- a tile of 128 (sequence, model) rows of
// one model computes D[128 x N] = X[128 x N] . A[N x N] per step, then the
// epilogue multiplies the emission row, scales by the late power of two and
// writes the next X -- but at these state counts one tile fills an SM:
//   * D (N FP32 columns, up to all 512) lives in tensor memory;
//   * X, the BF16 rescaled alpha rows, lives in shared memory as the K-major A
//     operand (128 x N x 2 bytes, up to 128 KB);
//   * A^T does not fit next to it (512 KB at N = 512): it is streamed every
//     step from a BF16 image in global memory (L2-resident, built by
//     `wide_image_kernel`) in chunks of 32 states of K, through a ring of
//     three shared-memory buffers filled by bulk copies; each chunk feeds
//     N/256 x 2 MMAs (M = 128, N = 256, K = 16);
//   * emission values are gathered from the padded table in memory, the first
//     32 columns of a step while its MMAs run, each further 32 while the
//     previous 32 are used.
// One CTA of 512 threads owns one tile (four threads per row, N/4 columns
// each); thread 0 issues the MMAs and copies, warp 1 polls the step's commit.
// Every mbarrier wait is bounded; on timeout the kernel records
// HMM_STATUS_TIMEOUT, waits (bounded) for its own copies and MMAs and leaves.
//
// This kernel serves the forward when the cluster kernel of mma_cluster.cu
// (one CTA per 64 columns, A resident) has no room for the emission table
// slice, i.e. N_pad = 512 with more than 173 symbols.
#include "hmm_internal.cuh"
#include "mma_rows.cuh"
#include "tc.cuh"

namespace hmmgb {

template <int NP>
struct WideCfg {
  static constexpr int NTH = 512;
  static constexpr int TPR = 4;              // threads per row
  static constexpr int COLS = NP / TPR;      // columns per thread
  static constexpr int CH = COLS / 32;       // 32-column chunks per thread
  static constexpr int CK = 32;              // states of K per A^T chunk
  static constexpr int NKC = NP / CK;        // chunks per step
  static constexpr int CHUNK = CK * NP * 2;  // bytes per chunk
  static constexpr int RING = 3;
  static constexpr int XB = 128 * NP * 2;    // X image
  static constexpr int OFF_X = 0;
  static constexpr int OFF_R = XB;
  static constexpr int OFF_PS = OFF_R + RING * CHUNK;          // partial row sums [TPR][128]
  static constexpr int OFF_BAR = OFF_PS + TPR * 128 * 4;  // full[RING], empty[RING], done, fin
  static constexpr int NBAR = 2 * RING + 2;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;          // tmem, item, abort, last
  static constexpr int TOTAL = OFF_MISC + 16 * 4;
  static_assert(NP % 256 == 0, "N-blocks of 256 columns");
  static_assert(TOTAL <= 227 * 1024, "shared memory budget");
};

constexpr uint32_t kWideWait = 1u << 24;  // polls of the teardown's drain waits

// BF16 image of A^T per model, chunk-major: chunk kc holds states i in
// [32 kc, 32 kc + 32) for every j, element (n = j, k = i) = a_ij at
//   (j / 8) * 512 + (il / 8) * 128 + (j % 8) * 16 + (il % 8) * 2,  il = i - 32 kc
// (K-major core matrices of 8 rows x 16 bytes; 512 = 32 K values x 16 bytes).
template <int NP>
__global__ void wide_image_kernel(const float* Ap, uint8_t* img, int K) {
  const long long n = (long long)K * NP * NP / 2;  // pairs along i
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / (NP * NP / 2));
    const int r = (int)(idx % (NP * NP / 2));
    const int i = (r / NP) * 2, j = r % NP;
    const float* Ak = Ap + (size_t)k * NP * NP;
    const int kc = i / 32, il = i % 32;
    const size_t off = (size_t)k * NP * NP * 2 + (size_t)kc * WideCfg<NP>::CHUNK +
                       (size_t)(j / 8) * 512 + (il / 8) * 128 + (j % 8) * 16 + (il % 8) * 2;
    const float v0 = Ak[(size_t)i * NP + j];
    const float v1 = Ak[(size_t)(i + 1) * NP + j];
    *reinterpret_cast<uint32_t*>(img + off) = tc::pack_bf16(v0, v1);
  }
}

// The work of one CTA (all of it: items come from a.queue until it runs dry).
template <int NP>
__device__ __forceinline__ void wide_body(const MmaWideLaunch& a) {
  using L = WideCfg<NP>;
  constexpr int COLS = L::COLS, CH = L::CH, NKC = L::NKC, RING = L::RING;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sX = smem + L::OFF_X;
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS);  // [TPR][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + RING;
  uint64_t* done = bars + 2 * RING;
  uint64_t* fin = bars + 2 * RING + 1;
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = warp >> 2;   // lane quarter, column quarter
  const int row = wq * 32 + lane;
  const int col0 = h * COLS;
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;

  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), 512);
  if (tid == 0) {
    for (int i = 0; i < L::NBAR; ++i) tc::mbar_init(&bars[i], 1);
    misc[2] = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t d_mine = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)col0;
  constexpr uint32_t idesc = tc::instr_desc(1, 128, 256);
  const uint32_t aX = tc::smem_u32(sX), aR = tc::smem_u32(smem + L::OFF_R);
  // this thread's X image bytes: row `row`, 8-column groups of its columns
  const uint32_t x_row = (uint32_t)((row / 8) * (NP * 16) + (row % 8) * 16);

  // issuer state (thread 0): every commit and copy completion is waited once
  uint32_t ph_full[RING] = {0, 0, 0}, ph_empty[RING] = {0, 0, 0};
  bool pend_full[RING] = {false, false, false}, pend_empty[RING] = {false, false, false};
  uint32_t ph_done = 0;
  bool abort_issue = false;

  for (;;) {
    __syncthreads();
    if (tid == 0) misc[1] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = misc[1];
    if (item >= a.n_items || misc[2]) break;
    const int tile = item / K, k = item % K;
    const int pos = tile * 128 + row;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    const bool bad_seq = T < 0;
    const int Tn = bad_seq ? 0 : T;
    {  // longest row of the tile: warps 0-3 hold every row once
      const int wm = __reduce_max_sync(HMM_FULL_MASK, Tn);
      if (h == 0 && lane == 0) misc[4 + wq] = wm;
    }
    __syncthreads();
    int Tmax = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) Tmax = max(Tmax, (int)misc[4 + w]);
    const float* Bk = a.mod.Btp + (size_t)k * M * NP;
    const uint8_t* img = a.img + (size_t)k * NP * NP * 2;
    const int32_t* o = a.seq.symbols + (has && !bad_seq ? a.seq.offsets[s] : 0);
    RowState st;
    st.F = 0; st.f = 0; st.dead = false; st.bad = bad_seq; st.written = (Tn == 0);
    st.err = 0; st.ll = 0.f;

    // the first chunks of A^T, in flight while the first epilogue runs
    const int total_chunks = Tmax > 1 ? (Tmax - 1) * NKC : 0;
    if (tid == 0) {
      for (int g = 0; g < RING && g < total_chunks; ++g) {
        tc::mbar_arrive_expect_tx(&full[g], L::CHUNK);
        tc::bulk_g2s(aR + g * L::CHUNK, img + (size_t)(g % NKC) * L::CHUNK, L::CHUNK, &full[g]);
        pend_full[g] = true;
      }
    }

    // t = 0: x_0 = pi . b(o_0), no scaling
    {
      int o0 = Tn > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; o0 = 0; }
      const bool live = Tn > 0 && !st.bad;
      const float4* b4 = reinterpret_cast<const float4*>(Bk + (size_t)o0 * NP + col0);
      const float4* p4 = reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * NP + col0);
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        float y[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 bb = __ldg(b4 + 8 * c + q);
          const float4 pp = __ldg(p4 + 8 * c + q);
          y[4 * q] = live ? pp.x * bb.x : 0.f; y[4 * q + 1] = live ? pp.y * bb.y : 0.f;
          y[4 * q + 2] = live ? pp.z * bb.z : 0.f; y[4 * q + 3] = live ? pp.w * bb.w : 0.f;
        }
        part += tree_sum<32>(y);
        uint32_t w[16];
        pack32(y, w);
#pragma unroll
        for (int g = 0; g < 4; ++g)
          *reinterpret_cast<uint4*>(sX + x_row + ((col0 + 32 * c) / 8 + g) * 128) =
              make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
      }
      psum[h * 128 + row] = part;
    }
    int o_next = (1 < Tn) ? __ldg(o + 1) : 0;
    int o_next2 = (2 < Tn) ? __ldg(o + 2) : 0;

    bool aborted = false;
    int g = 0;  // chunk counter of this item
    for (int t = 1; t < Tmax; ++t) {
      tc::fence_proxy_async();  // X image writes -> tensor core
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0 && !abort_issue) {
        tc::fence_after_sync();
        for (int kc = 0; kc < NKC; ++kc, ++g) {
          const int sl = g % RING;
          if (!tc::mbar_wait_bounded(&full[sl], ph_full[sl], a.wait_limit)) { abort_issue = true; break; }
          ph_full[sl] ^= 1;
          pend_full[sl] = false;
#pragma unroll
          for (int nb = 0; nb < NP / 256; ++nb)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
              tc::mma_bf16(tmem + (uint32_t)(nb * 256),
                           tc::smem_desc(aX + (4 * kc + 2 * ks) * 128, 128, NP * 16),
                           tc::smem_desc(aR + sl * L::CHUNK + nb * 16384 + ks * 256, 128, 512),
                           idesc, (kc > 0 || ks > 0) ? 1u : 0u);
          tc::mma_commit(&empty[sl]);
          pend_empty[sl] = true;
          // the previous chunk's buffer refills with the chunk RING - 1 ahead
          if (g >= 1) {
            const int pg = g - 1, ps = pg % RING;
            if (!tc::mbar_wait_bounded(&empty[ps], ph_empty[ps], a.wait_limit)) { abort_issue = true; break; }
            ph_empty[ps] ^= 1;
            pend_empty[ps] = false;
            const int ng = pg + RING;
            if (ng < total_chunks) {
              tc::mbar_arrive_expect_tx(&full[ps], L::CHUNK);
              tc::bulk_g2s(aR + ps * L::CHUNK, img + (size_t)(ng % NKC) * L::CHUNK, L::CHUNK,
                           &full[ps]);
              pend_full[ps] = true;
            }
          }
        }
        tc::mma_commit(done);
        if (abort_issue) misc[2] = 1;
      }
      close_step(st, psum[row] + psum[128 + row] + psum[256 + row] + psum[384 + row], t - 1, Tn);
      const int ot = o_next;
      o_next = o_next2;
      if (t + 2 < Tn) o_next2 = __ldg(o + t + 2);
      if (t < Tn && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
      const bool live = t < Tn && !st.dead && !st.bad;
      if (live) st.F += st.f;
      const float2 fac2 = make_float2(exp2i(-st.f), exp2i(-st.f));
      const float4* eb = reinterpret_cast<const float4*>(
          Bk + (size_t)((unsigned)ot < (unsigned)M ? ot : 0) * NP + col0);
      float4 bq[8];  // emission values of the first 32 columns, in flight during the MMAs
#pragma unroll
      for (int q = 0; q < 8; ++q) bq[q] = __ldg(eb + q);
      bool ok = true;
      if (warp == 1) ok = tc::mbar_wait_bounded(done, ph_done, a.wait_limit);
      ph_done ^= 1;
      // everyone agrees (and has read the partial sums) before they are rewritten
      if (!tc::bar_and(1, 512, ok && misc[2] == 0)) {
        aborted = true;
        break;
      }
      tc::fence_after_sync();
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        float4 bn[8];
        if (c + 1 < CH)
#pragma unroll
          for (int q = 0; q < 8; ++q) bn[q] = __ldg(eb + 8 * (c + 1) + q);
        float y[32];
        tc::tmem_ld32(d_mine + (uint32_t)(c * 32), y);
        tc::tmem_ld_wait();
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float2 lo = __fmul2_rn(__fmul2_rn(make_float2(y[4 * q], y[4 * q + 1]),
                                            make_float2(bq[q].x, bq[q].y)), fac2);
          float2 hi = __fmul2_rn(__fmul2_rn(make_float2(y[4 * q + 2], y[4 * q + 3]),
                                            make_float2(bq[q].z, bq[q].w)), fac2);
          if (!live) { lo = make_float2(0.f, 0.f); hi = lo; }
          acc = __fadd2_rn(acc, __fadd2_rn(lo, hi));
          y[4 * q] = lo.x; y[4 * q + 1] = lo.y; y[4 * q + 2] = hi.x; y[4 * q + 3] = hi.y;
        }
        part += acc.x + acc.y;
        uint32_t w[16];
        pack32(y, w);
#pragma unroll
        for (int gg = 0; gg < 4; ++gg)
          *reinterpret_cast<uint4*>(sX + x_row + ((col0 + 32 * c) / 8 + gg) * 128) =
              make_uint4(w[4 * gg], w[4 * gg + 1], w[4 * gg + 2], w[4 * gg + 3]);
        if (c + 1 < CH)
#pragma unroll
          for (int q = 0; q < 8; ++q) bq[q] = bn[q];
      }
      psum[h * 128 + row] = part;
    }
    if (tid == 0 && !abort_issue) {  // the last chunk's commit (its MMAs are done by now)
      for (int i = 0; i < RING; ++i)
        if (pend_empty[i]) {
          if (!tc::mbar_wait_bounded(&empty[i], ph_empty[i], a.wait_limit)) { abort_issue = true; break; }
          ph_empty[i] ^= 1;
          pend_empty[i] = false;
        }
      if (abort_issue) misc[2] = 1;
    }
    __syncthreads();
    if (!aborted && Tmax > 0)
      close_step(st, psum[row] + psum[128 + row] + psum[256 + row] + psum[384 + row], Tmax - 1, Tn);
    if (aborted && tid == 0) {
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
    // recognition: the last model of a tile takes the argmax over models
    if (a.argmax) {
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        misc[3] = (atomicAdd(a.done + tile, 1) == K - 1) ? 1 : 0;
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

  // teardown: no copy or MMA of ours may still be in flight
  __syncthreads();
  if (tid == 0 && misc[2]) {
    if (misc[2]) set_status(a.status, HMM_STATUS_TIMEOUT);
    tc::mma_commit(fin);  // arrives once every MMA issued so far is done
    tc::mbar_wait_bounded(fin, 0, kWideWait);
    for (int i = 0; i < RING; ++i)
      if (pend_full[i]) tc::mbar_wait_bounded(&full[i], ph_full[i], kWideWait);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <int NP>
__global__ void __launch_bounds__(512, 1) hmm_forward_wide(const __grid_constant__ MmaWideLaunch a) {
  wide_body<NP>(a);
}

template <int NP>
static cudaError_t build_wide_image(const MmaWideLaunch& a, cudaStream_t st) {
  const long long n = (long long)a.seq.K * NP * NP / 2;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  wide_image_kernel<NP><<<blocks, 256, 0, st>>>(a.mod.Ap, a.img, a.seq.K);
  return cudaGetLastError();
}

template <int NP>
static cudaError_t launch_wide_t(const MmaWideLaunch& a, cudaStream_t st) {
  using L = WideCfg<NP>;
  cudaError_t err = build_wide_image<NP>(a, st);
  if (err != cudaSuccess) return err;
  auto kern = hmm_forward_wide<NP>;
  const int smem = L::TOTAL > 120 * 1024 ? L::TOTAL : 120 * 1024;  // one CTA per SM
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  int blocks = num_sms();
  if (blocks > a.n_items) blocks = a.n_items > 0 ? a.n_items : 1;
  kern<<<blocks, L::NTH, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_forward_wide(int NP, const MmaWideLaunch& a, cudaStream_t st) {
  if (a.xs) return cudaErrorInvalidValue;  // the adjoint's passes: launch_cluster_passes
  if (NP == 256) return launch_wide_t<256>(a, st);
  if (NP == 512) return launch_wide_t<512>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
