// mma_pass_tf32.cu -- the forward-backward adjoint with TF32 operands for
// 32 < N <= 128 states (Sec. 2.7 "Baum-Welch", its E-step; Rabiner 1989
// eqs. 19-21 forward and 24-25 backward variables): the forward and the
// backward recursion of every tile of the adjoint's tile plan, each keeping
// every step's row for the count kernels of fb_wide.cu (gamma and xi from
// the rows, xi as one contraction over all steps on the tensor cores):
//
//   forward   X_t  = D_t . b(o_t) . 2^-f_t,  D_t = X_{t-1} A       (scaled alpha_t)
//   backward  Bh_t = D_t . 2^-f_t,  D_t = A (b(o_{t+1}) . Bh_{t+1}),  Bh_{T-1} = 1
//             (scaled beta_t before the emission product, with its exponent f_t)
//
// Both are the per-row recursion D = X . B_op with B_op = A (forward) or A^T
// (backward) -- the backward in reversed time, each row starting at its own
// last step -- computed as tcgen05.mma kind::tf32 (M = 128 rows of the tile,
// N = N_pad, K = 8 per instruction) with the row operand in tensor memory
// (TF32, round to nearest) and the transition image in shared memory; FP32
// accumulation. The scale exponent f_t is that of the previous step's row sum
// (one step late, as everywhere on the tensor cores); every rescaling is by an
// exact power of two.
//
// Rows are stored at row rp[s] + t of [rows][N_pad] FP32 buffers (model k's
// block starts at k * rows when every sequence meets every model), rp the
// exclusive prefix of the lengths in the plan's order, so that when sequences
// are labelled the rows of one model are contiguous. One tile per CTA of
// 128 * TPR threads (TPR = N_pad / 32 threads per row, 32 columns each); the
// model's FP32 emission table sits in shared memory. Every mbarrier wait is
// bounded; on timeout the kernel records HMM_STATUS_TIMEOUT, waits (bounded)
// for its own products and leaves.
#include "hmm_internal.cuh"
#include "mma_rows.cuh"
#include "tc.cuh"

namespace hmmgb {

constexpr uint32_t kTf32Drain = 1u << 24;  // polls of the teardown's drain wait

// One 32-byte store (256-bit vector store, sm_100+).
__device__ __forceinline__ void st_v8r(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               :: "l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]),
                  "f"(v[6]), "f"(v[7]) : "memory");
}

template <int NP>
__global__ void __launch_bounds__(128 * (NP / 32), 1) hmm_fb_pass_tf32(const __grid_constant__ MmaPassLaunch a) {
  constexpr int TPR = NP / 32;       // threads per row
  constexpr int NTH = 128 * TPR;
  using L = MmaFwdSmem<NP, 1, TPR, 2, true>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem + L::OFF_B;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS);  // [TPR][128]
  uint64_t* mbar = &bars[0];
  uint64_t* fbar = &bars[2];
  const uint8_t* etab = smem + L::OFF_E;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = warp >> 2;   // lane quarter, column share
  const int row = wq * 32 + lane;
  const int K = a.seq.K, M = a.seq.M;

  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), 256);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(fbar, 1);
    misc[2] = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t d_tmem = tmem;                      // D: NP FP32 columns
  const uint32_t x_tmem = tmem + (uint32_t)NP;       // X: NP TF32 columns
  const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
  const uint32_t d_mine = d_tmem + lane_off + (uint32_t)(h * 32);
  const uint32_t x_mine = x_tmem + lane_off + (uint32_t)(h * 32);
  constexpr uint32_t idesc = tc::instr_desc(2, 128, NP);
  const uint32_t b_base = tc::smem_u32(sB);
  constexpr uint32_t SBO = NP * 32;  // next 8 rows of the TF32 image
  uint32_t mphase = 0;
  int cur_key = -1;
  auto row_total = [&]() {
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
    const int tile = a.pass_tiles[grp];
    const int k = tile >= 0 ? a.tile_model[tile] : 0;

    if (2 * k + dir != cur_key) {
      // B operand, K-major TF32: forward (n = j, k = i) = a_ij; backward (n = i, k = j) = a_ij
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
      for (int idx = tid; idx < NP * NP; idx += NTH) {
        const int n = idx / NP, kk = idx % NP;
        const float v = dir ? __ldg(Ak + n * NP + kk) : __ldg(Ak + kk * NP + n);
        const uint32_t off = (n / 8) * SBO + (kk / 4) * 128 + (n % 8) * 16 + (kk % 4) * 4;
        *reinterpret_cast<uint32_t*>(sB + off) = tc::to_tf32(v);
      }
      if (cur_key < 0 || (cur_key >> 1) != k)
        fill_emission_table<NP, 2, L::kET>(smem + L::OFF_E, a.mod.Btp + (size_t)k * M * NP, M, tid, NTH);
      cur_key = 2 * k + dir;
      tc::fence_proxy_async();
      __syncthreads();
    }

    const int rows = tile >= 0 ? a.tile_rows[tile] : 0;
    const bool has = row < rows;
    const int s = has ? a.sorted[a.tile_start[tile] + row] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;  // >= 1 for every row of a tile
    const int Tmax = tile >= 0 ? a.tile_len[tile] : 0;
    // the row's first tile step: 0 forward; backward, its last step's, counted
    // from the end of the tile's longest row
    const int u0 = dir ? Tmax - T : 0;
    const int32_t* o = a.seq.symbols + (has ? a.seq.offsets[s] : 0);
    const int64_t r0 = has ? (a.labelled ? 0 : (int64_t)k * a.rtot) + a.rp[s] : 0;
    float* xrow = has ? (dir ? a.bhs : a.xs) + r0 * NP + h * 32 : nullptr;
    int32_t* xerow = (has && dir && h == 0) ? a.xe + r0 : nullptr;
    // sequence step of tile step u, and its symbol (0 outside the row)
    auto tseq = [&](int u) { return dir ? Tmax - 1 - u : u; };
    auto sym_at = [&](int u) -> int {
      if (!has || u < u0 || u >= u0 + T) return 0;
      return __ldg(o + tseq(u));
    };
    auto store_row = [&](int u, const float (&v)[32]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) st_v8r(xrow + (size_t)tseq(u) * NP + 8 * q, v + 8 * q);
    };
    RowState st;
    st.F = 0; st.f = 0; st.dead = false; st.bad = false; st.written = false;
    st.err = 0; st.ll = 0.f; st.slast = 0.f;

    // step 0: forward x_0 = pi . b(o_0); backward, the rows whose last step is
    // the tile's last: Bh = 1, Y = b(o_{T-1}); no scaling
    {
      int o0 = sym_at(0);
      if ((unsigned)o0 >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; o0 = 0; }
      const bool live = has && u0 == 0 && !st.bad;
      float b[8], y[32], sv[32];
      const float4* p4 = reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * NP + h * 32);
      const uint8_t* eb = etab + o0 * L::kET;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        emission8<2>(eb, h * 32 + 8 * q, b);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = 8 * q + i;
          const float pv = dir ? 1.f : __ldg(reinterpret_cast<const float*>(p4) + c);
          y[c] = live ? pv * b[i] : 0.f;
          sv[c] = dir ? (live ? 1.f : 0.f) : y[c];
        }
      }
      // every step of a row is stored (zero where the row is dead or invalid)
      if (has && u0 == 0) store_row(0, sv);
      if (xerow && u0 == 0) xerow[tseq(0)] = 0;
      const float part = tree_sum<32>(y);
      store_x<2>(x_mine, 0, y);
      tc::tmem_st_wait();
      psum[h * 128 + row] = part;
    }
    int o_next = sym_at(1);
    int o_next2 = sym_at(2);

    bool aborted = false;
    for (int t = 1; t < Tmax; ++t) {
      tc::fence_before_sync();
      tc::bar_sync(1, NTH);
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < NP / 8; ++ks)
          tc::mma_tf32_ts(d_tmem, x_tmem + (uint32_t)(ks * 8),
                          tc::smem_desc(b_base + ks * 256, 128, SBO), idesc, ks > 0 ? 1u : 0u);
        tc::mma_commit(mbar);
      }
      const float sig = row_total();
      if (!dir) {
        close_step(st, sig, t - 1, T);
      } else if (has && t - 1 >= u0 && !st.dead && !st.bad) {
        // backward: any positive scale will do; a zero row stays zero
        if (!(sig > 0.f) || isinf(sig)) st.dead = true;
        else st.f = min(126, max(-126, exponent_of(sig)));
      }
      const int ot = o_next;
      o_next = o_next2;
      o_next2 = sym_at(t + 2);
      const bool inrow = has && t >= u0 && t < u0 + T;
      // an invalid symbol ends the row in both directions: no counts anywhere
      if (inrow && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
      const uint8_t* eb = etab + ((unsigned)ot < (unsigned)M ? ot : 0) * L::kET;
      const bool start = dir && t == u0;   // the backward row starts here: Bh = 1
      const bool live = inrow && !st.dead && !st.bad;
      const int f = start ? 0 : st.f;
      if (!dir && live) st.F += f;
      const float2 fac2 = make_float2(exp2i(-f), exp2i(-f));
      bool ok = true;
      if (warp == 0) ok = tc::mbar_wait_bounded(mbar, mphase, a.wait_limit);
      mphase ^= 1;
      if (!tc::bar_and(1, NTH, ok)) {
        aborted = true;
        break;
      }
      tc::fence_after_sync();
      float y[32], sv[32];
      tc::tmem_ld32(d_mine, y);
      tc::tmem_ld_wait();
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float b[8];
        emission8<2>(eb, h * 32 + 8 * q, b);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = 8 * q + 2 * i;
          float2 yv = make_float2(y[c], y[c + 1]);
          if (start) yv = make_float2(1.f, 1.f);
          float2 v, keep;
          if (!dir) {
            v = __fmul2_rn(__fmul2_rn(yv, make_float2(b[2 * i], b[2 * i + 1])), fac2);
            if (!live) v = make_float2(0.f, 0.f);
            keep = v;
          } else {
            keep = __fmul2_rn(yv, fac2);
            if (!live) keep = make_float2(0.f, 0.f);
            v = __fmul2_rn(keep, make_float2(b[2 * i], b[2 * i + 1]));
          }
          acc = __fadd2_rn(acc, v);
          y[c] = v.x; y[c + 1] = v.y;
          sv[c] = keep.x; sv[c + 1] = keep.y;
        }
      }
      if (inrow) store_row(t, sv);
      if (xerow && inrow) xerow[tseq(t)] = live ? f : 0;
      store_x<2>(x_mine, 0, y);
      tc::tmem_st_wait();
      psum[h * 128 + row] = acc.x + acc.y;
    }
    tc::bar_sync(1, NTH);
    if (!dir && !aborted && Tmax > 0) close_step(st, row_total(), Tmax - 1, T);
    if (aborted && tid == 0) {
      misc[2] = 1;
      set_status(a.status, HMM_STATUS_TIMEOUT);
    }
    if (has && h == 0 && st.bad && st.err) set_status(a.status, st.err);
    if (!dir && has && h == 0) {
      float out = st.ll;
      if (st.bad || aborted) out = __int_as_float(0x7fc00000);
      else if (st.dead) out = -INFINITY;
      else if (!st.written) out = __int_as_float(0x7fc00000);
      a.loglik[a.labelled ? (size_t)s : (size_t)s * K + k] = out;
    }
  }

  // teardown: no product of ours may still be in flight
  tc::fence_before_sync();
  __syncthreads();
  if (misc[2] && tid == 0) {
    tc::mma_commit(fbar);
    tc::mbar_wait_bounded(fbar, 0, kTf32Drain);
  }
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// rp[sorted[p]] = sum of the lengths of the plan's sequences before position
// p (exclusive prefix in the plan's order), and pos_row[p] the same by
// position. Model k's rows are [mrow[k], mrow[K + 1 + k]): labelled, its
// sequences are contiguous in the plan's order; otherwise every model has a
// block of rows_unlabelled rows of which the first (all lengths) are used.
// One block.
__global__ void __launch_bounds__(1024) tf32_rows_kernel(const int32_t* sorted, const int32_t* n_valid,
                                                         const int32_t* seqlen,
                                                         const int32_t* model_of_seq, int K,
                                                         int64_t* rp, int64_t* pos_row,
                                                         int64_t* mrow, int64_t rows_unlabelled) {
  __shared__ int64_t part[1024];
  const int n = *n_valid, tid = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int p0 = min(n, tid * per), p1 = min(n, p0 + per);
  int64_t sum = 0;
  for (int p = p0; p < p1; ++p) sum += seqlen[sorted[p]];
  part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    for (int i = 0; i < 1024; ++i) {
      const int64_t v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  int64_t run = part[tid];
  for (int p = p0; p < p1; ++p) {
    const int s = sorted[p];
    rp[s] = run;
    pos_row[p] = run;
    run += seqlen[s];
  }
  __syncthreads();
  const int64_t total = n > 0 ? pos_row[n - 1] + seqlen[sorted[n - 1]] : 0;
  int64_t* mend = mrow + K + 1;
  if (model_of_seq) {
    // model k's block starts at its first sequence in the plan's order
    for (int k = tid; k < K; k += 1024) mrow[k] = -1;
    __syncthreads();
    for (int p = tid; p < n; p += 1024) {
      const int k = model_of_seq[sorted[p]];
      if (p == 0 || model_of_seq[sorted[p - 1]] != k) mrow[k] = pos_row[p];
    }
    __syncthreads();
    if (tid == 0) {
      int64_t next = total;
      for (int k = K - 1; k >= 0; --k) {
        if (mrow[k] < 0) mrow[k] = next;  // a model without sequences: an empty block
        mend[k] = next;
        next = mrow[k];
      }
      mrow[K] = total;
    }
  } else {
    for (int k = tid; k < K; k += 1024) {
      mrow[k] = (int64_t)k * rows_unlabelled;
      mend[k] = mrow[k] + total;
    }
    if (tid == 0) mrow[K] = (int64_t)K * rows_unlabelled;
  }
}

template <int NP>
static cudaError_t launch_tf32_t(const MmaPassLaunch& a, cudaStream_t st) {
  using L = MmaFwdSmem<NP, 1, NP / 32, 2, true>;
  const int smem = L::total(a.seq.M);
  if (smem > kFwdSmemMax) return cudaErrorInvalidValue;
  auto kern = hmm_fb_pass_tf32<NP>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem > 120 * 1024 ? smem : 120 * 1024);
  if (err != cudaSuccess) return err;
  kern<<<num_sms(), 128 * (NP / 32), smem > 120 * 1024 ? smem : 120 * 1024, st>>>(a);
  return cudaGetLastError();
}

bool fb_tf32_supported(int NP, int M) {
  if (NP == 64) return MmaFwdSmem<64, 1, 2, 2, true>::total(M) <= kFwdSmemMax;
  if (NP == 128) return MmaFwdSmem<128, 1, 4, 2, true>::total(M) <= kFwdSmemMax;
  return false;
}

cudaError_t launch_fb_pass_tf32(int NP, const MmaPassLaunch& a, const int32_t* n_valid,
                                int64_t* pos_row, int64_t* mrow, cudaStream_t st) {
  if (!a.xs || !a.bhs || !a.xe || !a.rp) return cudaErrorInvalidValue;
  tf32_rows_kernel<<<1, 1024, 0, st>>>(a.sorted, n_valid, a.seq.seqlen, a.seq.model_of_seq,
                                      a.seq.K, const_cast<int64_t*>(a.rp), pos_row, mrow,
                                      a.rtot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (NP == 64) return launch_tf32_t<64>(a, st);
  if (NP == 128) return launch_tf32_t<128>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
