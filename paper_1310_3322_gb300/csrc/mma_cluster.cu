// mma_cluster.cu -- scaled forward algorithm on the tensor cores for 128 < N <= 512
// states over a thread-block cluster (Sec. 2.7 "Forward"; Sec. 5.6 quotes the
// cited forward kernel at 512 states x 512 sequences; Rabiner 1989 eqs. 19-21).
//
// The recursion of mma_wide.cu -- a tile of 128 (sequence, model) rows of one
// model computes D[128 x N] = X[128 x N] . A[N x N] per step, multiplies each
// row's emission row, scales by the late power of two and writes the next X --
// with the state dimension split over CL = N / 64 CTAs of a cluster instead of
// streaming A^T through one SM:
//   * CTA c owns output columns [64 c, 64 c + 64): its column slice of A (the B
//     operand, 64 x N BF16, up to 64 KB) and its slice of the model's emission
//     table stay in shared memory for the whole item, and its 64 accumulator
//     columns live in tensor memory;
//   * every CTA holds the whole X (128 x N BF16, K-major, up to 128 KB), laid
//     out slice-major: the 64 states of K of CTA c are one contiguous 16 KB
//     block (core matrices of 8 rows x 16 bytes, 1 KB per 8 rows);
//   * after its epilogue a CTA writes its slice of the next X into its own X and
//     sends it, with its 128 partial row sums, to every other CTA of the
//     cluster by bulk copies into their shared memory, completing on the
//     receiver's `full` mbarrier of that sender; the receiver starts the
//     product over each slice as soon as it lands (its own slice first, then
//     in the order the senders send), so the products overlap the exchange;
//     the row sums of a step are the sums of the CL partials,
//     added in rank order by every CTA alike, so all CTAs keep the same row
//     state (exponents, log-likelihood);
//   * a CTA may write a peer's X only after that peer's product has read it: each
//     CTA, its product done, arrives on every peer's `free` mbarrier, and waits
//     on its own for all peers before it overwrites its slice or sends it.
// A tile has TR = 128 rows, or 32 / 64 when the batch is small enough that the
// clusters of the smaller tiles still fit the GPU in one wave: the product
// stays M = 128 (rows TR .. 127 of X are zero in every CTA and never sent), so
// each step moves TR / 128 of the bytes over the cluster. The same code runs
// the adjoint's backward recursion (A^T slices, reversed time) and keeps every
// step's rows for its count kernels (cluster_body's DIR and STORE).
// 512 threads, four per row (16 columns each); thread 0 issues the products and
// copies. Every mbarrier wait is bounded; on timeout the kernel records
// HMM_STATUS_TIMEOUT and leaves the loop. At the end every CTA meets the others
// at a cluster barrier (after it no CTA sends), reads how many steps each peer
// sent, waits (bounded) for exactly those copies, drains its own products and
// meets them again before it exits, so no copy lands in a CTA that has left.
#include "hmm_internal.cuh"
#include "mma_rows.cuh"
#include "tc.cuh"

namespace hmmgb {

template <int NP>
struct ClusterCfg {
  static constexpr int CL = NP / 64;            // CTAs per cluster
  static constexpr int NTH = 512;
  static constexpr int TPR = 4;                 // threads per row
  static constexpr int COLS = 16;               // columns per thread
  static constexpr int SLICE = 128 * 64 * 2;    // one CTA's slice of X (16 KB)
  static constexpr int XB = CL * SLICE;         // the whole X
  static constexpr int BB = 64 * NP * 2;        // the A column slice (B operand)
  static constexpr int ES = 64 * 2 + 16;        // padded BF16 row of the emission slice
  static constexpr int OFF_X = 0;
  static constexpr int OFF_B = OFF_X + XB;
  static constexpr int OFF_PX = OFF_B + BB;                 // row sums [2][CL][128]
  static constexpr int OFF_PS = OFF_PX + 2 * CL * 128 * 4;  // partials [TPR][128]
  static constexpr int OFF_PO = OFF_PS + TPR * 128 * 4;     // this CTA's row sums [128]
  static constexpr int OFF_BAR = OFF_PO + 128 * 4;          // full [CL], free, mma, fin
  static constexpr int OFF_MISC = OFF_BAR + (CL + 3) * 8;   // tmem, abort, done flag, sent, row maxima [4]
  static constexpr int OFF_E = (OFF_MISC + 32 + 127) / 128 * 128;  // emission slice [M][ES]
  static constexpr int fixed() { return OFF_E; }
  static constexpr int total(int M) { return OFF_E + M * ES; }
  static_assert(NP == 256 || NP == 512, "64-column slices, cluster of 4 or 8");
};

// Byte offset of (row m, state k) in the slice-major X image.
constexpr uint32_t kClusterDrain = 1u << 24;  // polls of the teardown's waits

template <int NP>
__device__ __forceinline__ uint32_t xs_off(int m, int k) {
  return (uint32_t)((k >> 6) * ClusterCfg<NP>::SLICE + (m >> 3) * 1024 + ((k & 63) >> 3) * 128 +
                    (m & 7) * 16 + (k & 7) * 2);
}

// One 32-byte store (256-bit vector store, sm_100+).
__device__ __forceinline__ void st_v8c(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               :: "l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]),
                  "f"(v[6]), "f"(v[7]) : "memory");
}

// The work of one cluster: item `item` of `a`. DIR = 1 runs the backward
// recursion Y_t = (Y_{t+1} A^T) o b(o_t) from Y_{T-1} = b(o_{T-1}) (the
// forward recursion with A^T in place of A); STORE keeps every step's row
// (forward: scaled alpha_t; backward: scaled beta_t before the emission
// product, with its exponent) for the adjoint's count kernels.
template <int NP, int DIR, bool STORE, int TR>
__device__ __forceinline__ void cluster_body(const MmaWideLaunch& a, int item) {
  using L = ClusterCfg<NP>;
  constexpr int CL = L::CL, SLICE = L::SLICE;
  static_assert(TR == 32 || TR == 64 || TR == 128, "rows per tile");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sX = smem + L::OFF_X;
  uint8_t* sB = smem + L::OFF_B;
  float* px = reinterpret_cast<float*>(smem + L::OFF_PX);   // [2][CL][128]
  float* psum = reinterpret_cast<float*>(smem + L::OFF_PS); // [TPR][128]
  float* pout = reinterpret_cast<float*>(smem + L::OFF_PO); // [128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint64_t* full = bars;            // [c]: the X slice + row sums of CTA c have arrived
  uint64_t* freeb = bars + CL;      // every other CTA's product has read its X
  uint64_t* mmab = bars + CL + 1;   // this step's product
  uint64_t* fin = bars + CL + 2;    // teardown
  volatile int32_t* misc = reinterpret_cast<volatile int32_t*>(smem + L::OFF_MISC);
  uint8_t* sE = smem + L::OFF_E;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3, h = warp >> 2;   // lane quarter, column quarter
  const int row = wq * 32 + lane;
  const uint32_t rank = tc::cluster_rank();
  const int c0 = 64 * (int)rank;            // this CTA's first state
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;
  const int tile = item / K, k = item % K;

  if (warp == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(smem + L::OFF_MISC), 64);
  if (tid == 0) {
    for (int c = 0; c < CL; ++c) tc::mbar_init(full + c, 1);
    tc::mbar_init(freeb, CL - 1);
    tc::mbar_init(mmab, 1);
    tc::mbar_init(fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    misc[1] = 0;
  }
  // rows TR .. 127 of X stay zero (the product is M = 128 rows)
  if (TR < 128)
    for (int i = tid; i < L::XB / 16; i += L::NTH) reinterpret_cast<uint4*>(sX)[i] = make_uint4(0, 0, 0, 0);
  // the model's column slice of A (B operand, K-major: (n = j - c0, k = i) =
  // a_ij; backward: a_ji)
  {
    const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
    for (int idx = tid; idx < 64 * NP / 2; idx += L::NTH) {
      const int n = idx / (NP / 2), i = (idx % (NP / 2)) * 2;
      const uint32_t w =
          DIR ? tc::pack_bf16(__ldg(Ak + (size_t)(c0 + n) * NP + i), __ldg(Ak + (size_t)(c0 + n) * NP + i + 1))
              : tc::pack_bf16(__ldg(Ak + (size_t)i * NP + c0 + n), __ldg(Ak + (size_t)(i + 1) * NP + c0 + n));
      *reinterpret_cast<uint32_t*>(sB + (n >> 3) * (NP * 16) + (i >> 3) * 128 + (n & 7) * 16 +
                                   (i & 7) * 2) = w;
    }
    // the emission slice: rows of 64 BF16 values (columns c0 .. c0 + 63)
    const uint16_t* Bk16 = a.mod.Btp16 + (size_t)k * M * NP + c0;
    for (int idx = tid; idx < M * 8; idx += L::NTH) {
      const int m = idx >> 3, q = idx & 7;
      *reinterpret_cast<uint4*>(sE + m * L::ES + q * 16) =
          __ldg(reinterpret_cast<const uint4*>(Bk16 + (size_t)m * NP) + q);
    }
  }
  tc::fence_proxy_async();  // the B operand -> tensor core
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = (uint32_t)misc[0];
  const uint32_t d_mine = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(h * 16);
  constexpr uint32_t idesc = tc::instr_desc(1, 128, 64);
  const uint32_t aX = tc::smem_u32(sX), aB = tc::smem_u32(sB);
  // the barriers of every CTA are initialised before anyone sends to them
  tc::cluster_sync();

  // this row's state (every CTA keeps all TR rows of the tile, alike; rows
  // TR .. 127 hold nothing and stay zero)
  const int pos = tile * TR + row;
  const bool has = row < TR && pos < S;
  const int s = has ? a.seq.order[pos] : 0;
  const int T = has ? a.seq.seqlen[s] : 0;
  const bool bad_seq = T < 0;
  const int Tn = bad_seq ? 0 : T;
  {  // longest row of the tile (warps 0-3 hold every row once)
    const int wm = __reduce_max_sync(HMM_FULL_MASK, Tn);
    if (h == 0 && lane == 0) misc[4 + wq] = wm;
  }
  __syncthreads();
  int Tmax = 0;  // alike in every CTA of the cluster
#pragma unroll
  for (int w = 0; w < 4; ++w) Tmax = max(Tmax, (int)misc[4 + w]);
  // thread 0: steps sent; steps whose slices have all been seen, and the
  // senders whose slice of the step after those has been seen
  uint32_t n_sent = 0, n_done = 0, got = 0;
  const int32_t* o = a.seq.symbols + (has && !bad_seq ? a.seq.offsets[s] : 0);
  // step t reads symbol o_t (forward) or o_{T-1-t} (backward)
  auto tix = [&](int t) { return DIR ? Tn - 1 - t : t; };
  // this thread's 16 columns of the row's per-step output rows
  float* xrow = (STORE && has && !bad_seq)
                    ? a.xs + ((size_t)k * a.rtot + (size_t)a.roff[s]) * NP + c0 + 16 * h : nullptr;
  int32_t* xerow = (STORE && DIR && has && !bad_seq && rank == 0 && h == 0)
                       ? a.xe + (size_t)k * a.rtot + (size_t)a.roff[s] : nullptr;
  RowState st;
  st.F = 0; st.f = 0; st.dead = false; st.bad = bad_seq; st.written = (Tn == 0);
  st.err = 0; st.ll = 0.f; st.slast = 0.f;

  // this thread's 16 columns of a BF16 emission row of the slice
  auto emis16 = [&](int sym, float (&b)[16]) {
    const uint4* p = reinterpret_cast<const uint4*>(sE + sym * L::ES + h * 32);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint4 v = p[q];
      const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        b[8 * q + 2 * i] = __uint_as_float(u[i] << 16);
        b[8 * q + 2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
      }
    }
  };
  // writes this thread's 16 values of the next X into the own slice and its
  // partial row sum; then the CTA's row sums (own copy in px[par][rank]),
  // visible to the bulk copies
  auto put_row = [&](const float (&y)[16], float part, int par) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = tc::pack_bf16(y[2 * i], y[2 * i + 1]);
#pragma unroll
    for (int g = 0; g < 2; ++g)
      *reinterpret_cast<uint4*>(sX + xs_off<NP>(row, c0 + 16 * h + 8 * g)) =
          make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
    psum[h * 128 + row] = part;
    tc::bar_sync(1, L::NTH);
    if (h == 0) {
      const float v = psum[row] + psum[128 + row] + psum[256 + row] + psum[384 + row];
      pout[row] = v;
      px[(par * CL + (int)rank) * 128 + row] = v;
    }
    tc::fence_proxy_async();
    tc::bar_sync(1, L::NTH);
  };
  // thread 0: this CTA's slice of X and its row sums to every other CTA
  auto send = [&](int par) {
    ++n_sent;
#pragma unroll 1
    for (int p = 1; p < CL; ++p) {
      const uint32_t peer = (rank + (uint32_t)p) % (uint32_t)CL;
      const uint32_t fb = tc::map_rank(tc::smem_u32(full + rank), peer);
      const uint32_t xs = aX + rank * SLICE;
      tc::bulk_s2peer(tc::map_rank(xs, peer), xs, TR * 128, fb);  // rows 0 .. TR - 1
      const uint32_t ps = tc::smem_u32(px + (par * CL + (int)rank) * 128);
      tc::bulk_s2peer(tc::map_rank(ps, peer), tc::smem_u32(pout), TR * 4, fb);
    }
  };
  // sum of the row's CL partial sums of step parity `par` (rank order)
  auto row_total = [&](int par) {
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < CL; ++c) v += px[(par * CL + c) * 128 + row];
    return v;
  };
  constexpr uint32_t kSliceTx = (uint32_t)(TR * 128 + TR * 4);

  // t = 0: x_0 = pi . b(o_0) (backward: Y_{T-1} = b(o_{T-1}), beta = 1), no scaling
  if (Tmax > 0) {
    int o0 = Tn > 0 ? __ldg(o + tix(0)) : 0;
    if ((unsigned)o0 >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; o0 = 0; }
    const bool live = Tn > 0 && !st.bad;
    float b[16], y[16];
    emis16(o0, b);
    const float4* p4 = reinterpret_cast<const float4*>(a.mod.pip + (size_t)k * NP + c0 + 16 * h);
    float part = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 pp = DIR ? make_float4(1.f, 1.f, 1.f, 1.f) : __ldg(p4 + q);
      y[4 * q] = live ? pp.x * b[4 * q] : 0.f;
      y[4 * q + 1] = live ? pp.y * b[4 * q + 1] : 0.f;
      y[4 * q + 2] = live ? pp.z * b[4 * q + 2] : 0.f;
      y[4 * q + 3] = live ? pp.w * b[4 * q + 3] : 0.f;
      part += (y[4 * q] + y[4 * q + 1]) + (y[4 * q + 2] + y[4 * q + 3]);
    }
    if (STORE && xrow && Tn > 0) {
      float sv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) sv[i] = DIR ? (live ? 1.f : 0.f) : y[i];
      st_v8c(xrow + (size_t)tix(0) * NP, sv);
      st_v8c(xrow + (size_t)tix(0) * NP + 8, sv + 8);
    }
    if (xerow && Tn > 0) xerow[tix(0)] = 0;
    put_row(y, part, 0);
    if (tid == 0) {
      for (int c = 0; c < CL; ++c)
        if (c != (int)rank) tc::mbar_arrive_expect_tx(full + c, kSliceTx);
      send(0);
    }
  }

  uint32_t ph_free = 0, ph_mma = 0;  // thread 0's barrier phases
  bool aborted = false;
  int o_next = (1 < Tn) ? __ldg(o + tix(1)) : 0;
  // step t: the product X_{t-1} . A and the epilogue writing X_t; at t = Tmax
  // only the row sums of the last step
  for (int t = 1; t <= Tmax; ++t) {
    const bool last = t == Tmax;
    const int ot = o_next;  // the emission row of step t does not wait for X_{t-1}
    if (t + 1 < Tn) o_next = __ldg(o + tix(t + 1));
    float b[16];
    emis16((unsigned)ot < (unsigned)M ? ot : 0, b);
    bool ok = true;
    if (tid == 0) {
      const uint32_t par = (uint32_t)(t - 1) & 1u;
#pragma unroll 1
      for (int j = 0; j < CL; ++j) {
        const int c = (int)((rank + (uint32_t)(CL - j)) % (uint32_t)CL);  // own slice first
        if (j > 0) {
          if (!tc::mbar_wait_cluster(full + c, par, a.wait_limit)) {
            ok = false;
            break;
          }
          got |= 1u << c;
          if (!last) tc::mbar_arrive_expect_tx(full + c, kSliceTx);  // the exchange of X_t
        }
        if (!last) {
          tc::fence_after_sync();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            tc::mma_bf16(tmem, tc::smem_desc(aX + c * SLICE + kk * 256, 128, 1024),
                         tc::smem_desc(aB + (4 * c + kk) * 256, 128, NP * 16), idesc,
                         (j | kk) ? 1u : 0u);
        }
      }
      if (ok) {
        ++n_done;
        got = 0;
        if (!last) tc::mma_commit(mmab);
      }
    }
    if (!tc::bar_and(1, L::NTH, ok)) {
      aborted = true;
      break;
    }
    close_step(st, row_total((t - 1) & 1), t - 1, Tn);
    if (last) break;
    if (t < Tn && (unsigned)ot >= (unsigned)M) { st.bad = true; st.err |= HMM_STATUS_SYMBOL; }
    const bool live = t < Tn && !st.dead && !st.bad;
    if (live) st.F += st.f;
    const float2 fac2 = make_float2(exp2i(-st.f), exp2i(-st.f));
    // the product is done: this CTA's X may be rewritten by the others; wait
    // until every other CTA's product is done too (then the own slice and the
    // row sums may be rewritten and sent)
    if (tid == 0) {
      ok = tc::mbar_wait_bounded(mmab, ph_mma, a.wait_limit);
      ph_mma ^= 1;
      if (ok) {
#pragma unroll 1
        for (int p = 1; p < CL; ++p)
          tc::mbar_arrive_remote(tc::map_rank(tc::smem_u32(freeb), (rank + (uint32_t)p) % (uint32_t)CL));
        ok = tc::mbar_wait_cluster(freeb, ph_free, a.wait_limit);
        ph_free ^= 1;
      }
    }
    if (!tc::bar_and(1, L::NTH, ok)) {
      aborted = true;
      break;
    }
    tc::fence_after_sync();
    float y[16];
    tc::tmem_ld16(d_mine, y);
    tc::tmem_ld_wait();
    tc::fence_before_sync();  // the next product may overwrite the accumulator
    float2 acc = make_float2(0.f, 0.f);
    float sv[16];  // the stored row: alpha_t (forward) or beta_t (backward)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float2 v;
      if constexpr (DIR == 0) {
        v = __fmul2_rn(__fmul2_rn(make_float2(y[2 * q], y[2 * q + 1]),
                                  make_float2(b[2 * q], b[2 * q + 1])), fac2);
        if (!live) v = make_float2(0.f, 0.f);
        sv[2 * q] = v.x;
        sv[2 * q + 1] = v.y;
      } else {  // beta_t = D 2^-f kept, Y_t = beta_t o b(o_t) is the next operand
        float2 p = __fmul2_rn(make_float2(y[2 * q], y[2 * q + 1]), fac2);
        if (!live) p = make_float2(0.f, 0.f);
        sv[2 * q] = p.x;
        sv[2 * q + 1] = p.y;
        v = __fmul2_rn(p, make_float2(b[2 * q], b[2 * q + 1]));
      }
      acc = __fadd2_rn(acc, v);
      y[2 * q] = v.x;
      y[2 * q + 1] = v.y;
    }
    if (STORE && xrow && t < Tn) {
      st_v8c(xrow + (size_t)tix(t) * NP, sv);
      st_v8c(xrow + (size_t)tix(t) * NP + 8, sv + 8);
    }
    if (xerow && t < Tn) xerow[tix(t)] = live ? st.f : 0;
    put_row(y, acc.x + acc.y, t & 1);
    if (tid == 0) send(t & 1);
  }
  if (aborted && tid == 0) {
    misc[1] = 1;
    set_status(a.status, HMM_STATUS_TIMEOUT);
  }
  if (DIR == 0 && rank == 0 && has && h == 0) {
    float out = st.ll;
    if (st.bad || aborted) out = __int_as_float(0x7fc00000);
    else if (st.dead) out = -INFINITY;
    else if (!st.written) out = __int_as_float(0x7fc00000);
    if (st.bad && st.err) set_status(a.status, st.err);
    a.loglik[(size_t)s * K + k] = out;
  }
  // recognition: the last model of a tile takes the argmax over models
  if (DIR == 0 && rank == 0 && a.argmax) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      misc[2] = (atomicAdd(a.done + tile, 1) == K - 1) ? 1 : 0;
    }
    __syncthreads();
    if (misc[2]) {
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

  // teardown. After the first cluster barrier no CTA sends. A peer that sent
  // n steps sent its slices of X_0 .. X_{n-1}; the counts of two CTAs differ
  // by one at most, and we have seen the peer's slices up to X_{seen - 1}:
  // wait (bounded) for the one that may still be on its way.
  if (tid == 0) misc[3] = (int32_t)n_sent;
  tc::cluster_sync();
  if (tid == 0) {
#pragma unroll 1
    for (int c = 0; c < CL; ++c) {
      if (c == (int)rank) continue;
      const uint32_t ns = tc::ld_cluster_u32(tc::map_rank(tc::smem_u32(smem + L::OFF_MISC + 12),
                                                          (uint32_t)c));
      const uint32_t seen = n_done + ((got >> c) & 1u);
      if (ns > seen) tc::mbar_wait_cluster(full + c, seen & 1u, kClusterDrain);
    }
    tc::mma_commit(fin);  // arrives once every product issued so far is done
    tc::mbar_wait_bounded(fin, 0, kClusterDrain);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
  tc::cluster_sync();  // no CTA leaves while a peer may still read its counts
}

// Recognition: the forward recursion alone, one item per cluster.
template <int NP, int TR>
__global__ void __launch_bounds__(512, 1) hmm_forward_cluster(const __grid_constant__ MmaWideLaunch a) {
  cluster_body<NP, 0, false, TR>(a, (int)(blockIdx.x / ClusterCfg<NP>::CL));
}

// Both passes of the adjoint in one launch (they are independent): clusters
// [0, nf) take the forward items of f, the others the backward items of b.
template <int NP, int TR>
__global__ void __launch_bounds__(512, 1)
hmm_cluster_passes(const __grid_constant__ MmaWideLaunch f, const __grid_constant__ MmaWideLaunch b,
                   int nf) {
  const int c = (int)(blockIdx.x / ClusterCfg<NP>::CL);
  if (c < nf) cluster_body<NP, 0, true, TR>(f, c);
  else cluster_body<NP, 1, true, TR>(b, c - nf);
}

// Clusters of CL CTAs, one CTA per SM (the shared memory takes it all).
template <int NP, typename Kern, typename... Args>
static cudaError_t launch_clusters(Kern kern, int n_clusters, int M, cudaStream_t st, Args... args) {
  using L = ClusterCfg<NP>;
  const int smem = L::total(M);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_clusters * L::CL), 1, 1);
  cfg.blockDim = dim3(L::NTH, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Whether the cluster forward serves N_pad = NP with M symbols (its emission
// slice must fit beside the resident X and A slice).
bool forward_cluster_fits(int NP, int M) {
  if (NP == 256) return ClusterCfg<256>::total(M) <= 227 * 1024;
  if (NP == 512) return ClusterCfg<512>::total(M) <= 227 * 1024;
  return false;
}

// Rows per tile: the fewest (32, 64 or 128) for which the clusters of all
// tiles (times `dirs` directions) still fit the GPU in one wave -- the product
// stays M = 128 (rows past the tile are zero) while each step's exchange
// shrinks with the rows; 128 when even that does not fit.
int cluster_tile_rows(int NP, int S, int K, int dirs) {
  const int cl = NP / 64;
  for (int tr = 32; tr < 128; tr *= 2)
    if ((long long)((S + tr - 1) / tr) * K * dirs * cl <= num_sms()) return tr;
  return 128;
}

template <int NP, int TR>
static cudaError_t forward_cluster_t(const MmaWideLaunch& a, cudaStream_t st) {
  return launch_clusters<NP>(hmm_forward_cluster<NP, TR>, a.n_items, a.seq.M, st, a);
}
template <int NP, int TR>
static cudaError_t passes_cluster_t(const MmaWideLaunch& f, const MmaWideLaunch& b, cudaStream_t st) {
  return launch_clusters<NP>(hmm_cluster_passes<NP, TR>, f.n_items + b.n_items, f.seq.M, st, f, b,
                             f.n_items);
}

cudaError_t launch_forward_cluster(int NP, const MmaWideLaunch& a, cudaStream_t st) {
  if (a.xs || a.n_items < 1 || a.n_tiles != (a.seq.S + a.rows - 1) / a.rows) return cudaErrorInvalidValue;
  if (NP == 256 && a.rows == 32) return forward_cluster_t<256, 32>(a, st);
  if (NP == 256 && a.rows == 64) return forward_cluster_t<256, 64>(a, st);
  if (NP == 256 && a.rows == 128) return forward_cluster_t<256, 128>(a, st);
  if (NP == 512 && a.rows == 32) return forward_cluster_t<512, 32>(a, st);
  if (NP == 512 && a.rows == 64) return forward_cluster_t<512, 64>(a, st);
  if (NP == 512 && a.rows == 128) return forward_cluster_t<512, 128>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_cluster_passes(int NP, const MmaWideLaunch& f, const MmaWideLaunch& b,
                                  cudaStream_t st) {
  if (!f.xs || !b.xs || !b.xe || !f.roff || f.n_items < 1 || b.n_items != f.n_items ||
      b.rows != f.rows || f.n_tiles != (f.seq.S + f.rows - 1) / f.rows)
    return cudaErrorInvalidValue;
  if (NP == 256 && f.rows == 32) return passes_cluster_t<256, 32>(f, b, st);
  if (NP == 256 && f.rows == 64) return passes_cluster_t<256, 64>(f, b, st);
  if (NP == 256 && f.rows == 128) return passes_cluster_t<256, 128>(f, b, st);
  if (NP == 512 && f.rows == 32) return passes_cluster_t<512, 32>(f, b, st);
  if (NP == 512 && f.rows == 64) return passes_cluster_t<512, 64>(f, b, st);
  if (NP == 512 && f.rows == 128) return passes_cluster_t<512, 128>(f, b, st);
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
