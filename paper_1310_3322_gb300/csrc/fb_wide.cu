// fb_wide.cu -- expected counts of the adjoint from every step's rows
// (Baum-Welch E-step, Sec. 2.7; Rabiner 1989 eqs. 37-38): above 128 states
// (BF16 passes of mma_cluster.cu, a block of rows per model) and for the TF32
// adjoint at N_pad = 128 (passes of mma_pass_tf32.cu, rows in the tile plan's
// order, each model's rows [mrow[k], mrow[K + 1 + k])). The passes leave:
//   X_t      scaled alpha_t (any power-of-two scale per step),
//   Bh_t     scaled beta_t = D_t 2^-f_t, D_t = A (b(o_{t+1}) o Bh_{t+1}) the
//            backward pass's product, f_t its exponent.
// With z_t = X_t . Bh_t (so that X_t . D_t = 2^f_t z_t):
//   gamma_t(i) = X_t(i) Bh_t(i) / z_t
//   xi_t(i, j) = [X_t(i) / z_t] a_ij [b_j(o_{t+1}) Bh_{t+1}(j) 2^-f_t]
// so the transition counts of a model are A o (U^T V), U_t = w X_t / z_t and
// V_t = b(o_{t+1}) o Bh_{t+1} 2^-f_t over every step t < T - 1 of every
// sequence: one contraction over all rows, run on the tensor cores with TF32
// operands (U and V rounded to TF32, relative error <= 2^-11 each; FP32
// accumulation) as a split-K GEMM whose partial tiles are summed in a fixed
// order (at N_pad = 128 its row chunks are staged by bulk copies). Emission
// and initial counts are
// sums of gamma rows by symbol and at t = 0: the rows of each model sorted by
// symbol (a stable counting sort), whole rows summed per piece of a symbol's
// rows, then the pieces in a fixed order. Everything is bitwise
// reproducible.
#include <algorithm>

#include "hmm_internal.cuh"
#include "tc.cuh"

namespace hmmgb {


// Largest s with roff[s] <= r (roff non-decreasing, roff[0] = 0).
__device__ __forceinline__ int seq_of_row(const int64_t* roff, int S, int64_t r) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(roff + mid) <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Rows in the plan's order: row_pos[rel] = the position whose rows
// [pos_row[p], pos_row[p + 1]) (the last: up to the rows used) hold rel --
// the largest p with pos_row[p] <= rel. One warp per position.
__global__ void fbw_rowpos_kernel(FbWideArgs a) {
  const int p = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int n = __ldg(a.n_valid);
  if (p >= n) return;
  const int64_t used = a.labelled ? a.mrow[a.K] : a.mrow[a.K + 1] - a.mrow[0];
  const int64_t b = a.pos_row[p];
  const int64_t e = min(used, p + 1 < n ? a.pos_row[p + 1] : used);
  for (int64_t r = b + lane; r < e; r += 32) a.row_pos[r] = p;
}

// Row r's model k, sequence s and step t (t = -1: no row).
__device__ __forceinline__ void locate_row(const FbWideArgs& a, int64_t r, int& k, int& s,
                                           int64_t& t) {
  k = 0;
  s = 0;
  t = -1;
  if (a.pos_row) {
    // rows in the plan's order: labelled, one run of rows for all models;
    // otherwise a block of rtot rows per model
    const int n = __ldg(a.n_valid);
    const int64_t rel = a.labelled ? r : r % a.rtot;
    const int64_t used = a.labelled ? a.mrow[a.K] : a.mrow[a.K + 1] - a.mrow[0];
    if (n > 0 && rel < used) {
      const int pos = a.row_pos ? a.row_pos[rel] : seq_of_row(a.pos_row, n, rel);
      s = a.sorted[pos];
      t = rel - a.pos_row[pos];
      k = a.labelled ? a.model_of_seq[s] : (int)(r / a.rtot);
    }
  } else {
    k = (int)(r / a.rtot);
    const int64_t rr = r % a.rtot;
    s = seq_of_row(a.roff, a.S, rr);
    t = rr - a.roff[s];
  }
}

// Rows of one combine block: 32 KB of X rows (and as many Bh rows plus the
// one after, whose emission product V needs), staged in shared memory by two
// bulk copies, beside 32 bytes of scalars per row.
template <int NP>
struct CombineCfg {
  static constexpr int RB = 8192 / NP;          // rows per block: 64, 32, 16
  static constexpr int XB = RB * NP * 4;        // X rows
  static constexpr int BB = (RB + 1) * NP * 4;  // Bh rows
  static constexpr int SC = XB + BB;            // per-row scalars [RB][8] ints
  static constexpr int BAR = SC + RB * 32;
  static constexpr int SMEM = BAR + 16;
};
constexpr uint32_t kCombineWait = 1u << 24;

// One block per RB consecutive rows (model k, step t of sequence s): V, G, the
// row's symbol code (m, or m | 1 << 30 at t = 0; -1 = no counts) and U: in
// place of X (u_in_x), or, where every row the contraction reads holds a
// finite X, X itself with w / z_t folded into V (U^T V is the same sum).
// Thread 0 starts the bulk copies of the block's X and Bh rows; meanwhile
// thread u < RB locates row u and loads its scalars; then each warp takes
// every eighth row from shared memory (lane l: float4 groups l, l + 32, ..).
// The copies' wait is bounded: a give-up records HMM_STATUS_TIMEOUT, waits
// for the copies once more and leaves the block's rows without counts.
template <int NP>
__global__ void __launch_bounds__(256) fbw_combine_kernel(FbWideArgs a) {
  using C = CombineCfg<NP>;
  constexpr int Q = NP / 128;  // float4 groups per lane
  extern __shared__ __align__(1024) uint8_t smem[];
  const float4* sX = reinterpret_cast<const float4*>(smem);
  const float4* sB = reinterpret_cast<const float4*>(smem + C::XB);
  int* sc = reinterpret_cast<int*>(smem + C::SC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t rb = (int64_t)blockIdx.x * C::RB;
  const int n = (int)min((int64_t)C::RB, a.nrows - rb);       // >= 1 (grid)
  const int nb = (int)min((int64_t)C::RB + 1, a.nrows - rb);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc::mbar_arrive_expect_tx(bar, (uint32_t)((n + nb) * NP * 4));
    tc::bulk_g2s(tc::smem_u32(smem), a.X + rb * NP, (uint32_t)(n * NP * 4), bar);
    tc::bulk_g2s(tc::smem_u32(smem + C::XB), a.Bh + rb * NP, (uint32_t)(nb * NP * 4), bar);
  }
  if (tid < n) {
    int k = 0, s = 0, T = 0, m = -1, on = 0, xe = 0;
    int64_t t = -1;
    float w = 1.f;
    locate_row(a, rb + tid, k, s, t);
    const int Ts = a.seqlen[s];
    if (Ts > 0 && t >= 0 && t < Ts) {
      T = Ts;
      const int32_t* o = a.symbols + a.offsets[s];
      if (a.weight) w = __ldg(a.weight + (a.labelled ? (size_t)s : (size_t)s * a.K + k));
      m = __ldg(o + t);
      if (t + 1 < Ts) {
        on = __ldg(o + t + 1);
        if ((unsigned)on >= (unsigned)a.M) on = 0;  // flagged by the passes already
        xe = a.xe[rb + tid];
      }
    } else {
      t = -1;
    }
    int* p = sc + tid * 8;
    p[0] = k; p[1] = T; p[2] = (int)t; p[3] = __float_as_int(w);
    p[4] = m; p[5] = on; p[6] = xe;
  }
  __syncthreads();  // the barrier's init and the scalars
  bool landed = tc::mbar_wait_bounded(bar, 0, kCombineWait);
  if (!landed) {
    if (tid == 0) set_status(a.status, HMM_STATUS_TIMEOUT);
    tc::mbar_wait_bounded(bar, 0, kCombineWait);  // the copies write this block's memory
  }
  for (int u = warp; u < n; u += 8) {
    const int64_t r = rb + u;
    const int* p = sc + u * 8;
    const int k = p[0], T = landed ? p[1] : 0, t = p[2];
    const float w = __int_as_float(p[3]);
    const int m = p[4], onext = p[5], xe = p[6];
    const bool ok = T > 0;
    float4 x[Q], bh[Q];
    float z = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      x[q] = ok ? sX[u * (NP / 4) + lane + 32 * q] : make_float4(0.f, 0.f, 0.f, 0.f);
      bh[q] = ok ? sB[u * (NP / 4) + lane + 32 * q] : make_float4(0.f, 0.f, 0.f, 0.f);
      z += (x[q].x * bh[q].x + x[q].y * bh[q].y) + (x[q].z * bh[q].z + x[q].w * bh[q].w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(HMM_FULL_MASK, z, o);
    // impossible, invalid or zero-weight pairs contribute nothing
    const bool use = ok && z > 0.f && z < INFINITY && w != 0.f && !isnan(w);
    const bool trans = use && t + 1 < T;
    const float iz = use ? w / z : 0.f;
    const float fac = trans ? exp2i(-xe) : 0.f;
    const float vs = a.u_in_x ? fac : fac * iz;  // V's factor
    const float4* bn = reinterpret_cast<const float4*>(a.Btp + ((size_t)k * a.M + onext) * NP);
    float4* Xw = reinterpret_cast<float4*>(a.X + r * NP);
    float4* Vr = reinterpret_cast<float4*>(a.V + r * NP);
    float4* Gr = reinterpret_cast<float4*>(a.G + r * NP);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float4 xv = x[q], bv = bh[q];
      Gr[lane + 32 * q] = make_float4(xv.x * bv.x * iz, xv.y * bv.y * iz, xv.z * bv.z * iz,
                                      xv.w * bv.w * iz);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (trans) {  // row u + 1 < nb: the sequence's next step is a row of the buffer
        const float4 e = __ldg(bn + lane + 32 * q), nbv = sB[(u + 1) * (NP / 4) + lane + 32 * q];
        v = make_float4(e.x * nbv.x * vs, e.y * nbv.y * vs, e.z * nbv.z * vs, e.w * nbv.w * vs);
      }
      Vr[lane + 32 * q] = v;
      if (a.u_in_x)
        Xw[lane + 32 * q] = trans ? make_float4(xv.x * iz, xv.y * iz, xv.z * iz, xv.w * iz)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (lane == 0) {
      int code = -1;
      if (use) code = (unsigned)m < (unsigned)a.M ? (m | (t == 0 ? (1 << 30) : 0)) : -1;
      a.sym[r] = code;
    }
  }
}

// Cp[k][split] = sum over the split's rows of U[r]^T V[r] on the tensor
// cores: one CTA per (128 x TN output tile, split, model; TN = 256, or 128 at
// N_pad = 128), D in tensor memory (TN FP32 columns). Model k's rows are
// [mrow[k], mrow[K + 1 + k]) (without mrow, the block k rtot .. (k + 1) rtot),
// cut into nsplit splits of a multiple of 32 rows. Rows are taken 32 at a
// time: 256 threads load the chunk's U columns (128 states) and V columns (TN
// states) from the
// row-major buffers -- every warp load reads 32 consecutive states of one
// row -- round them to TF32 and write them as K-major core matrices (8
// states x 4 rows, 16 bytes per state) into one of two shared-memory stages;
// thread 0 then issues four MMAs (M = 128, N = TN, K = 8 rows each,
// kind::tf32) and commits them to the stage's mbarrier, while the threads
// load the next chunk into the other stage. Rows past the split's end count
// as zero. Every wait is bounded; a give-up records HMM_STATUS_TIMEOUT.
constexpr int kFbwTileN = 256;      // output tile: 128 states i x 256 states j
constexpr int kFbwRows = 32;        // rows per chunk (K of four MMAs)
constexpr uint32_t kFbwWait = 1u << 24;
constexpr int kFbwStageA = 128 * kFbwRows * 4;         // 16 KB
constexpr int kFbwStageB = kFbwTileN * kFbwRows * 4;   // 32 KB
constexpr int kFbwSmem = 2 * (kFbwStageA + kFbwStageB) + 64;

template <int NP, int TN>
__global__ void __launch_bounds__(256, 1) fbw_gemm_kernel(FbWideArgs a) {
  constexpr int NJ = NP / TN;
  constexpr int VQ = TN / 32;  // row quads of V per thread (8 or 4)
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                              // [2][kFbwStageA]
  uint8_t* sB = smem + 2 * kFbwStageA;             // [2][kFbwStageB]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * (kFbwStageA + kFbwStageB));
  uint64_t* done = bars;      // [2]: the chunk's MMAs have read the stage
  uint64_t* fin = bars + 2;   // every MMA of the CTA is done
  volatile uint32_t* slot = reinterpret_cast<volatile uint32_t*>(bars + 3);
  const int mi = blockIdx.x / NJ, nj = blockIdx.x % NJ;
  const int split = blockIdx.y, k = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t beg = a.mrow ? a.mrow[k] : (int64_t)k * a.rtot;
  const int64_t end = a.mrow ? a.mrow[a.K + 1 + k] : beg + a.rtot;
  const int64_t rps = ((end - beg + a.nsplit - 1) / a.nsplit + kFbwRows - 1) / kFbwRows * kFbwRows;
  const int64_t r0 = beg + (int64_t)split * rps;
  const int64_t r1 = min(end, r0 + rps);
  const int nch = r1 > r0 ? (int)((r1 - r0 + kFbwRows - 1) / kFbwRows) : 0;
  const float* Uk = a.X + 128 * mi;
  const float* Vk = a.V + TN * nj;

  if (warp == 0) tc::tmem_alloc(const_cast<uint32_t*>(slot), 256);
  if (tid == 0) {
    tc::mbar_init(&done[0], 1);
    tc::mbar_init(&done[1], 1);
    tc::mbar_init(fin, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  constexpr uint32_t idesc = tc::instr_desc(2, 128, TN);
  bool ok = true;

  // this thread's share of a chunk: U column ia for row quads qa, qa + 2, ..;
  // V column jb for row quads qb, qb + 256 / TN, ..
  const int ia = tid & 127, qa = tid >> 7;
  const int jb = tid % TN, qb = tid / TN;
  for (int ch = 0; ch < nch; ++ch) {
    const int st = ch & 1;
    const int64_t rb = r0 + (int64_t)ch * kFbwRows;
    float u[4][4], v[VQ][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t r = rb + 4 * (qa + 2 * m) + e;
        u[m][e] = r < r1 ? __ldg(Uk + r * NP + ia) : 0.f;
      }
#pragma unroll
    for (int q = 0; q < VQ; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t r = rb + 4 * (qb + (256 / TN) * q) + e;
        v[q][e] = r < r1 ? __ldg(Vk + r * NP + jb) : 0.f;
      }
    // the stage's previous chunk (ch - 2) must have been read by its MMAs
    if (ch >= 2 && !tc::mbar_wait_bounded(&done[st], (uint32_t)((ch >> 1) + 1) & 1u, kFbwWait))
      ok = false;
    uint8_t* A = sA + st * kFbwStageA;
    uint8_t* B = sB + st * kFbwStageB;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      *reinterpret_cast<uint4*>(A + (ia >> 3) * 1024 + (qa + 2 * m) * 128 + (ia & 7) * 16) =
          make_uint4(tc::to_tf32(u[m][0]), tc::to_tf32(u[m][1]), tc::to_tf32(u[m][2]),
                     tc::to_tf32(u[m][3]));
#pragma unroll
    for (int q = 0; q < VQ; ++q)
      *reinterpret_cast<uint4*>(B + (jb >> 3) * 1024 + (qb + (256 / TN) * q) * 128 + (jb & 7) * 16) =
          make_uint4(tc::to_tf32(v[q][0]), tc::to_tf32(v[q][1]), tc::to_tf32(v[q][2]),
                     tc::to_tf32(v[q][3]));
    tc::fence_proxy_async();  // the stage's generic writes -> tensor core
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t aA = tc::smem_u32(A), aB = tc::smem_u32(B);
#pragma unroll
      for (int kk = 0; kk < kFbwRows / 8; ++kk)
        tc::mma_tf32(tmem, tc::smem_desc(aA + kk * 256, 128, 1024),
                     tc::smem_desc(aB + kk * 256, 128, 1024), idesc, (ch | kk) ? 1u : 0u);
      tc::mma_commit(&done[st]);
    }
  }
  if (tid == 0) tc::mma_commit(fin);  // arrives once every MMA above is done
  if (!tc::mbar_wait_bounded(fin, 0, kFbwWait)) ok = false;
  tc::fence_after_sync();
  if (!ok) set_status(a.status, HMM_STATUS_TIMEOUT);
  // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (states i), columns
  // TN / 2 (w / 4) .. + TN / 2 - 1 (states j)
  const int i = 128 * mi + 32 * (warp & 3) + lane;
  const int jc = (TN / 2) * (warp >> 2);
  float* dst = a.Cp + ((size_t)k * a.nsplit + split) * NP * NP + (size_t)i * NP + TN * nj + jc;
#pragma unroll 1
  for (int c = 0; c < TN / 64; ++c) {
    float y[32];
    tc::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(jc + 32 * c), y);
    tc::tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(dst + 32 * c + 4 * q) =
          nch > 0 ? make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3])
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// The contraction at N_pad = 128 (the TF32 adjoint, one 128 x 128 output
// tile): whole 32-row chunks of X and V (16 KB each) are copied by thread 0
// with cp.async.bulk into kFbwRaw shared-memory stages, kFbwRaw - 1 chunks
// ahead, so about 96 KB of rows are in flight per SM without registers (one
// CTA per SM); the threads then take the chunk from shared memory and form
// the operands as the kernel above. A stage is refilled at the top of the
// chunk after its last reader's barrier. Every wait is bounded; after a
// give-up the last copy into every stage is awaited once more before exit.
constexpr int kFbwRaw = 4;
constexpr int kFbwRawFloats = 2 * kFbwRows * 128;              // X and V rows of a chunk
constexpr int kFbwOp128 = 2 * kFbwRows * 128 * 4;              // A and B stage: 32 KB
constexpr int kFbwSmem128 = 2 * kFbwOp128 + kFbwRaw * kFbwRawFloats * 4 + 128;

__global__ void __launch_bounds__(256, 1) fbw_gemm128_kernel(FbWideArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sOp = smem;                                                // [2][A | B]
  float* sRaw = reinterpret_cast<float*>(smem + 2 * kFbwOp128);       // [kFbwRaw][X | V]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kFbwOp128 + kFbwRaw * kFbwRawFloats * 4);
  uint64_t* done = bars;            // [2]: the chunk's MMAs have read the operand stage
  uint64_t* fin = bars + 2;         // every MMA of the CTA is done
  uint64_t* full = bars + 3;        // [kFbwRaw]: the chunk's rows have landed
  volatile uint32_t* slot = reinterpret_cast<volatile uint32_t*>(bars + 3 + kFbwRaw);
  const int split = blockIdx.y, k = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t beg = a.mrow ? a.mrow[k] : (int64_t)k * a.rtot;
  const int64_t end = a.mrow ? a.mrow[a.K + 1 + k] : beg + a.rtot;
  const int64_t rps = ((end - beg + a.nsplit - 1) / a.nsplit + kFbwRows - 1) / kFbwRows * kFbwRows;
  const int64_t r0 = beg + (int64_t)split * rps;
  const int64_t r1 = min(end, r0 + rps);
  const int nch = r1 > r0 ? (int)((r1 - r0 + kFbwRows - 1) / kFbwRows) : 0;
  auto issue = [&](int c) {  // thread 0: chunk c into raw stage c % kFbwRaw
    const int64_t rb = r0 + (int64_t)c * kFbwRows;
    const uint32_t bytes = (uint32_t)min((int64_t)kFbwRows, r1 - rb) * 512u;
    float* dst = sRaw + (size_t)(c % kFbwRaw) * kFbwRawFloats;
    uint64_t* b = &full[c % kFbwRaw];
    tc::mbar_arrive_expect_tx(b, 2 * bytes);
    tc::bulk_g2s(tc::smem_u32(dst), a.X + rb * 128, bytes, b);
    tc::bulk_g2s(tc::smem_u32(dst + kFbwRows * 128), a.V + rb * 128, bytes, b);
  };

  if (warp == 0) tc::tmem_alloc(const_cast<uint32_t*>(slot), 256);
  if (tid == 0) {
    tc::mbar_init(&done[0], 1);
    tc::mbar_init(&done[1], 1);
    tc::mbar_init(fin, 1);
    for (int i = 0; i < kFbwRaw; ++i) tc::mbar_init(&full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int c = 0; c < kFbwRaw - 1 && c < nch; ++c) issue(c);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  constexpr uint32_t idesc = tc::instr_desc(2, 128, 128);
  bool ok = true;

  // this thread's share of a chunk: U column ia and V column ia, row quads
  // qa, qa + 2, ..
  const int ia = tid & 127, qa = tid >> 7;
  for (int ch = 0; ch < nch; ++ch) {
    const int st = ch & 1;
    if (tid == 0 && ch + kFbwRaw - 1 < nch) issue(ch + kFbwRaw - 1);
    const int rs = ch % kFbwRaw;
    const bool landed = tc::mbar_wait_bounded(&full[rs], (uint32_t)(ch / kFbwRaw) & 1u, kFbwWait);
    if (!landed) ok = false;
    const float* sX = sRaw + (size_t)rs * kFbwRawFloats;
    const float* sV = sX + kFbwRows * 128;
    const int64_t rb = r0 + (int64_t)ch * kFbwRows;
    float u[4][4], v[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int rl = 4 * (qa + 2 * m) + e;
        const bool in = landed && rb + rl < r1;
        u[m][e] = in ? sX[rl * 128 + ia] : 0.f;
        v[m][e] = in ? sV[rl * 128 + ia] : 0.f;
      }
    // the operand stage's previous chunk (ch - 2) must have been read by its MMAs
    if (ch >= 2 && !tc::mbar_wait_bounded(&done[st], (uint32_t)((ch >> 1) + 1) & 1u, kFbwWait))
      ok = false;
    uint8_t* A = sOp + st * kFbwOp128;
    uint8_t* B = A + kFbwOp128 / 2;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int off = (ia >> 3) * 1024 + (qa + 2 * m) * 128 + (ia & 7) * 16;
      *reinterpret_cast<uint4*>(A + off) =
          make_uint4(tc::to_tf32(u[m][0]), tc::to_tf32(u[m][1]), tc::to_tf32(u[m][2]),
                     tc::to_tf32(u[m][3]));
      *reinterpret_cast<uint4*>(B + off) =
          make_uint4(tc::to_tf32(v[m][0]), tc::to_tf32(v[m][1]), tc::to_tf32(v[m][2]),
                     tc::to_tf32(v[m][3]));
    }
    tc::fence_proxy_async();  // the stage's generic writes -> tensor core
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t aA = tc::smem_u32(A), aB = tc::smem_u32(B);
#pragma unroll
      for (int kk = 0; kk < kFbwRows / 8; ++kk)
        tc::mma_tf32(tmem, tc::smem_desc(aA + kk * 256, 128, 1024),
                     tc::smem_desc(aB + kk * 256, 128, 1024), idesc, (ch | kk) ? 1u : 0u);
      tc::mma_commit(&done[st]);
    }
  }
  if (tid == 0) tc::mma_commit(fin);  // arrives once every MMA above is done
  if (!tc::mbar_wait_bounded(fin, 0, kFbwWait)) ok = false;
  tc::fence_after_sync();
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      set_status(a.status, HMM_STATUS_TIMEOUT);
      for (int s = 0; s < kFbwRaw && s < nch; ++s) {  // the last copy into each stage
        const int last = s + kFbwRaw * ((nch - 1 - s) / kFbwRaw);
        tc::mbar_wait_bounded(&full[s], (uint32_t)(last / kFbwRaw) & 1u, kFbwWait);
      }
    }
    __syncthreads();
  }
  // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (states i), columns
  // 64 (w / 4) .. + 63 (states j)
  const int i = 32 * (warp & 3) + lane;
  const int jc = 64 * (warp >> 2);
  float* dst = a.Cp + ((size_t)k * a.nsplit + split) * 128 * 128 + (size_t)i * 128 + jc;
#pragma unroll 1
  for (int c = 0; c < 2; ++c) {
    float y[32];
    tc::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(jc + 32 * c), y);
    tc::tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(dst + 32 * c + 4 * q) =
          nch > 0 ? make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3])
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// cnt_A[k][i][j] = a_ij * sum over splits (fixed order).
__global__ void fbw_reduce_a_kernel(FbWideArgs a) {
  const int64_t n = (int64_t)a.K * a.N * a.N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / ((int64_t)a.N * a.N));
    const int i = (int)((idx / a.N) % a.N), j = (int)(idx % a.N);
    const float* c = a.Cp + (size_t)k * a.nsplit * a.NP * a.NP + (size_t)i * a.NP + j;
    float sum = 0.f;
    for (int p = 0; p < a.nsplit; ++p) sum += c[(size_t)p * a.NP * a.NP];
    a.cnt_A[idx] = sum * __ldg(a.A + ((size_t)k * a.N + i) * a.N + j);
  }
}

// Emission and initial counts by symbol: a stable counting sort of each
// model's rows by bucket (bucket m < M: rows whose symbol is m; bucket M: the
// rows at t = 0, which also sit in their symbol's bucket), then one warp per
// piece of at most kEmisPiece entries of a bucket sums those gamma rows in
// registers (whole rows, NP / 4 float4 per row), then the pieces of every
// bucket are summed in order. The sort and the pieces depend on the symbols
// only, so the counts are bitwise reproducible.
constexpr int kEmisPiece = 256;

__device__ __forceinline__ void model_rows(const FbWideArgs& a, int k, int64_t& beg,
                                           int64_t& end) {
  beg = a.mrow ? a.mrow[k] : (int64_t)k * a.rtot;
  end = a.mrow ? a.mrow[a.K + 1 + k] : beg + a.rtot;
}

// Exclusive scan of v over a block of 1024 threads; total = the sum.
__device__ __forceinline__ int scan1024(int v, int* s, int& total) {
  const int tid = threadIdx.x;
  s[tid] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int y = tid >= o ? s[tid - o] : 0;
    __syncthreads();
    s[tid] += y;
    __syncthreads();
  }
  total = s[1023];
  const int r = s[tid] - v;
  __syncthreads();
  return r;
}

// One block: cbase[k] = first chunk of model k (ceil(rows / ech) chunks a
// model), cbase[K] = all chunks.
__global__ void __launch_bounds__(1024) fbw_echunks_kernel(FbWideArgs a) {
  __shared__ int s[1024];
  const int per = (a.K + 1023) / 1024;
  const int k0 = min(a.K, (int)threadIdx.x * per), k1 = min(a.K, k0 + per);
  auto chunks = [&](int k) {
    int64_t beg, end;
    model_rows(a, k, beg, end);
    return end > beg ? (int)((end - beg + a.ech - 1) / a.ech) : 0;
  };
  int v = 0;
  for (int k = k0; k < k1; ++k) v += chunks(k);
  int total;
  int o = scan1024(v, s, total);
  for (int k = k0; k < k1; ++k) {
    a.cbase[k] = o;
    o += chunks(k);
  }
  if (threadIdx.x == 0) a.cbase[a.K] = total;
}

// Chunk g (< cbase[K]): its model k (the last one whose first chunk is <= g)
// and its rows [r0, r1).
__device__ __forceinline__ int chunk_rows(const FbWideArgs& a, int g, int64_t& r0, int64_t& r1) {
  int lo = 0, hi = a.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.cbase[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  int64_t beg, end;
  model_rows(a, lo, beg, end);
  r0 = beg + (int64_t)(g - a.cbase[lo]) * a.ech;
  r1 = min(end, r0 + a.ech);
  return lo;
}

// ehist[m][g] = entries of bucket m among the rows of chunk g.
__global__ void __launch_bounds__(256) fbw_ehist_kernel(FbWideArgs a) {
  extern __shared__ int h[];  // [M + 1]
  const int g = blockIdx.x, nb = a.M + 1;
  if (g >= a.cbase[a.K]) return;
  for (int m = threadIdx.x; m < nb; m += blockDim.x) h[m] = 0;
  __syncthreads();
  int64_t r0, r1;
  chunk_rows(a, g, r0, r1);
#pragma unroll 4
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int code = __ldg(a.sym + r);
    if (code < 0) continue;
    atomicAdd(&h[code & 0xffffff], 1);
    if (code >> 30) atomicAdd(&h[a.M], 1);
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nb; m += blockDim.x) a.ehist[(size_t)m * a.ncc + g] = h[m];
}

// One warp per bucket b = (k, m): ehist[m][g] over model k's chunks g
// becomes the bucket's entries in the chunks before g, ebase[b] its total.
__global__ void fbw_escan1_kernel(FbWideArgs a) {
  const int nb = a.M + 1;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= (int64_t)a.K * nb) return;
  const int k = (int)(b / nb), m = (int)(b % nb);
  int* hrow = a.ehist + (size_t)m * a.ncc;
  const int g1 = min(a.cbase[k + 1], a.ncc);
  int carry = 0;
  for (int g0 = a.cbase[k]; g0 < g1; g0 += 32) {
    const int g = g0 + lane;
    const int v = g < g1 ? hrow[g] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(HMM_FULL_MASK, x, o);
      if (lane >= o) x += y;
    }
    if (g < g1) hrow[g] = carry + x - v;
    carry += __shfl_sync(HMM_FULL_MASK, x, 31);
  }
  if (lane == 0) a.ebase[b] = carry;
}

// One block: ebase becomes the first entry of every bucket (ebase[nbk] = all
// entries) and epbase the first piece (epbase[nbk] = all pieces).
__global__ void __launch_bounds__(1024) fbw_escan2_kernel(FbWideArgs a) {
  __shared__ int s[1024];
  const int nbk = a.K * (a.M + 1);
  const int per = (nbk + 1023) / 1024;
  const int b0 = min(nbk, (int)threadIdx.x * per), b1 = min(nbk, b0 + per);
  int se = 0, sp = 0;
  for (int b = b0; b < b1; ++b) {
    const int t = a.ebase[b];
    se += t;
    sp += (t + kEmisPiece - 1) / kEmisPiece;
  }
  int te, tp;
  int oe = scan1024(se, s, te);
  int op = scan1024(sp, s, tp);
  for (int b = b0; b < b1; ++b) {
    const int t = a.ebase[b];
    a.ebase[b] = oe;
    a.epbase[b] = op;
    oe += t;
    op += (t + kEmisPiece - 1) / kEmisPiece;
  }
  if (threadIdx.x == 0) {
    a.ebase[nbk] = te;
    a.epbase[nbk] = tp;
  }
}

// One warp per chunk, its rows in order (256 codes loaded at a time): each
// entry goes to elist at its bucket's base + the chunk's offset + its rank
// among the chunk's earlier entries of the bucket.
__global__ void __launch_bounds__(32) fbw_escatter_kernel(FbWideArgs a) {
  extern __shared__ int cur[];  // [M + 1] next position per bucket
  const int g = blockIdx.x, nb = a.M + 1, lane = threadIdx.x;
  if (g >= a.cbase[a.K]) return;
  int64_t r0, r1;
  const int k = chunk_rows(a, g, r0, r1);
  const int64_t bk = (int64_t)k * nb;
  for (int m = lane; m < nb; m += 32) cur[m] = a.ebase[bk + m] + a.ehist[(size_t)m * a.ncc + g];
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t rb = r0; rb < r1; rb += 256) {
    int code[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t r = rb + u * 32 + lane;
      code[u] = r < r1 ? __ldg(a.sym + r) : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int32_t r = (int32_t)(rb + u * 32 + lane);
      const int key = code[u] < 0 ? -1 : (code[u] & 0xffffff);
      const unsigned same = __match_any_sync(HMM_FULL_MASK, key);
      const int pos = key >= 0 ? cur[key] + __popc(same & lt) : 0;
      __syncwarp();
      if (key >= 0) {
        a.elist[pos] = r;
        if ((same & lt) == 0) cur[key] += __popc(same);  // first lane of the group
      }
      const bool first = key >= 0 && (code[u] >> 30) != 0;
      const unsigned fm = __ballot_sync(HMM_FULL_MASK, first);
      if (first) a.elist[cur[a.M] + __popc(fm & lt)] = r;
      __syncwarp();
      if (lane == 0) cur[a.M] += __popc(fm);
      __syncwarp();
    }
  }
}

// Warps over pieces (grid-stride): piece p of bucket b sums the gamma rows of
// entries ebase[b] + (p - epbase[b]) kEmisPiece ... (at most kEmisPiece) into
// epart[p]; lane l holds the float4 groups l, l + 32, ... of a row.
template <int NP>
__global__ void __launch_bounds__(256) fbw_epiece_kernel(FbWideArgs a) {
  constexpr int Q = NP / 128;   // float4 groups per lane
  constexpr int UN = 8 / Q;     // rows in flight per lane (4 KB per warp)
  const int nbk = a.K * (a.M + 1);
  const int npieces = a.epbase[nbk];
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float4* G = reinterpret_cast<const float4*>(a.G);
  for (int64_t p = wid; p < npieces; p += nw) {
    int lo = 0, hi = nbk - 1;  // the last bucket whose first piece is <= p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.epbase + mid) <= p) lo = mid;
      else hi = mid - 1;
    }
    const int e0 = __ldg(a.ebase + lo) + (int)(p - __ldg(a.epbase + lo)) * kEmisPiece;
    const int e1 = min(__ldg(a.ebase + lo + 1), e0 + kEmisPiece);
    float4 acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int eb = e0; eb < e1; eb += 32) {
      const int n = min(32, e1 - eb);
      const int myrow = lane < n ? __ldg(a.elist + eb + lane) : 0;
      for (int u0 = 0; u0 < n; u0 += UN) {
        float4 g[UN][Q];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const int64_t row = __shfl_sync(HMM_FULL_MASK, myrow, u0 + u);
#pragma unroll
          for (int q = 0; q < Q; ++q)
            g[u][q] = u0 + u < n ? __ldg(G + row * (NP / 4) + lane + 32 * q)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            acc[q].x += g[u][q].x;
            acc[q].y += g[u][q].y;
            acc[q].z += g[u][q].z;
            acc[q].w += g[u][q].w;
          }
      }
    }
    float4* out = reinterpret_cast<float4*>(a.epart + p * NP);
#pragma unroll
    for (int q = 0; q < Q; ++q) out[lane + 32 * q] = acc[q];
  }
}

// cnt_B[k][j][m] (bucket m < M) and cnt_pi[k][j] (bucket M): the pieces of
// the bucket summed in order.
__global__ void fbw_ereduce_kernel(FbWideArgs a) {
  const int nb = a.M + 1;
  const int64_t n = (int64_t)a.K * nb * a.N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % a.N);
    const int b = (int)(idx / a.N);
    const int k = b / nb, m = b % nb;
    const int p1 = a.epbase[b + 1];
    float sum = 0.f;
    for (int p = a.epbase[b]; p < p1; ++p) sum += a.epart[(size_t)p * a.NP + j];
    if (m < a.M) a.cnt_B[((size_t)k * a.N + j) * a.M + m] = sum;
    else a.cnt_pi[(size_t)k * a.N + j] = sum;
  }
}

FbwEmisSizes fbw_emis_sizes(int K, int M, int NP, int64_t nrows) {
  FbwEmisSizes z;
  const int64_t rows = nrows > 0 ? nrows : 1;
  int64_t ech = (rows + 2047) / 2048;
  if (ech < 2048) ech = 2048;
  z.ech = (ech + 255) & ~(int64_t)255;
  z.ncc = (rows + z.ech - 1) / z.ech + K;  // sum over models of ceil(rows_k / ech)
  const int64_t nbk = (int64_t)K * (M + 1);
  z.ehist = (int64_t)(M + 1) * z.ncc;
  z.ebase = nbk + 1;
  z.elist = 2 * rows;  // a row is in its symbol's bucket, at t = 0 also in bucket M
  // sum over buckets of ceil(entries / piece) <= entries / piece + non-empty buckets
  z.epart = (z.elist / kEmisPiece + 1 + std::min(nbk, z.elist)) * NP;
  return z;
}

cudaError_t launch_fbw_counts(const FbWideArgs& a, cudaStream_t st) {
  cudaError_t e;
  if (a.row_pos) {
    if (!a.pos_row) return cudaErrorInvalidValue;
    fbw_rowpos_kernel<<<(unsigned)(((int64_t)a.S * 32 + 255) / 256), 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  auto combine = [&](auto kern, int rb, int sm) {
    const int64_t blocks = (a.nrows + rb - 1) / rb;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (ce != cudaSuccess) return ce;
    kern<<<(unsigned)blocks, 256, sm, st>>>(a);
    return cudaGetLastError();
  };
  if (a.nrows <= 0) return cudaErrorInvalidValue;
  if (a.NP == 128) e = combine(fbw_combine_kernel<128>, CombineCfg<128>::RB, CombineCfg<128>::SMEM);
  else if (a.NP == 256) e = combine(fbw_combine_kernel<256>, CombineCfg<256>::RB, CombineCfg<256>::SMEM);
  else if (a.NP == 512) e = combine(fbw_combine_kernel<512>, CombineCfg<512>::RB, CombineCfg<512>::SMEM);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  if (a.NP == 128) {
    if ((e = cudaFuncSetAttribute(fbw_gemm128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kFbwSmem128)) != cudaSuccess)
      return e;
    fbw_gemm128_kernel<<<dim3(1, a.nsplit, a.K), 256, kFbwSmem128, st>>>(a);
  } else {
    const dim3 gg((a.NP / 128) * (a.NP / kFbwTileN), a.nsplit, a.K);
    auto gk = a.NP == 256 ? fbw_gemm_kernel<256, 256> : fbw_gemm_kernel<512, 256>;
    if ((e = cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, kFbwSmem)) !=
        cudaSuccess)
      return e;
    gk<<<gg, 256, kFbwSmem, st>>>(a);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_reduce_a_kernel<<<1024, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t hsm = (size_t)(a.M + 1) * 4;
  // entries (<= 2 nrows) and row indices are 32-bit
  if (hsm > 48 * 1024 || 2 * a.nrows > INT32_MAX) return cudaErrorInvalidValue;
  fbw_echunks_kernel<<<1, 1024, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_ehist_kernel<<<a.ncc, 256, hsm, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t nbk = (int64_t)a.K * (a.M + 1);
  fbw_escan1_kernel<<<(unsigned)((nbk * 32 + 255) / 256), 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_escan2_kernel<<<1, 1024, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_escatter_kernel<<<a.ncc, 32, hsm, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned pg = (unsigned)(8 * num_sms());
  if (a.NP == 128) fbw_epiece_kernel<128><<<pg, 256, 0, st>>>(a);
  else if (a.NP == 256) fbw_epiece_kernel<256><<<pg, 256, 0, st>>>(a);
  else fbw_epiece_kernel<512><<<pg, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_ereduce_kernel<<<1024, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hmmgb
