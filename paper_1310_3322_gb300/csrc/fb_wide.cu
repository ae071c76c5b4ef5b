// fb_wide.cu -- expected counts of the adjoint above 128 states (Baum-Welch
// E-step, Sec. 2.7; Rabiner 1989 eqs. 37-38), from the per-step rows the
// tensor-core forward and backward passes of mma_wide.cu leave in memory:
//   X_t      scaled alpha_t (any power-of-two scale per step),
//   Bh_t     scaled beta_t = D_t 2^-f_t, D_t = A (b(o_{t+1}) o Bh_{t+1}) the
//            backward pass's product, f_t its exponent.
// With z_t = X_t . Bh_t (so that X_t . D_t = 2^f_t z_t):
//   gamma_t(i) = X_t(i) Bh_t(i) / z_t
//   xi_t(i, j) = [X_t(i) / z_t] a_ij [b_j(o_{t+1}) Bh_{t+1}(j) 2^-f_t]
// so the transition counts of a model are A o (U^T V), U_t = w X_t / z_t and
// V_t = b(o_{t+1}) o Bh_{t+1} 2^-f_t over every step t < T - 1 of every
// sequence: one contraction over all rows, run as a split-K SIMT GEMM whose
// partial tiles are summed in a fixed order. Emission and initial counts are
// sums of gamma rows by symbol and at t = 0, per chunk of rows in shared
// memory (thread j owns state j: no atomics), then over chunks in a fixed
// order. Everything is bitwise reproducible.
#include "hmm_internal.cuh"

namespace hmmgb {

constexpr int kFbwGemmTile = 128;   // output tile of the contraction (128 x 128)
constexpr int kFbwGemmRows = 8;     // rows per shared-memory stage

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

// One warp per row (model k, step t of sequence s): U (in place of X), V, G
// and the row's symbol code (m, or m | 1 << 30 at t = 0; -1 = no counts).
template <int NP>
__global__ void __launch_bounds__(256) fbw_combine_kernel(FbWideArgs a) {
  constexpr int Q = NP / 128;  // float4 groups per lane
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= (int64_t)a.K * a.rtot) return;
  const int k = (int)(r / a.rtot);
  const int64_t rr = r % a.rtot;
  const int s = seq_of_row(a.roff, a.S, rr);
  const int T = a.seqlen[s];
  const int64_t t64 = rr - a.roff[s];
  const bool row_ok = T > 0 && t64 >= 0 && t64 < T;
  const int t = row_ok ? (int)t64 : 0;
  float4* Xr = reinterpret_cast<float4*>(a.X + r * NP);
  const float4* Br = reinterpret_cast<const float4*>(a.Bh + r * NP);
  float4* Vr = reinterpret_cast<float4*>(a.V + r * NP);
  float4* Gr = reinterpret_cast<float4*>(a.G + r * NP);
  float4 x[Q], bh[Q];
  float z = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    x[q] = row_ok ? Xr[lane + 32 * q] : make_float4(0.f, 0.f, 0.f, 0.f);
    bh[q] = row_ok ? __ldg(Br + lane + 32 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
    z += (x[q].x * bh[q].x + x[q].y * bh[q].y) + (x[q].z * bh[q].z + x[q].w * bh[q].w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(HMM_FULL_MASK, z, o);
  const float w = (row_ok && a.weight) ? __ldg(a.weight + (size_t)s * a.K + k) : 1.f;
  // impossible, invalid or zero-weight pairs contribute nothing
  const bool use = row_ok && z > 0.f && z < INFINITY && w != 0.f && !isnan(w);
  const bool trans = use && t + 1 < T;
  const float iz = use ? w / z : 0.f;
  float fac = 0.f;
  int onext = 0;
  const int32_t* o = a.symbols + (row_ok ? a.offsets[s] : 0);
  if (trans) {
    fac = exp2i(-a.xe[r]);
    onext = __ldg(o + t + 1);
    if ((unsigned)onext >= (unsigned)a.M) onext = 0;  // flagged by the passes already
  }
  const int kmod = a.labelled ? 0 : k;  // model of this row's parameters
  const float4* bn = reinterpret_cast<const float4*>(a.Btp + ((size_t)kmod * a.M + onext) * NP);
  const float4* bhn = reinterpret_cast<const float4*>(a.Bh + (r + 1) * NP);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float4 xv = x[q], bv = bh[q];
    Gr[lane + 32 * q] = make_float4(xv.x * bv.x * iz, xv.y * bv.y * iz, xv.z * bv.z * iz,
                                    xv.w * bv.w * iz);
    float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
    if (trans) {
      u = make_float4(xv.x * iz, xv.y * iz, xv.z * iz, xv.w * iz);
      const float4 e = __ldg(bn + lane + 32 * q), nb = __ldg(bhn + lane + 32 * q);
      v = make_float4(e.x * nb.x * fac, e.y * nb.y * fac, e.z * nb.z * fac, e.w * nb.w * fac);
    }
    Xr[lane + 32 * q] = u;
    Vr[lane + 32 * q] = v;
  }
  if (lane == 0) {
    int code = -1;
    if (use) {
      const int m = __ldg(o + t);
      code = (unsigned)m < (unsigned)a.M ? (m | (t == 0 ? (1 << 30) : 0)) : -1;
    }
    a.sym[r] = code;
  }
}

// Cp[k][split] = sum over the split's rows of U[r]^T V[r] (128 x 128 tile
// per block, 8 x 8 outputs per thread, rows staged 8 at a time).
template <int NP>
__global__ void __launch_bounds__(256) fbw_gemm_kernel(FbWideArgs a) {
  constexpr int TL = kFbwGemmTile, BK = kFbwGemmRows, NT = NP / TL;
  __shared__ __align__(16) float Us[BK][TL];
  __shared__ __align__(16) float Vs[BK][TL];
  const int ti = blockIdx.x / NT, tj = blockIdx.x % NT;
  const int split = blockIdx.y, k = blockIdx.z;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t r0 = (int64_t)split * a.rows_per_split;
  const int64_t r1 = min(a.rtot, r0 + a.rows_per_split);
  const float* Uk = a.X + (size_t)k * a.rtot * NP + ti * TL;
  const float* Vk = a.V + (size_t)k * a.rtot * NP + tj * TL;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int lr = tid / 32, lc = 4 * (tid % 32);  // staging: row lr, columns lc .. lc + 3
  for (int64_t rb = r0; rb < r1; rb += BK) {
    const int64_t rr = rb + lr;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 uv = rr < r1 ? __ldg(reinterpret_cast<const float4*>(Uk + rr * NP + lc)) : z4;
    const float4 vv = rr < r1 ? __ldg(reinterpret_cast<const float4*>(Vk + rr * NP + lc)) : z4;
    __syncthreads();
    *reinterpret_cast<float4*>(&Us[lr][lc]) = uv;
    *reinterpret_cast<float4*>(&Vs[lr][lc]) = vv;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Us[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Us[kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Vs[kk][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Vs[kk][tx * 8 + 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }
  float* C = a.Cp + ((size_t)k * a.nsplit + split) * NP * NP;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float* dst = C + (size_t)(ti * TL + ty * 8 + i) * NP + tj * TL + tx * 8;
    *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    *reinterpret_cast<float4*>(dst + 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
  }
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
    const int kmod = a.labelled ? 0 : k;
    a.cnt_A[idx] = sum * __ldg(a.A + ((size_t)kmod * a.N + i) * a.N + j);
  }
}

// Per chunk of rows: Ep[k][chunk][j][m] = sum of G[r][j] over the chunk's rows
// with symbol m, Pp[k][chunk][j] the same over rows at t = 0. Thread j owns
// state j's accumulators (shared memory, row stride M + 1).
__global__ void fbw_emis_kernel(FbWideArgs a) {
  extern __shared__ float acc[];  // [NP][M + 1]
  const int chunk = blockIdx.x, k = blockIdx.y, j = threadIdx.x;
  const int ld = a.M + 1;
  for (int m = 0; m < a.M; ++m) acc[j * ld + m] = 0.f;
  float pacc = 0.f;
  const int64_t r0 = (int64_t)chunk * a.rows_per_chunk;
  const int64_t r1 = min(a.rtot, r0 + a.rows_per_chunk);
  const int32_t* sym = a.sym + (size_t)k * a.rtot;
  const float* G = a.G + (size_t)k * a.rtot * a.NP + j;
  for (int64_t r = r0; r < r1; ++r) {
    const int code = __ldg(sym + r);
    if (code < 0) continue;
    const float g = __ldg(G + r * a.NP);
    acc[j * ld + (code & 0xffffff)] += g;
    if (code >> 30) pacc += g;
  }
  float* E = a.Ep + (((size_t)k * a.nchunks + chunk) * a.NP + j) * a.M;
  for (int m = 0; m < a.M; ++m) E[m] = acc[j * ld + m];
  a.Pp[((size_t)k * a.nchunks + chunk) * a.NP + j] = pacc;
}

__global__ void fbw_reduce_b_kernel(FbWideArgs a) {
  const int64_t nB = (int64_t)a.K * a.N * a.M, nP = (int64_t)a.K * a.N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nB + nP;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nB) {
      const int k = (int)(idx / ((int64_t)a.N * a.M));
      const int j = (int)((idx / a.M) % a.N), m = (int)(idx % a.M);
      const float* e = a.Ep + ((size_t)k * a.nchunks * a.NP + j) * a.M + m;
      float sum = 0.f;
      for (int c = 0; c < a.nchunks; ++c) sum += e[(size_t)c * a.NP * a.M];
      a.cnt_B[idx] = sum;
    } else {
      const int64_t q = idx - nB;
      const int k = (int)(q / a.N), j = (int)(q % a.N);
      const float* p = a.Pp + (size_t)k * a.nchunks * a.NP + j;
      float sum = 0.f;
      for (int c = 0; c < a.nchunks; ++c) sum += p[(size_t)c * a.NP];
      a.cnt_pi[q] = sum;
    }
  }
}

size_t fbw_emis_smem(int NP, int M) { return (size_t)NP * (M + 1) * 4; }

cudaError_t launch_fbw_counts(const FbWideArgs& a, cudaStream_t st) {
  const int64_t rows = (int64_t)a.K * a.rtot;
  const int64_t cblocks = (rows * 32 + 255) / 256;
  if (a.NP == 256) fbw_combine_kernel<256><<<(unsigned)cblocks, 256, 0, st>>>(a);
  else if (a.NP == 512) fbw_combine_kernel<512><<<(unsigned)cblocks, 256, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 gg((a.NP / kFbwGemmTile) * (a.NP / kFbwGemmTile), a.nsplit, a.K);
  if (a.NP == 256) fbw_gemm_kernel<256><<<gg, 256, 0, st>>>(a);
  else fbw_gemm_kernel<512><<<gg, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_reduce_a_kernel<<<1024, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = fbw_emis_smem(a.NP, a.M);
  if ((e = cudaFuncSetAttribute(fbw_emis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  fbw_emis_kernel<<<dim3(a.nchunks, a.K), a.NP, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fbw_reduce_b_kernel<<<1024, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hmmgb
