// fb_common.cuh -- register-level building blocks of the FP32 SIMT adjoint
// kernels (fb.cu, fb_seg.cu): exact power-of-two scaling, paired group sums,
// and the backward step over a lane's rows of A (Rabiner 1989 eqs. 24-25, 37).
#pragma once

#include "hmm_internal.cuh"

namespace hmmgb {

// x * 2^k for any k in [-252, 254], as two exact multiplies.
__device__ __forceinline__ float mul_pow2(float x, int k) {
  const int k1 = k / 2, k2 = k - k1;
  return x * exp2i(k1) * exp2i(k2);
}

// Butterfly over the G lanes of a pair for two values at once.
template <int G>
__device__ __forceinline__ float2 group_sum2(float2 v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(HMM_FULL_MASK, v.x, o);
    v.y += __shfl_xor_sync(HMM_FULL_MASK, v.y, o);
  }
  return v;
}

// beta(ii) = sum_j a_{i,j} v_j for the lane's rows i = j0 + ii, and the xi
// accumulator update xa[ii][j] += aw[ii] * v_j, from the broadcast row v.
template <int NP, int J>
__device__ __forceinline__ void rows_step(const float* vb, const float2 (&ar)[J][NP / 2],
                                          const float (&aw)[J], float2 (&xa)[J][NP / 2],
                                          float (&beta)[J]) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  float2 acc[NS][J];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = make_float2(0.f, 0.f);
  float2 aw2[J];
#pragma unroll
  for (int ii = 0; ii < J; ++ii) aw2[ii] = make_float2(aw[ii], aw[ii]);
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 vv = *reinterpret_cast<const float4*>(vb + 4 * q);
    const float2 lo = make_float2(vv.x, vv.y), hi = make_float2(vv.z, vv.w);
    const int s = q % NS;
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = __ffma2_rn(lo, ar[ii][2 * q], acc[s][ii]);
#pragma unroll
    for (int ii = 0; ii < J; ++ii) xa[ii][2 * q] = __ffma2_rn(aw2[ii], lo, xa[ii][2 * q]);
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = __ffma2_rn(hi, ar[ii][2 * q + 1], acc[s][ii]);
#pragma unroll
    for (int ii = 0; ii < J; ++ii) xa[ii][2 * q + 1] = __ffma2_rn(aw2[ii], hi, xa[ii][2 * q + 1]);
  }
#pragma unroll
  for (int ii = 0; ii < J; ++ii) {
    float2 t = acc[0][ii];
#pragma unroll
    for (int s = 1; s < NS; ++s) t = __fadd2_rn(t, acc[s][ii]);
    beta[ii] = t.x + t.y;
  }
}

// beta(ii) = sum_j a_{i,j} v_j for the lane's rows i = j0 + ii (no xi update).
template <int NP, int J>
__device__ __forceinline__ void rows_matvec(const float* vb, const float2 (&ar)[J][NP / 2],
                                            float (&beta)[J]) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  float2 acc[NS][J];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 vv = *reinterpret_cast<const float4*>(vb + 4 * q);
    const float2 lo = make_float2(vv.x, vv.y), hi = make_float2(vv.z, vv.w);
    const int s = q % NS;
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = __ffma2_rn(lo, ar[ii][2 * q], acc[s][ii]);
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = __ffma2_rn(hi, ar[ii][2 * q + 1], acc[s][ii]);
  }
#pragma unroll
  for (int ii = 0; ii < J; ++ii) {
    float2 t = acc[0][ii];
#pragma unroll
    for (int s = 1; s < NS; ++s) t = __fadd2_rn(t, acc[s][ii]);
    beta[ii] = t.x + t.y;
  }
}

}  // namespace hmmgb
