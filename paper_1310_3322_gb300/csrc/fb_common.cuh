// fb_common.cuh -- register-level building blocks of the FP32 SIMT adjoint
// kernels (fb.cu, fb_seg.cu): exact power-of-two scaling from a row's sum,
// the forward product over a lane's columns of A and the backward step over
// its rows (Rabiner 1989 eqs. 19-21, 24-25, 37), each returning the sum of the
// broadcast row it reads.
#pragma once

#include "hmm_internal.cuh"

namespace hmmgb {

// The power of two that a step applies to its result, from the sum s of its
// input row: 2^-f with f the exponent of s (s 2^-f in [1, 2)) for normal s
// below 2^127. Two integer operations on the bit pattern, no branch: a zero
// or subnormal s gets f = -127 (2^127 keeps any such sum below 2), s at or
// above 2^127 gets f = 126; negative, infinite and NaN sums are flagged by
// the callers, which discard what the factor is applied to.
__device__ __forceinline__ float pow2_scale(float s, int& f) {
  const int eb = min(__float_as_int(s) & 0x7f800000, 253 << 23);
  f = (eb >> 23) - 127;
  return __int_as_float((254 << 23) - eb);
}

// Classifies a row sum for the liveness checks: 1 zero (the sequence is
// impossible under the model), 2 invalid (negative, infinite or NaN), else 0.
__device__ __forceinline__ int sum_class(float s) {
  const unsigned b = __float_as_uint(s);
  if ((b & 0x7fffffffu) == 0u) return 1;
  return (b > 0x80000000u || (b & 0x7fffffffu) >= 0x7f800000u) ? 2 : 0;
}

// Sum of a register array of float2 pairs (balanced tree of packed adds).
template <int H>
__device__ __forceinline__ float2 tree_sum2(const float2 (&x)[H]) {
  if constexpr (H == 1) {
    return x[0];
  } else {
    float2 t[H / 2];
#pragma unroll
    for (int i = 0; i < H / 2; ++i) t[i] = __fadd2_rn(x[2 * i], x[2 * i + 1]);
    return tree_sum2<H / 2>(t);
  }
}

// out[jj] = sum_i x_i a_{i, j0+jj} (hmm_internal.cuh's matvec_cols) and the
// sum of the broadcast row x, from the same shared-memory loads: every lane of
// a pair reads the whole row and adds it in the same order, so all of them get
// the same sum without a cross-lane reduction.
template <int NP, int J>
__device__ __forceinline__ void matvec_cols_sum(const float* xb, const float2 (&a2)[NP / 2][J],
                                                float (&out)[J], float& sum) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  constexpr int NQ = NP / 4 < 4 ? NP / 4 : 4;  // partial sums of the row
  float2 acc[NS][J];
  float2 xs[NQ];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[s][jj] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 xv = *reinterpret_cast<const float4*>(xb + 4 * q);
    const float2 lo = make_float2(xv.x, xv.y), hi = make_float2(xv.z, xv.w);
    const float2 lh = __fadd2_rn(lo, hi);
    xs[q % NQ] = q < NQ ? lh : __fadd2_rn(xs[q % NQ], lh);
    const int s = q % NS;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[s][jj] = __ffma2_rn(lo, a2[2 * q][jj], acc[s][jj]);
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[s][jj] = __ffma2_rn(hi, a2[2 * q + 1][jj], acc[s][jj]);
  }
#pragma unroll
  for (int jj = 0; jj < J; ++jj) {
    float2 t = acc[0][jj];
#pragma unroll
    for (int s = 1; s < NS; ++s) t = __fadd2_rn(t, acc[s][jj]);
    out[jj] = t.x + t.y;
  }
  const float2 t = tree_sum2<NQ>(xs);
  sum = t.x + t.y;
}

// beta(ii) = sum_j a_{i,j} v_j for the lane's rows i = j0 + ii and the xi
// accumulator update xa[ii][j] += aw[ii] v_j, from the broadcast row v; also
// returns the sum of v (same order in every lane).
template <int NP, int J>
__device__ __forceinline__ void rows_step_sum(const float* vb, const float2 (&ar)[J][NP / 2],
                                              const float (&aw)[J], float2 (&xa)[J][NP / 2],
                                              float (&beta)[J], float& sum) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  constexpr int NQ = NP / 4 < 4 ? NP / 4 : 4;  // partial sums of the row
  float2 acc[NS][J];
  float2 vs[NQ];
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
    const float2 lh = __fadd2_rn(lo, hi);
    vs[q % NQ] = q < NQ ? lh : __fadd2_rn(vs[q % NQ], lh);
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
  const float2 t = tree_sum2<NQ>(vs);
  sum = t.x + t.y;
}

// beta(ii) = sum_j a_{i,j} v_j for the lane's rows (no xi update), and the
// sum of the broadcast row v (same order in every lane).
template <int NP, int J>
__device__ __forceinline__ void rows_matvec_sum(const float* vb, const float2 (&ar)[J][NP / 2],
                                                float (&beta)[J], float& sum) {
  constexpr int NS = (J >= 4) ? 1 : (4 / J < NP / 4 ? 4 / J : NP / 4);
  constexpr int NQ = NP / 4 < 4 ? NP / 4 : 4;
  float2 acc[NS][J];
  float2 vs[NQ];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int ii = 0; ii < J; ++ii) acc[s][ii] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NP / 4; ++q) {
    const float4 vv = *reinterpret_cast<const float4*>(vb + 4 * q);
    const float2 lo = make_float2(vv.x, vv.y), hi = make_float2(vv.z, vv.w);
    const float2 lh = __fadd2_rn(lo, hi);
    vs[q % NQ] = q < NQ ? lh : __fadd2_rn(vs[q % NQ], lh);
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
  const float2 t = tree_sum2<NQ>(vs);
  sum = t.x + t.y;
}

}  // namespace hmmgb
