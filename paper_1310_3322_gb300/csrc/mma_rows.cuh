// mma_rows.cuh -- per-row state and epilogue helpers of the scaled forward
// recursion shared by the tensor-core forward kernels (Rabiner 1989 eqs. 19-21 with exact power-of-two
// scaling applied one step late).
#pragma once

#include "hmm_internal.cuh"
#include "tc.cuh"

namespace hmmgb {

// Exponent e with s * 2^-e in [1, 2) for finite s > 0 (subnormals included).
__device__ __forceinline__ int exponent_of(float s) {
  if (s < 0x1p-120f) return frexp2(s * 0x1p64f) - 64;
  return frexp2(s);
}

// Per-row state of the recursion (kept identically by both threads of a row).
struct RowState {
  int F;        // sum of the scale exponents applied so far
  int f;        // exponent applied at the next step, within [-126, 126]
  bool dead, bad, written;
  int err;
  float ll;
};

// Starts the bulk copy of emission row `sym` into this row's slot.
template <int NP>
__device__ __forceinline__ void stage_emission(uint32_t slot, const float* Bk, int sym,
                                               uint64_t* ebar) {
  tc::fence_proxy_async();  // this row's reads of the slot precede the copy
  tc::mbar_arrive_expect_tx(ebar, NP * 4);
  tc::bulk_g2s(slot, Bk + (size_t)sym * NP, NP * 4, ebar);
}

// 32 values -> 16 packed BF16 pairs (even k in the low half).
__device__ __forceinline__ void pack32(const float (&y)[32], uint32_t (&w)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = tc::pack_bf16(y[2 * i], y[2 * i + 1]);
}

// Chunk c (32 values) of this thread's share of the next X row into tensor
// memory: BF16 pairs (16 columns) or TF32 values (32 columns).
template <int AB>
__device__ __forceinline__ void store_x(uint32_t x_mine, int c, const float (&y)[32]) {
  if constexpr (AB == 1) {
    uint32_t w[16];
    pack32(y, w);
    tc::tmem_st16(x_mine + (uint32_t)(16 * c), w);
  } else {
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = tc::to_tf32(y[i]);
    tc::tmem_st16(x_mine + (uint32_t)(32 * c), w);
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = tc::to_tf32(y[16 + i]);
    tc::tmem_st16(x_mine + (uint32_t)(32 * c + 16), w);
  }
}

// After step t's row sum sigma: liveness checks, the log-likelihood at the
// row's last step, and the exponent for the next step.
__device__ __forceinline__ void close_step(RowState& st, float sigma, int t, int Tn) {
  if (t >= Tn || st.dead || st.bad) return;
  if (sigma == 0.f) {
    st.dead = true;
    return;
  }
  if (!(sigma > 0.f) || isinf(sigma)) {
    st.bad = true;
    st.err |= HMM_STATUS_PARAM;
    return;
  }
  if (t == Tn - 1) {
    st.ll = (float)(log((double)sigma) + (double)st.F * 0.69314718055994530942);
    st.written = true;
  }
  st.f = min(126, max(-126, exponent_of(sigma)));
}

}  // namespace hmmgb
