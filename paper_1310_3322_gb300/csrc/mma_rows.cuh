// mma_rows.cuh -- per-row state and epilogue helpers of the scaled forward
// recursion shared by the tensor-core forward kernels (Rabiner 1989 eqs. 19-21 with exact power-of-two
// scaling applied one step late).
#pragma once

#include "hmm_internal.cuh"
#include "tc.cuh"

namespace hmmgb {

// AB: operand type, 1 = BF16 (kind::f16, two values per 32-bit column of
// tensor memory), 2 = TF32 (kind::tf32, one value per column).
// EMIS: the model's emission table lives in shared memory (M padded rows,
// after the fixed part); otherwise NT tiles of per-row staging slots.
template <int NP, int NT, int TPR, int AB = 1, bool EMIS = false>
struct MmaFwdSmem {
  static constexpr int kB = NP * NP * (AB == 1 ? 2 : 4);  // A^T
  static constexpr int kES = NP * 4 + 16;         // padded emission row, FP32
  static constexpr int kE = 128 * kES;            // one tile of emission rows
  // EMIS: padded row of the shared table, BF16 values on the BF16 path (the
  // values the tables hold are BF16 there, so the conversion is exact), FP32
  // on the TF32 path
  static constexpr int kET = (AB == 1 ? NP * 2 : NP * 4) + 16;
  static constexpr int OFF_B = 0;
  static constexpr int OFF_PS = kB;               // partial row sums [NT][TPR][128]
  static constexpr int OFF_BAR = OFF_PS + NT * TPR * 128 * 4;  // mma[NT], emission[NT], fin[NT]
  static constexpr int OFF_MISC = OFF_BAR + 3 * NT * 8;        // tmem, item, abort, last, warp max
  static constexpr int OFF_E = (OFF_MISC + 24 * 4 + 127) / 128 * 128;  // staging or table
  static constexpr int FIXED = OFF_E + (EMIS ? 0 : NT * kE);
  // total bytes for M symbols
  static constexpr int total(int M) { return FIXED + (EMIS ? M * kET : 0); }
};
constexpr int kFwdSmemMax = 227 * 1024;
static_assert(MmaFwdSmem<128, 2, 2, 2>::total(0) <= kFwdSmemMax, "shared memory budget");
static_assert(MmaFwdSmem<64, 4, 1, 2>::total(0) <= kFwdSmemMax, "shared memory budget");

// Byte offset of 8-column group c8 of row m in a 128 x NP BF16 "row image"
// (8-row x 16-byte core matrices: row m, columns 8 c8 .. 8 c8 + 7). The same
// bytes are the K-major operand of a per-row product and the MN-major operand
// of a contraction over rows; the adjoint's checkpoints are stored this way.
template <int NP>
__device__ __forceinline__ uint32_t img_off(int m, int c8) {
  return (uint32_t)((m & 7) * 16 + c8 * 128 + (m >> 3) * NP * 16);
}

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
  float slast;  // the row sum at the row's last step (set with ll)
};

// Copies the model's emission table (M rows of NP FP32 values) into shared
// memory as rows of kET bytes: BF16 (AB 1) or FP32 (AB 2).
template <int NP, int AB, int ET>
__device__ __forceinline__ void fill_emission_table(uint8_t* dst, const float* Bk, int M, int tid,
                                                    int nthreads) {
  if constexpr (AB == 1) {
    const float4* src = reinterpret_cast<const float4*>(Bk);
    for (int idx = tid; idx < M * NP / 8; idx += nthreads) {
      const int m = idx / (NP / 8), c = idx % (NP / 8);
      const float4 lo = __ldg(src + 2 * idx), hi = __ldg(src + 2 * idx + 1);
      *reinterpret_cast<uint4*>(dst + m * ET + c * 16) =
          make_uint4(tc::pack_bf16(lo.x, lo.y), tc::pack_bf16(lo.z, lo.w), tc::pack_bf16(hi.x, hi.y),
                     tc::pack_bf16(hi.z, hi.w));
    }
  } else {
    const float4* src = reinterpret_cast<const float4*>(Bk);
    for (int idx = tid; idx < M * NP / 4; idx += nthreads) {
      const int m = idx / (NP / 4), c = idx % (NP / 4);
      *reinterpret_cast<float4*>(dst + m * ET + c * 16) = __ldg(src + idx);
    }
  }
}

// Eight emission values, columns col .. col + 7 (col a multiple of 8), of one
// row of the shared table.
template <int AB>
__device__ __forceinline__ void emission8(const uint8_t* rowp, int col, float (&b)[8]) {
  if constexpr (AB == 1) {
    const uint4 w = *reinterpret_cast<const uint4*>(rowp + col * 2);
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      b[2 * i] = __uint_as_float(u[i] << 16);
      b[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
    }
  } else {
    const float4 lo = *reinterpret_cast<const float4*>(rowp + col * 4);
    const float4 hi = *reinterpret_cast<const float4*>(rowp + col * 4 + 16);
    b[0] = lo.x; b[1] = lo.y; b[2] = lo.z; b[3] = lo.w;
    b[4] = hi.x; b[5] = hi.y; b[6] = hi.z; b[7] = hi.w;
  }
}

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
    st.slast = sigma;
    st.written = true;
  }
  st.f = min(126, max(-126, exponent_of(sigma)));
}

}  // namespace hmmgb
