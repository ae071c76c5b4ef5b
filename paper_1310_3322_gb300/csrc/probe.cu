// probe.cu -- FP32 FMA throughput probe: the measured denominator of the
// roofline of the SIMT kernels (forward, Viterbi, adjoint at N <= 64), which
// are bound by FP32 issue, not by memory.
//
// Every thread runs `iters` rounds of 16 independent FMA chains
// x <- x * m + c (m slightly below 1, so the values settle near c / (1 - m)
// and never leave the normal range); 16 chains per thread and several
// resident warps per scheduler hide the FMA latency, so the launch measures
// the pipe's throughput. Mode 0 issues scalar fma.rn.f32, mode 1 the packed
// fma.rn.f32x2 of the sm_100 family (two FMAs per instruction, as the
// kernels' inner loops use). The chains' sums are reduced per block and
// written out so the work cannot be optimised away.
#include "hmm_internal.cuh"

namespace hmmgb {

template <int MODE>
__global__ void __launch_bounds__(1024) fma_probe_kernel(int64_t iters, float* out) {
  __shared__ float red[32];
  const float seed = 1e-3f * (float)(threadIdx.x & 63);
  float r = 0.f;
  if constexpr (MODE == 0) {
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = seed + (float)i;
    const float m = 0.999f, c = 1e-3f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = __fmaf_rn(x[i], m, c);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) r += x[i];
  } else {
    float2 x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = make_float2(seed + (float)i, seed - (float)i);
    const float2 m = make_float2(0.999f, 0.998f), c = make_float2(1e-3f, 2e-3f);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = __ffma2_rn(x[i], m, c);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) r += x[i].x + x[i].y;
  }
  r = group_sum<32>(r);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[blockIdx.x] = s;
  }
}

}  // namespace hmmgb

extern "C" int hmm_fma_probe(int32_t blocks, int32_t threads, int64_t iters, int32_t mode,
                             float* out, hmm_stream_t stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !out ||
      (mode != 0 && mode != 1))
    return HMM_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (mode == 0) hmmgb::fma_probe_kernel<0><<<blocks, threads, 0, st>>>(iters, out);
  else hmmgb::fma_probe_kernel<1><<<blocks, threads, 0, st>>>(iters, out);
  return cudaGetLastError() == cudaSuccess ? HMM_OK : HMM_ERR_CUDA;
}
