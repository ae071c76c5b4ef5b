// setup.cu -- per-call preparation and the small elementwise kernels.
//
//  * setup_kernel: one launch per hmm_* call. Block 0 validates every
//    sequence, sorts the sequences by decreasing length (bucketed counting
//    sort; the persistent kernels then take work longest-first) and, for
//    Viterbi, assigns backpointer storage. The other blocks copy pi, A and
//    B^T into the padded tables the recursions read (probabilities, or
//    natural logs for Viterbi) and flag negative or non-finite parameters.
//  * softmax_rows / softmax_grad: the row-softmax parameterisation used for
//    learning and its chain rule, one warp per row.
//  * adam: one fused Adam update.
//  * reduce1 / reduce2: the fixed-order two-level sum of the adjoint's
//    per-pair count partials (bitwise reproducible).
#include <cuda_bf16.h>

#include "hmm_internal.cuh"

namespace hmmgb {

// Exclusive scan over a 1024-thread block; `tmp` holds 32 entries.
template <typename T>
__device__ T block_exclusive_scan(T v, T* tmp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(HMM_FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = tmp[lane];
    T wx = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(HMM_FULL_MASK, wx, o);
      if (lane >= o) wx += y;
    }
    tmp[lane] = wx - w;  // exclusive prefix of warp totals
    if (lane == 31 && total) *total = wx;
  }
  __syncthreads();
  const T r = x - v + tmp[warp];
  __syncthreads();
  return r;
}

// Prefix units of a validated length: backpointer rows (kind 0, Viterbi) or
// chunks of the parallel-in-time forward (kind 1: steps 1 .. T-1 in chunks of
// scan_chunk).
__device__ __forceinline__ long long prefix_units(const SetupArgs& a, int T, int kind) {
  if (T <= 0) return 0;
  if (kind == 0) return T;
  return (T - 1 + (long long)a.scan_chunk - 1) / a.scan_chunk;
}

// The plan for S <= kPlanRegs * kPlanThreads with every sequence's length
// held in registers: thread t validates sequences t + i * kPlanThreads (all
// of its loads in flight together) and sorts them by length bucket; the
// prefix sums in sequence order (backpointer rows, scan chunks) take
// contiguous runs of kPlanRegs per thread and one block scan.
constexpr int kPlanRegs = 16;

__device__ void plan_block_cached(const SetupArgs& a) {
  __shared__ int hist[kLenBuckets];
  __shared__ int itmp[32];
  __shared__ long long ltmp[32];
  __shared__ long long total;
  const int tid = threadIdx.x;
  hist[tid] = 0;  // kLenBuckets == kPlanThreads
  for (int i = tid; i < a.ndone; i += kPlanThreads) a.done[i] = 0;
  // every load first, none behind a test, so all of them are in flight
  // together (a load under a data-dependent branch waits for the branch)
  int Ts[kPlanRegs];
  int bad = 0;
#pragma unroll
  for (int i = 0; i < kPlanRegs; ++i) {
    const int s = tid + i * kPlanThreads;
    const bool in = s < a.S;
    const int T = in ? __ldg(a.lengths + s) : 0;
    const long long off = in ? __ldg(a.offsets + s) : 0;
    const int mk = (in && a.model_of_seq) ? __ldg(a.model_of_seq + s) : 0;
    const int mb = (in && a.model_base) ? __ldg(a.model_base + s) : 0;
    bool ok = T >= 0 && T <= a.max_len && off >= 0 && off <= a.total_obs - (long long)T;
    if (a.model_of_seq) ok = ok && mk >= 0 && mk < a.K;
    if (a.model_base) ok = ok && mb >= 0 && mb <= a.K - a.span;
    Ts[i] = in ? (ok ? T : -1) : 0;
    if (in && !ok) bad = 1;
  }
#pragma unroll
  for (int i = 0; i < kPlanRegs; ++i) {
    const int s = tid + i * kPlanThreads;
    if (s < a.S) a.seqlen[s] = Ts[i];
  }
  __syncthreads();  // hist cleared; seqlen visible to the whole block
#pragma unroll
  for (int i = 0; i < kPlanRegs; ++i) {
    const int s = tid + i * kPlanThreads;
    if (s < a.S && !a.skip_order)
      atomicAdd(&hist[kLenBuckets - 1 - length_bucket(max(Ts[i], 0))], 1);
  }
  if (bad) set_status(a.status, HMM_STATUS_SEQ);
  if (!a.skip_order) {
    __syncthreads();
    const int start = block_exclusive_scan<int>(hist[tid], itmp, nullptr);
    hist[tid] = start;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPlanRegs; ++i) {
      const int s = tid + i * kPlanThreads;
      if (s < a.S) {
        const int pos = atomicAdd(&hist[kLenBuckets - 1 - length_bucket(max(Ts[i], 0))], 1);
        a.order[pos] = s;
      }
    }
  }
  // prefix sums in sequence order: thread t owns the contiguous run
  // [t R, t R + R) of the validated lengths (read back from seqlen), so one
  // block scan of the per-thread totals serves all of them
  for (int kind = 0; kind < 2; ++kind) {
    if (kind == 0 ? !a.want_bpoff : a.scan_chunk <= 0) continue;
    int64_t* out = kind == 0 ? a.bpoff : a.coff;
    const long long cap = kind == 0 ? a.bp_cap_rows : a.coff_cap;
    const int b0 = tid * kPlanRegs;
    long long u[kPlanRegs];
    long long local = 0;
#pragma unroll
    for (int i = 0; i < kPlanRegs; ++i) {
      const int s = b0 + i;
      u[i] = s < a.S ? prefix_units(a, a.seqlen[s], kind) : 0;
      local += u[i];
    }
    long long run = block_exclusive_scan<long long>(local, ltmp, &total);
    bool over = false;
#pragma unroll
    for (int i = 0; i < kPlanRegs; ++i) {
      const int s = b0 + i;
      if (s < a.S) {
        out[s] = run;
        if (u[i] > 0 && run + u[i] > cap) {  // storage exhausted
          a.seqlen[s] = -1;
          over = true;
        }
        run += u[i];
      }
    }
    if (over) set_status(a.status, HMM_STATUS_SEQ);
    if (kind == 1 && tid == 0) a.coff[a.S] = total < cap ? total : cap;
    __syncthreads();  // seqlen rewrites and `total` settle before the next kind
  }
}

__device__ void plan_block(const SetupArgs& a) {
  __shared__ int hist[kLenBuckets];
  __shared__ int itmp[32];
  __shared__ long long ltmp[32];
  const int tid = threadIdx.x;
  for (int b = tid; b < kLenBuckets; b += kPlanThreads) hist[b] = 0;
  for (int i = tid; i < a.ndone; i += kPlanThreads) a.done[i] = 0;
  __syncthreads();

#pragma unroll 4
  for (int s = tid; s < a.S; s += kPlanThreads) {
    // loads first, none behind a test (see plan_block_cached)
    const int T = __ldg(a.lengths + s);
    const long long off = __ldg(a.offsets + s);
    const int mk = a.model_of_seq ? __ldg(a.model_of_seq + s) : 0;
    const int mb = a.model_base ? __ldg(a.model_base + s) : 0;
    bool ok = T >= 0 && T <= a.max_len && off >= 0 && off <= a.total_obs - (long long)T;
    if (a.model_of_seq) ok = ok && mk >= 0 && mk < a.K;
    if (a.model_base) ok = ok && mb >= 0 && mb <= a.K - a.span;
    if (!ok) set_status(a.status, HMM_STATUS_SEQ);
    a.seqlen[s] = ok ? T : -1;
    if (!a.skip_order) atomicAdd(&hist[kLenBuckets - 1 - length_bucket(ok ? T : 0)], 1);
  }
  if (a.skip_order) return;
  __syncthreads();

  // one bucket per thread (kLenBuckets == kPlanThreads)
  const int start = block_exclusive_scan<int>(hist[tid], itmp, nullptr);
  hist[tid] = start;
  __syncthreads();

  for (int s = tid; s < a.S; s += kPlanThreads) {
    const int T = a.seqlen[s];
    const int key = kLenBuckets - 1 - length_bucket(T < 0 ? 0 : T);
    const int pos = atomicAdd(&hist[key], 1);
    a.order[pos] = s;
  }

  __shared__ long long total;
  for (int kind = 0; kind < 2; ++kind) {
    if (kind == 0 ? !a.want_bpoff : a.scan_chunk <= 0) continue;
    int64_t* out = kind == 0 ? a.bpoff : a.coff;
    const long long cap = kind == 0 ? a.bp_cap_rows : a.coff_cap;
    __syncthreads();
    const int chunk = (a.S + kPlanThreads - 1) / kPlanThreads;
    const int b0 = min(a.S, tid * chunk), b1 = min(a.S, b0 + chunk);
    long long local = 0;
    for (int s = b0; s < b1; ++s) local += prefix_units(a, a.seqlen[s], kind);
    long long run = block_exclusive_scan<long long>(local, ltmp, &total);
    for (int s = b0; s < b1; ++s) {
      const long long v = prefix_units(a, a.seqlen[s], kind);
      out[s] = run;
      if (v > 0) {
        if (run + v > cap) {  // storage exhausted
          a.seqlen[s] = -1;
          set_status(a.status, HMM_STATUS_SEQ);
        }
        run += v;
      }
    }
    if (kind == 1 && tid == 0) a.coff[a.S] = total < cap ? total : cap;
  }
}

__device__ __forceinline__ float prep_value(float v, int log_mode, int32_t* status) {
  if (!(v >= 0.f) || isinf(v)) {
    set_status(status, HMM_STATUS_PARAM);
    return __int_as_float(0x7fc00000);
  }
  return log_mode ? logf(v) : v;
}

__device__ void prep_blocks(const SetupArgs& a, int blk, int nblk) {
  const long long n_pi = (long long)a.K * a.NP;
  const long long n_A = n_pi * a.NP;
  const long long n_B = (long long)a.K * a.M * a.NP;
  const float pad = a.log_mode ? -INFINITY : 0.f;
  const long long stride = (long long)nblk * blockDim.x;
  for (long long idx = (long long)blk * blockDim.x + threadIdx.x; idx < n_pi + n_A + n_B;
       idx += stride) {
    if (idx < n_pi) {
      const int k = (int)(idx / a.NP), j = (int)(idx % a.NP);
      a.pip[idx] = j < a.N ? prep_value(a.pi[(size_t)k * a.N + j], a.log_mode, a.status) : pad;
    } else if (idx < n_pi + n_A) {
      const long long r = idx - n_pi;
      const int k = (int)(r / ((long long)a.NP * a.NP));
      const int i = (int)((r / a.NP) % a.NP), j = (int)(r % a.NP);
      a.Ap[r] = (i < a.N && j < a.N)
                    ? prep_value(a.A[((size_t)k * a.N + i) * a.N + j], a.log_mode, a.status)
                    : pad;
    } else {
      const long long r = idx - n_pi - n_A;
      const int k = (int)(r / ((long long)a.M * a.NP));
      const int m = (int)((r / a.NP) % a.M), j = (int)(r % a.NP);
      float v = j < a.N ? prep_value(a.B[((size_t)k * a.N + j) * a.M + m], a.log_mode, a.status)
                        : pad;
      if (a.bf16_b) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        v = __bfloat162float(h);
        a.Btp16[r] = *reinterpret_cast<const uint16_t*>(&h);
      }
      a.Btp[r] = v;
    }
  }
}

__global__ void __launch_bounds__(kPlanThreads) setup_kernel(SetupArgs a) {
  if (blockIdx.x == 0) {
    if (a.S <= kPlanRegs * kPlanThreads)
      plan_block_cached(a);
    else
      plan_block(a);
  }
  else
    prep_blocks(a, blockIdx.x - 1, gridDim.x - 1);
}

// ---------------------------------------------------------------------------
// the same plan over many blocks (S > kPlanSingleMax): one block per
// kPlanBlockSeqs consecutive sequences validates them and counts their
// length buckets and prefix units (kernel A, beside the table blocks); one
// block turns the per-block counts into per-block starting offsets (kernel B);
// every plan block then places its sequences and writes its prefix sums
// (kernel C). Same outputs as the single block (within a length bucket the
// order of sequences is the atomics' order in both).
// ---------------------------------------------------------------------------
constexpr int kPlanPer = 4;                                   // sequences per thread
constexpr int kPlanBlockSeqs = kPlanPer * kPlanThreads;      // 4096 per block
constexpr int kPlanSingleMax = 4096;

int plan_blocks(int S) { return (S + kPlanBlockSeqs - 1) / kPlanBlockSeqs; }

__global__ void __launch_bounds__(kPlanThreads) plan_mb_a_kernel(SetupArgs a, int nb) {
  if ((int)blockIdx.x >= nb) {
    prep_blocks(a, blockIdx.x - nb, gridDim.x - nb);
    return;
  }
  __shared__ int hist[kLenBuckets];
  __shared__ long long red[2][32];
  const int tid = threadIdx.x, b = blockIdx.x;
  hist[tid] = 0;
  for (int i = b * kPlanThreads + tid; i < a.ndone; i += nb * kPlanThreads) a.done[i] = 0;
  int Ts[kPlanPer];
  int bad = 0;
#pragma unroll
  for (int i = 0; i < kPlanPer; ++i) {  // loads first, none behind a test
    const int s = b * kPlanBlockSeqs + tid + i * kPlanThreads;
    const bool in = s < a.S;
    const int T = in ? __ldg(a.lengths + s) : 0;
    const long long off = in ? __ldg(a.offsets + s) : 0;
    const int mk = (in && a.model_of_seq) ? __ldg(a.model_of_seq + s) : 0;
    const int mb = (in && a.model_base) ? __ldg(a.model_base + s) : 0;
    bool ok = T >= 0 && T <= a.max_len && off >= 0 && off <= a.total_obs - (long long)T;
    if (a.model_of_seq) ok = ok && mk >= 0 && mk < a.K;
    if (a.model_base) ok = ok && mb >= 0 && mb <= a.K - a.span;
    Ts[i] = in ? (ok ? T : -1) : 0;
    if (in && !ok) bad = 1;
  }
  long long u0 = 0, u1 = 0;
#pragma unroll
  for (int i = 0; i < kPlanPer; ++i) {
    const int s = b * kPlanBlockSeqs + tid + i * kPlanThreads;
    if (s < a.S) {
      a.seqlen[s] = Ts[i];
      if (a.want_bpoff) u0 += prefix_units(a, Ts[i], 0);
      if (a.scan_chunk > 0) u1 += prefix_units(a, Ts[i], 1);
    }
  }
  if (bad) set_status(a.status, HMM_STATUS_SEQ);
  __syncthreads();  // hist cleared
  if (!a.skip_order) {
#pragma unroll
    for (int i = 0; i < kPlanPer; ++i) {
      const int s = b * kPlanBlockSeqs + tid + i * kPlanThreads;
      if (s < a.S) atomicAdd(&hist[kLenBuckets - 1 - length_bucket(max(Ts[i], 0))], 1);
    }
  }
  // block sums of the prefix units
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u0 += __shfl_xor_sync(HMM_FULL_MASK, u0, o);
    u1 += __shfl_xor_sync(HMM_FULL_MASK, u1, o);
  }
  if ((tid & 31) == 0) { red[0][tid >> 5] = u0; red[1][tid >> 5] = u1; }
  __syncthreads();
  if (tid < 2) {
    long long t = 0;
    for (int w = 0; w < kPlanThreads / 32; ++w) t += red[tid][w];
    a.punits[(size_t)tid * nb + b] = t;
  }
  if (!a.skip_order) a.phist[(size_t)b * kLenBuckets + tid] = hist[tid];
}

__global__ void __launch_bounds__(kPlanThreads) plan_mb_b_kernel(SetupArgs a, int nb) {
  __shared__ int itmp[32];
  const int tid = threadIdx.x;
  if (!a.skip_order) {  // thread = bucket: per-block starting offsets, in place
    int tot = 0;
    for (int b = 0; b < nb; ++b) tot += a.phist[(size_t)b * kLenBuckets + tid];
    int base = block_exclusive_scan<int>(tot, itmp, nullptr);
    for (int b = 0; b < nb; ++b) {
      int* h = a.phist + (size_t)b * kLenBuckets + tid;
      const int v = *h;
      *h = base;
      base += v;
    }
  }
  if (tid < 2) {  // per-block offsets of the prefix units (blocks in sequence order)
    const int kind = tid;
    if (kind == 0 ? !a.want_bpoff : a.scan_chunk <= 0) return;
    long long run = 0;
    for (int b = 0; b < nb; ++b) {
      int64_t* u = a.punits + (size_t)kind * nb + b;
      const long long v = *u;
      *u = run;
      run += v;
    }
    if (kind == 1) a.coff[a.S] = run < a.coff_cap ? run : a.coff_cap;
  }
}

__global__ void __launch_bounds__(kPlanThreads) plan_mb_c_kernel(SetupArgs a, int nb) {
  __shared__ int hist[kLenBuckets];
  __shared__ long long ltmp[32];
  const int tid = threadIdx.x, b = blockIdx.x;
  if (!a.skip_order) {
    hist[tid] = a.phist[(size_t)b * kLenBuckets + tid];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPlanPer; ++i) {
      const int s = b * kPlanBlockSeqs + tid + i * kPlanThreads;
      if (s < a.S) {
        const int T = a.seqlen[s];
        const int pos = atomicAdd(&hist[kLenBuckets - 1 - length_bucket(max(T, 0))], 1);
        a.order[pos] = s;
      }
    }
  }
  for (int kind = 0; kind < 2; ++kind) {
    if (kind == 0 ? !a.want_bpoff : a.scan_chunk <= 0) continue;
    int64_t* out = kind == 0 ? a.bpoff : a.coff;
    const long long cap = kind == 0 ? a.bp_cap_rows : a.coff_cap;
    const int s0 = b * kPlanBlockSeqs + tid * kPlanPer;  // a contiguous run per thread
    long long u[kPlanPer];
    long long local = 0;
#pragma unroll
    for (int i = 0; i < kPlanPer; ++i) {
      u[i] = s0 + i < a.S ? prefix_units(a, a.seqlen[s0 + i], kind) : 0;
      local += u[i];
    }
    long long run = a.punits[(size_t)kind * nb + b] +
                    block_exclusive_scan<long long>(local, ltmp, nullptr);
    bool over = false;
#pragma unroll
    for (int i = 0; i < kPlanPer; ++i) {
      const int s = s0 + i;
      if (s < a.S) {
        out[s] = run;
        if (u[i] > 0 && run + u[i] > cap) {  // storage exhausted
          a.seqlen[s] = -1;
          over = true;
        }
        run += u[i];
      }
    }
    if (over) set_status(a.status, HMM_STATUS_SEQ);
    __syncthreads();  // seqlen rewrites settle before the next kind reads them
  }
}

cudaError_t launch_setup(const SetupArgs& a, cudaStream_t st) {
  const long long work = (long long)a.K * a.NP * (1 + a.NP + a.M);
  int nprep = (int)((work + kPlanThreads * 4 - 1) / (kPlanThreads * 4));
  nprep = max(1, min(nprep, 2 * num_sms()));
  if (a.S <= kPlanSingleMax || !a.phist || !a.punits) {
    setup_kernel<<<1 + nprep, kPlanThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
  const int nb = plan_blocks(a.S);
  plan_mb_a_kernel<<<nb + nprep, kPlanThreads, 0, st>>>(a, nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.skip_order && !a.want_bpoff && a.scan_chunk <= 0) return cudaSuccess;
  plan_mb_b_kernel<<<1, kPlanThreads, 0, st>>>(a, nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  plan_mb_c_kernel<<<nb, kPlanThreads, 0, st>>>(a, nb);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// plan of the tensor-core adjoint (one 1024-thread block)
// ---------------------------------------------------------------------------
// One stable counting-sort pass over (key, item) pairs: the outputs receive
// the inputs ordered by the digit (key >> shift) & 255, pairs with equal
// digits keeping their input order. A chunk is 4096 pairs, 128 consecutive
// ones per warp. Within a warp, equal digits are found with eight ballots
// (one per digit bit) and ranked in index order; per-(digit, warp) counts in
// `wh` ([256][32], digit-major, zero on entry and on return) become offsets
// by a scan over the warps of each digit (four threads per digit). Each chunk
// is first placed in digit order in shared memory and then written out in
// runs, so the global stores are coalesced; the next chunk's pairs are loaded
// while the current one is ranked.
constexpr int kSortIpt = 4;                          // pairs per thread and chunk
constexpr int kSortChunk = kSortIpt * kPlanThreads;  // 4096

struct SortSmem {
  int base[256];    // output start of each digit (running over chunks)
  int lstart[256];  // start of each digit within the chunk
  int tot[256];     // the chunk's count per digit
  int wh[256 * 32];
  int st_item[kSortChunk];
  uint32_t st_key[kSortChunk];
};

__device__ __forceinline__ unsigned digit_peers(int d, bool valid) {
  unsigned peers = __ballot_sync(HMM_FULL_MASK, valid);
  if (!valid) peers = ~peers;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1;
    const unsigned bal = __ballot_sync(HMM_FULL_MASK, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// wh[d][w] (counts) -> sum over warps w' < w of wh[d][w'], tot[d] = the
// digit's total. Thread t owns digit t / 4, warps 8(t % 4)..+7.
__device__ __forceinline__ void scan_warp_counts(SortSmem& m) {
  const int tid = threadIdx.x, d = tid >> 2, q = tid & 3;
  int4* p = reinterpret_cast<int4*>(m.wh + d * 32 + q * 8);
  const int4 a = p[0], b = p[1];
  const int s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
  int x = s;  // inclusive scan over the digit's four threads (consecutive lanes)
  int y = __shfl_up_sync(HMM_FULL_MASK, x, 1);
  if (q >= 1) x += y;
  y = __shfl_up_sync(HMM_FULL_MASK, x, 2);
  if (q >= 2) x += y;
  int run = x - s;
  int4 oa, ob;
  oa.x = run; run += a.x; oa.y = run; run += a.y; oa.z = run; run += a.z; oa.w = run; run += a.w;
  ob.x = run; run += b.x; ob.y = run; run += b.y; ob.z = run; run += b.z; ob.w = run; run += b.w;
  p[0] = oa;
  p[1] = ob;
  if (q == 3) m.tot[d] = x;
}

// dst[d] = exclusive prefix of src[0..256) (one warp).
__device__ __forceinline__ void warp_scan256(const int* src, int* dst) {
  const int lane = threadIdx.x & 31;
  int v[8], sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) { v[q] = src[lane * 8 + q]; sum += v[q]; }
  int x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(HMM_FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  int run = x - sum;
#pragma unroll
  for (int q = 0; q < 8; ++q) { dst[lane * 8 + q] = run; run += v[q]; }
}

__device__ __forceinline__ void zero_wh(SortSmem& m) {
  int4* p = reinterpret_cast<int4*>(m.wh + (threadIdx.x >> 2) * 32 + (threadIdx.x & 3) * 8);
  p[0] = make_int4(0, 0, 0, 0);
  p[1] = make_int4(0, 0, 0, 0);
}

// Ranks the chunk of 4096 pairs starting at c0 (digit = (key >> shift) & 255)
// and writes it out stably: digit d's pairs go to m.base[d] onwards, in input
// order. m.wh must be zero on entry; it is zero again on return.
__device__ void scatter_chunk(const int32_t* in_i, const uint32_t* in_k, int32_t* out_i,
                              uint32_t* out_k, int n, int c0, int shift, SortSmem& m) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int cn = min(kSortChunk, n - c0);
  uint32_t key[kSortIpt];
  int item[kSortIpt], dv[kSortIpt], off[kSortIpt];
#pragma unroll
  for (int u = 0; u < kSortIpt; ++u) {
    const int i = c0 + warp * (32 * kSortIpt) + u * 32 + lane;
    key[u] = i < n ? __ldcg(in_k + i) : 0u;
    item[u] = i < n ? __ldcg(in_i + i) : 0;
    dv[u] = i < n ? (int)((key[u] >> shift) & 255u) : 256;
  }
  // ranks within the warp, in index order (slot by slot)
#pragma unroll
  for (int u = 0; u < kSortIpt; ++u) {
    const bool valid = dv[u] < 256;
    const unsigned peers = digit_peers(dv[u] & 255, valid);
    const int cur = valid ? m.wh[dv[u] * 32 + warp] : 0;
    off[u] = cur + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) m.wh[dv[u] * 32 + warp] = cur + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  scan_warp_counts(m);
  __syncthreads();
  if (warp == 0) warp_scan256(m.tot, m.lstart);
  __syncthreads();
  // the chunk in digit order in shared memory
#pragma unroll
  for (int u = 0; u < kSortIpt; ++u)
    if (dv[u] < 256) {
      const int lp = m.lstart[dv[u]] + m.wh[dv[u] * 32 + warp] + off[u];
      m.st_item[lp] = item[u];
      m.st_key[lp] = key[u];
    }
  __syncthreads();
  // ... and out in runs: local position j of digit d goes to base[d] + j - lstart[d]
  for (int j = tid; j < cn; j += kPlanThreads) {
    const uint32_t k = m.st_key[j];
    const int d = (int)((k >> shift) & 255u);
    const int pos = m.base[d] + j - m.lstart[d];
    out_i[pos] = m.st_item[j];
    out_k[pos] = k;
  }
  __syncthreads();
  zero_wh(m);
  __syncthreads();
}

// The digit counts of the chunk at c0 into m.tot (m.wh zero on entry and return).
__device__ void chunk_histogram(const uint32_t* in_k, int n, int c0, int shift, SortSmem& m) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int dv[kSortIpt];
#pragma unroll
  for (int u = 0; u < kSortIpt; ++u) {
    const int i = c0 + warp * (32 * kSortIpt) + u * 32 + lane;
    dv[u] = i < n ? (int)((__ldcg(in_k + i) >> shift) & 255u) : 256;
  }
#pragma unroll
  for (int u = 0; u < kSortIpt; ++u) {
    const bool valid = dv[u] < 256;
    const unsigned peers = digit_peers(dv[u] & 255, valid);
    if (valid && (peers & lt) == 0) m.wh[dv[u] * 32 + warp] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  scan_warp_counts(m);  // tot[d] = the chunk's count of digit d
  __syncthreads();
  zero_wh(m);
  __syncthreads();
}

// One stable counting-sort pass in one block (the tile order of the plan).
__device__ void stable_pass(const int32_t* in_i, const uint32_t* in_k, int32_t* out_i,
                            uint32_t* out_k, int n, int shift, SortSmem& m) {
  static_assert(kPlanThreads == 1024, "one thread per (digit, quarter of the warps)");
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid < 256) m.base[tid] = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += kSortChunk) {
    chunk_histogram(in_k, n, c0, shift, m);
    if (tid < 256) m.base[tid] += m.tot[tid];
    __syncthreads();
  }
  if (warp == 0) {  // digit totals -> exclusive digit starts
    warp_scan256(m.base, m.lstart);
    __syncwarp();
    for (int d = threadIdx.x; d < 256; d += 32) m.base[d] = m.lstart[d];
  }
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += kSortChunk) {
    scatter_chunk(in_i, in_k, out_i, out_k, n, c0, shift, m);
    if (tid < 256) m.base[tid] += m.tot[tid];
    __syncthreads();
  }
}

__device__ __forceinline__ int len_key(int T) { return kLenBuckets - 1 - length_bucket(T); }
static_assert(kLenBuckets == 1024, "sort keys hold the length key in 10 bits");

// Length of every tile = its longest row (the length buckets above 255 are
// wider than one length, so the first row is not always the longest); one
// warp per tile.
__device__ void tile_lengths(const MmaPlanArgs& a, int n_tiles) {
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int id = warp; id < n_tiles; id += kPlanThreads / 32) {
    const int p = a.tile_start[id], rows = a.tile_rows[id];
    int mx = 0;
    for (int q = lane; q < rows; q += 32) mx = max(mx, a.seqlen[a.sorted[p + q]]);
    mx = __reduce_max_sync(HMM_FULL_MASK, mx);
    if (lane == 0) a.tile_len[id] = mx;
  }
  __syncthreads();
}

// Plan stage 1 (one block per 4 * kPlanThreads rows): rows with T >= 1 are
// counted per block; the other rows get their log-likelihood here.
__global__ void __launch_bounds__(kPlanThreads) plan_count_kernel(MmaPlanArgs a) {
  __shared__ int itmp[32];
  __shared__ int total;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * 4 * kPlanThreads;
  int cnt = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int s = c0 + 4 * tid + u;
    const int T = s < a.S ? a.seqlen[s] : 0;
    const bool keep = s < a.S && T >= 1;
    cnt += keep ? 1 : 0;
    if (s < a.S && !keep) {
      const float v = T == 0 ? 0.f : __int_as_float(0x7fc00000);
      if (a.labelled) a.loglik[s] = v;
      else
        for (int k = 0; k < a.K; ++k) a.loglik[(size_t)s * a.K + k] = v;
    }
  }
  block_exclusive_scan<int>(cnt, itmp, &total);
  if (tid == 0) a.bcnt[blockIdx.x] = total;
}

// Exclusive prefix of `n` counts in place (one block); the total to *sum.
__global__ void __launch_bounds__(kPlanThreads) plan_scan_kernel(int32_t* v, int n, int32_t* sum) {
  __shared__ int itmp[32];
  __shared__ int total;
  int carry = 0;
  for (int c0 = 0; c0 < n; c0 += kPlanThreads) {
    const int i = c0 + threadIdx.x;
    const int x = i < n ? v[i] : 0;
    const int ex = block_exclusive_scan<int>(x, itmp, &total);
    if (i < n) v[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && sum) *sum = carry;
}

// Plan stage 2: every block writes its valid rows, in index order, with their
// sort keys (model << 10 | length key) at its offset.
__global__ void __launch_bounds__(kPlanThreads) plan_rows_kernel(MmaPlanArgs a) {
  __shared__ int itmp[32];
  __shared__ int total;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * 4 * kPlanThreads;
  int keep[4], cnt = 0;
  uint32_t key[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int s = c0 + 4 * tid + u;
    const int T = s < a.S ? a.seqlen[s] : 0;
    keep[u] = (s < a.S && T >= 1) ? 1 : 0;
    key[u] = keep[u] ? (((a.labelled ? (uint32_t)a.model_of_seq[s] : 0u) << 10) |
                        (uint32_t)len_key(T))
                     : 0u;
    cnt += keep[u];
  }
  int pos = a.bcnt[blockIdx.x] + block_exclusive_scan<int>(cnt, itmp, &total);
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (keep[u]) {
      a.sorted[pos] = c0 + 4 * tid + u;
      a.key[pos] = key[u];
      ++pos;
    }
}

// One pass of the stable LSD sort over many blocks, a 4096-pair chunk each:
// per-chunk digit counts (digit-major [256][chunks]) ...
__global__ void __launch_bounds__(kPlanThreads) plan_hist_kernel(const uint32_t* in_k,
                                                                 const int32_t* n_valid,
                                                                 int shift, int32_t* hist,
                                                                 int nchunks) {
  extern __shared__ __align__(16) uint8_t plan_smem[];
  SortSmem& m = *reinterpret_cast<SortSmem*>(plan_smem);
  const int tid = threadIdx.x;
  for (int i = tid; i < 32 * 256; i += kPlanThreads) m.wh[i] = 0;
  __syncthreads();
  const int n = *n_valid;
  const int c0 = blockIdx.x * kSortChunk;
  if (c0 < n) chunk_histogram(in_k, n, c0, shift, m);
  if (tid < 256) hist[(size_t)tid * nchunks + blockIdx.x] = c0 < n ? m.tot[tid] : 0;
}

// ... and, after their exclusive prefix, every chunk written out stably.
__global__ void __launch_bounds__(kPlanThreads) plan_scatter_kernel(
    const int32_t* in_i, const uint32_t* in_k, int32_t* out_i, uint32_t* out_k,
    const int32_t* n_valid, int shift, const int32_t* off, int nchunks) {
  extern __shared__ __align__(16) uint8_t plan_smem[];
  SortSmem& m = *reinterpret_cast<SortSmem*>(plan_smem);
  const int tid = threadIdx.x;
  const int n = *n_valid;
  const int c0 = blockIdx.x * kSortChunk;
  if (c0 >= n) return;
  for (int i = tid; i < 32 * 256; i += kPlanThreads) m.wh[i] = 0;
  if (tid < 256) m.base[tid] = off[(size_t)tid * nchunks + blockIdx.x];
  __syncthreads();
  scatter_chunk(in_i, in_k, out_i, out_k, n, c0, shift, m);
}

// Plan stage 3 (one block): tiles of at most 128 rows of one model, their
// lengths, and the longest-first tile order.
__global__ void __launch_bounds__(kPlanThreads) plan_tiles_kernel(MmaPlanArgs a) {
  extern __shared__ __align__(16) uint8_t plan_smem[];
  SortSmem& m = *reinterpret_cast<SortSmem*>(plan_smem);
  __shared__ int itmp[32];
  __shared__ int total;
  const int tid = threadIdx.x;
  for (int i = tid; i < 32 * 256; i += kPlanThreads) m.wh[i] = 0;
  __syncthreads();
  const int n = *a.n_valid;

  // tiles of at most 128 rows of one model
  int n_tiles = 0;
  if (a.labelled) {
    const uint32_t* keys = a.key;
    auto model_at = [keys](int p) { return (int)(__ldcg(keys + p) >> 10); };
    // first and one-past-last position of every model's group
    for (int p = tid; p < n; p += kPlanThreads) {
      const int k = model_at(p);
      if (p == 0 || model_at(p - 1) != k) a.group_start[k] = p;
      if (p == n - 1 || model_at(p + 1) != k) a.group_end[k] = p + 1;
    }
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 4 * kPlanThreads) {
      int flag[4], kk[4], ge[4], cnt = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = c0 + 4 * tid + u;
        flag[u] = 0; kk[u] = 0; ge[u] = 0;
        if (p < n) {
          kk[u] = model_at(p);
          ge[u] = a.group_end[kk[u]];
          flag[u] = ((p - a.group_start[kk[u]]) % 128) == 0 ? 1 : 0;
        }
        cnt += flag[u];
      }
      int id = n_tiles + block_exclusive_scan<int>(cnt, itmp, &total);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = c0 + 4 * tid + u;
        if (flag[u]) {
          if (id < a.n_tiles_cap) {
            a.tile_start[id] = p;
            a.tile_rows[id] = min(128, ge[u] - p);
            a.tile_model[id] = kk[u];
            a.tile_order[id] = id;
          }
          ++id;
        }
      }
      n_tiles += total;
      __syncthreads();
    }
    n_tiles = min(n_tiles, a.n_tiles_cap);
    tile_lengths(a, n_tiles);
    // longest tiles first (stable in tile index): keys = length keys; the
    // row keys are no longer needed, their buffers hold the tile keys
    for (int id = tid; id < n_tiles; id += kPlanThreads) {
      a.tile_tmp[id] = id;
      a.key_tmp[id] = (uint32_t)len_key(a.tile_len[id]);
    }
    __syncthreads();
    stable_pass(a.tile_tmp, a.key_tmp, a.tile_order, a.key, n_tiles, 0, m);
    stable_pass(a.tile_order, a.key, a.tile_tmp, a.key_tmp, n_tiles, 8, m);
    for (int id = tid; id < n_tiles; id += kPlanThreads) a.tile_order[id] = a.tile_tmp[id];
    __syncthreads();
  } else {
    // every length-sorted chunk of 128 rows against every model, chunk-major
    // (already longest first)
    const int n_chunks = (n + 127) / 128;
    n_tiles = min(n_chunks * a.K, a.n_tiles_cap);
    for (int id = tid; id < n_tiles; id += kPlanThreads) {
      const int c = id / a.K, k = id % a.K;
      a.tile_start[id] = 128 * c;
      a.tile_rows[id] = min(128, n - 128 * c);
      a.tile_model[id] = k;
      a.tile_order[id] = id;
    }
    __syncthreads();
    tile_lengths(a, n_tiles);
  }
  for (int id = n_tiles + tid; id < a.n_tiles_cap; id += kPlanThreads) {
    a.tile_len[id] = -1;
    a.tile_model[id] = 0;
  }
  if (tid == 0) *a.n_tiles = n_tiles;
}

// Work lists of the adjoint's two kernels (one block, after the tile stage).
//  * pass groups: `group` tiles of one model that one CTA of the pass kernel
//    runs side by side -- the tiles of a model in decreasing-length order
//    (consecutive tile ids in labelled mode, every K-th id otherwise), cut
//    into runs of `group`; groups ordered by their longest tile, longest
//    first (stable in the leader's id);
//  * range items: every tile's checkpoint segments cut into runs of `spr`
//    (the last run shorter), tiles in tile_order (longest first).
__global__ void __launch_bounds__(kPlanThreads) plan_items_kernel(MmaPlanArgs a) {
  extern __shared__ __align__(16) uint8_t plan_smem[];
  SortSmem& m = *reinterpret_cast<SortSmem*>(plan_smem);
  __shared__ int itmp[32];
  __shared__ int total;
  const int tid = threadIdx.x;
  for (int i = tid; i < 32 * 256; i += kPlanThreads) m.wh[i] = 0;
  const int n = *a.n_tiles;
  const int step = a.labelled ? 1 : a.K;  // id distance of consecutive tiles of a model

  // ---- pass groups: leaders (rank within the model a multiple of group)
  int n_groups = 0;
  int32_t* lead = a.pass_tmp;                  // leaders, id order
  uint32_t* lkey = a.key_tmp;                  // their length keys
  for (int c0 = 0; c0 < n; c0 += kPlanThreads) {
    const int id = c0 + tid;
    int flag = 0;
    if (id < n) {
      const int k = a.tile_model[id];
      const int rank = a.labelled ? (a.tile_start[id] - a.group_start[k]) / 128 : id / a.K;
      flag = (rank % a.group) == 0 ? 1 : 0;
    }
    const int pos = n_groups + block_exclusive_scan<int>(flag, itmp, &total);
    if (flag && pos < a.pass_cap) {
      lead[pos] = id;
      lkey[pos] = (uint32_t)len_key(a.tile_len[id]);
    }
    n_groups += total;
    __syncthreads();
  }
  n_groups = min(n_groups, a.pass_cap);
  int32_t* srt = a.pass_tmp + a.pass_cap;
  stable_pass(lead, lkey, srt, a.key, n_groups, 0, m);
  stable_pass(srt, a.key, lead, lkey, n_groups, 8, m);
  for (int g = tid; g < n_groups; g += kPlanThreads) {
    const int id = lead[g], k = a.tile_model[id];
    for (int j = 0; j < a.group; ++j) {
      const int q = id + j * step;
      a.pass_tiles[g * a.group + j] = (q < n && a.tile_model[q] == k) ? q : -1;
    }
  }
  if (tid == 0) *a.n_pass = n_groups;

  // ---- range items, tiles longest first
  int n_items = 0;
  for (int c0 = 0; c0 < n; c0 += kPlanThreads) {
    const int j = c0 + tid;
    int nr = 0, tile = 0, ns = 0;
    if (j < n) {
      tile = a.tile_order[j];
      const int L = a.tile_len[tile];
      const int C = fb_mma_segment(L);
      ns = (L + C - 1) / C;
      nr = (ns + a.spr - 1) / a.spr;
    }
    const int base = n_items + block_exclusive_scan<int>(nr, itmp, &total);
    for (int r = 0; r < nr; ++r) {
      const int i = base + r;
      if (i >= a.rng_cap) break;
      const int lo = r * a.spr, hi = min(ns - 1, lo + a.spr - 1);
      a.rng_tile[i] = tile;
      a.rng_seg[i] = lo | (hi << 16);
      a.rng_model[i] = a.tile_model[tile];
      a.rng_len[i] = a.tile_len[tile];
    }
    n_items += total;
    __syncthreads();
  }
  n_items = min(n_items, a.rng_cap);
  for (int i = n_items + tid; i < a.rng_cap; i += kPlanThreads) {
    a.rng_len[i] = -1;
    a.rng_model[i] = 0;
  }
  if (tid == 0) *a.n_rng = n_items;
}

cudaError_t launch_mma_plan(const MmaPlanArgs& a, cudaStream_t st) {
  const int smem = (int)sizeof(SortSmem);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(plan_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem)))
    return e;
  if ((e = cudaFuncSetAttribute(plan_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem)))
    return e;
  if ((e = cudaFuncSetAttribute(plan_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem)))
    return e;
  const int nrb = (a.S + 4 * kPlanThreads - 1) / (4 * kPlanThreads);  // row blocks
  const int nch = (a.S + kSortChunk - 1) / kSortChunk;                // sort chunks
  if (nrb < 1 || nch < 1) return cudaErrorInvalidValue;
  plan_count_kernel<<<nrb, kPlanThreads, 0, st>>>(a);
  plan_scan_kernel<<<1, kPlanThreads, 0, st>>>(a.bcnt, nrb, a.n_valid);
  plan_rows_kernel<<<nrb, kPlanThreads, 0, st>>>(a);
  // key bits: 10 of length, then the model; an even number of 8-bit passes
  // so the result lands back in (sorted, key)
  int bits = 10;
  if (a.labelled)
    while (bits < 32 && ((a.K - 1) >> (bits - 10)) != 0) ++bits;
  int passes = (bits + 7) / 8;
  passes += passes & 1;
  int32_t* ci = a.sorted;
  uint32_t* ck = a.key;
  int32_t* oi = a.tmp;
  uint32_t* ok = a.key_tmp;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    plan_hist_kernel<<<nch, kPlanThreads, smem, st>>>(ck, a.n_valid, shift, a.hist, nch);
    plan_scan_kernel<<<1, kPlanThreads, 0, st>>>(a.hist, 256 * nch, nullptr);
    plan_scatter_kernel<<<nch, kPlanThreads, smem, st>>>(ci, ck, oi, ok, a.n_valid, shift,
                                                         a.hist, nch);
    int32_t* ti = ci; ci = oi; oi = ti;
    uint32_t* tk = ck; ck = ok; ok = tk;
  }
  plan_tiles_kernel<<<1, kPlanThreads, smem, st>>>(a);
  if (a.pass_tiles) {
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(plan_items_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem)))
      return e;
    plan_items_kernel<<<1, kPlanThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// row softmax and its chain rule (one warp per row)
// ---------------------------------------------------------------------------
struct RowMap {
  int K, N, M;
  __device__ __forceinline__ bool row(long long r, long long& base, int& width) const {
    const long long r_pi = K, r_A = (long long)K * N, r_B = (long long)K * N;
    if (r < r_pi) { base = r * N; width = N; return true; }
    r -= r_pi;
    if (r < r_A) { base = (long long)K * N + r * N; width = N; return true; }
    r -= r_A;
    if (r < r_B) { base = (long long)K * N + (long long)K * N * N + r * M; width = M; return true; }
    return false;
  }
};

// Tables are addressed as one virtual array [pi | A | B]; `sel` picks the
// real pointer for a virtual base.
struct Tables {
  const float* pi; const float* A; const float* B;
  long long nA0, nB0;  // virtual starts of A and B
  __device__ __forceinline__ const float* at(long long base) const {
    if (base < nA0) return pi + base;
    if (base < nB0) return A + (base - nA0);
    return B + (base - nB0);
  }
};
struct MTables {
  float* pi; float* A; float* B;
  long long nA0, nB0;
  __device__ __forceinline__ float* at(long long base) const {
    if (base < nA0) return pi + base;
    if (base < nB0) return A + (base - nA0);
    return B + (base - nB0);
  }
};

__global__ void softmax_rows_kernel(RowMap map, Tables in, MTables out, long long nrows) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  long long base; int width;
  map.row(r, base, width);
  const float* x = in.at(base);
  float* y = out.at(base);
  float mx = -INFINITY;
  for (int c = lane; c < width; c += 32) mx = fmaxf(mx, x[c]);
  mx = group_max<32>(mx);
  float s = 0.f;
  for (int c = lane; c < width; c += 32) s += expf(x[c] - mx);
  s = group_sum<32>(s);
  const float inv = 1.f / s;
  for (int c = lane; c < width; c += 32) y[c] = expf(x[c] - mx) * inv;
}

__global__ void softmax_grad_kernel(RowMap map, Tables p, Tables c, MTables g, long long nrows) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  long long base; int width;
  map.row(r, base, width);
  const float* pp = p.at(base);
  const float* cc = c.at(base);
  float* gg = g.at(base);
  float tot = 0.f;
  for (int q = lane; q < width; q += 32) tot += cc[q];
  tot = group_sum<32>(tot);
  __syncwarp();
  for (int q = lane; q < width; q += 32) gg[q] = cc[q] - pp[q] * tot;
}

// Baum-Welch re-estimation (Rabiner eq. 40): every row of pi, A and B becomes
// its expected counts normalised to sum 1; a row whose counts sum to zero keeps
// its old values. Outputs may alias the old parameters (each element depends
// on its own row only).
__global__ void mstep_kernel(RowMap map, Tables p, Tables c, MTables out, long long nrows) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  long long base; int width;
  map.row(r, base, width);
  const float* pp = p.at(base);
  const float* cc = c.at(base);
  float* oo = out.at(base);
  float tot = 0.f;
  for (int q = lane; q < width; q += 32) tot += cc[q];
  tot = group_sum<32>(tot);
  const float inv = tot > 0.f ? 1.f / tot : 0.f;
  __syncwarp();
  for (int q = lane; q < width; q += 32) oo[q] = tot > 0.f ? cc[q] * inv : pp[q];
}

static long long n_rows(int K, int N) { return (long long)K + 2LL * K * N; }

cudaError_t launch_mstep(int K, int N, int M, const float* pi, const float* A, const float* B,
                         const float* cpi, const float* cA, const float* cB, float* opi,
                         float* oA, float* oB, cudaStream_t st) {
  RowMap map{K, N, M};
  const long long nA0 = (long long)K * N, nB0 = nA0 + (long long)K * N * N;
  Tables p{pi, A, B, nA0, nB0};
  Tables c{cpi, cA, cB, nA0, nB0};
  MTables o{opi, oA, oB, nA0, nB0};
  const long long rows = n_rows(K, N);
  const int threads = 256;
  const long long blocks = (rows * 32 + threads - 1) / threads;
  mstep_kernel<<<(unsigned)blocks, threads, 0, st>>>(map, p, c, o, rows);
  return cudaGetLastError();
}

cudaError_t launch_softmax_rows(int K, int N, int M, const float* lpi, const float* lA,
                                const float* lB, float* pi, float* A, float* B, cudaStream_t st) {
  RowMap map{K, N, M};
  const long long nA0 = (long long)K * N, nB0 = nA0 + (long long)K * N * N;
  Tables in{lpi, lA, lB, nA0, nB0};
  MTables out{pi, A, B, nA0, nB0};
  const long long rows = n_rows(K, N);
  const int threads = 256;
  const long long blocks = (rows * 32 + threads - 1) / threads;
  softmax_rows_kernel<<<(unsigned)blocks, threads, 0, st>>>(map, in, out, rows);
  return cudaGetLastError();
}

cudaError_t launch_softmax_grad(int K, int N, int M, const float* pi, const float* A,
                                const float* B, const float* cpi, const float* cA,
                                const float* cB, float* gpi, float* gA, float* gB,
                                cudaStream_t st) {
  RowMap map{K, N, M};
  const long long nA0 = (long long)K * N, nB0 = nA0 + (long long)K * N * N;
  Tables p{pi, A, B, nA0, nB0};
  Tables c{cpi, cA, cB, nA0, nB0};
  MTables g{gpi, gA, gB, nA0, nB0};
  const long long rows = n_rows(K, N);
  const int threads = 256;
  const long long blocks = (rows * 32 + threads - 1) / threads;
  softmax_grad_kernel<<<(unsigned)blocks, threads, 0, st>>>(map, p, c, g, rows);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adam
// ---------------------------------------------------------------------------
__global__ void adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float gs, const int32_t* __restrict__ step) {
  const float t = (float)(*step + 1);
  const float inv_bc1 = 1.f / (1.f - powf(b1, t));
  const float inv_bc2 = 1.f / (1.f - powf(b2, t));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = gs * g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
  }
}

__global__ void step_increment_kernel(int32_t* step) { *step += 1; }

cudaError_t launch_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr,
                        float b1, float b2, float eps, float gs, int32_t* step, cudaStream_t st) {
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  blocks = blocks < 4LL * num_sms() ? blocks : 4LL * num_sms();
  if (blocks < 1) blocks = 1;
  adam_kernel<<<(unsigned)blocks, threads, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, gs, step);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  step_increment_kernel<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fixed-order reduction of the adjoint's per-pair count partials
// ---------------------------------------------------------------------------
constexpr int kReduceModels = 16;  // models per first-level block

__global__ void __launch_bounds__(kReduceTile) reduce1_kernel(ReduceLaunch a, int chunk) {
  __shared__ float acc[kReduceModels][kReduceTile];
  const int tid = threadIdx.x;
  const int64_t e = (int64_t)blockIdx.x * kReduceTile + tid;
  const int c = blockIdx.y;
  const int k0 = blockIdx.z * kReduceModels;
  const int k1 = min(a.K, k0 + kReduceModels);
#pragma unroll
  for (int q = 0; q < kReduceModels; ++q) acc[q][tid] = 0.f;
  const int Stot = a.S * a.planes;  // slot rows: plane-major, sequence index q % S
  const int s0 = c * chunk, s1 = min(Stot, s0 + chunk);
  if (e >= a.slot_floats) return;
  constexpr int U = 8;  // independent loads in flight
  if (a.model_of_seq) {
    for (int s = s0; s < s1; s += U) {
      float v[U];
      int kk[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = s + u;
        kk[u] = -1;
        v[u] = 0.f;
        if (q < s1 && a.seqlen[q % a.S] >= 0) {
          const int k = a.model_of_seq[q % a.S];
          if (k >= k0 && k < k1) {
            kk[u] = k - k0;
            v[u] = a.partial[(int64_t)q * a.slot_floats + e];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (kk[u] >= 0) acc[kk[u]][tid] += v[u];
    }
  } else {
    for (int s = s0; s < s1; ++s) {
      if (a.seqlen[s % a.S] < 0) continue;
      const float* row = a.partial + (int64_t)s * a.K * a.slot_floats + e;
      float v[kReduceModels];
#pragma unroll
      for (int q = 0; q < kReduceModels; ++q)
        v[q] = (k0 + q < k1) ? row[(int64_t)(k0 + q) * a.slot_floats] : 0.f;
#pragma unroll
      for (int q = 0; q < kReduceModels; ++q) acc[q][tid] += v[q];
    }
  }
  for (int k = k0; k < k1; ++k) a.red1[((int64_t)c * a.K + k) * a.slot_floats + e] = acc[k - k0][tid];
}

__global__ void reduce2_kernel(ReduceLaunch a) {
  const int64_t nA = (int64_t)a.K * a.N;
  const int64_t nAA = nA * a.N;
  const int64_t nB = nA * a.M;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nA + nAA + nB) return;
  int k;
  int64_t e;
  float* out;
  if (idx < nA) {
    k = (int)(idx / a.N);
    const int i = (int)(idx % a.N);
    e = i;
    out = a.cnt_pi + idx;
  } else if (idx < nA + nAA) {
    const int64_t r = idx - nA;
    k = (int)(r / ((int64_t)a.N * a.N));
    const int i = (int)((r / a.N) % a.N), j = (int)(r % a.N);
    e = a.NP + (int64_t)i * a.NP + j;
    out = a.cnt_A + r;
  } else {
    const int64_t r = idx - nA - nAA;
    k = (int)(r / ((int64_t)a.N * a.M));
    const int j = (int)((r / a.M) % a.N), m = (int)(r % a.M);
    e = a.NP + (int64_t)a.NP * a.NP + (int64_t)j * a.M + m;
    out = a.cnt_B + r;
  }
  // chunks in order, eight loads in flight
  const int64_t stride = (int64_t)a.K * a.slot_floats;
  const float* p = a.red1 + (int64_t)k * a.slot_floats + e;
  float s = 0.f;
  int c = 0;
  for (; c + 8 <= a.nchunks; c += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = p[(int64_t)(c + u) * stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; c < a.nchunks; ++c) s += p[(int64_t)c * stride];
  *out = s;
}

cudaError_t launch_reduce(const ReduceLaunch& a, cudaStream_t st) {
  const int chunk = (a.S * a.planes + a.nchunks - 1) / a.nchunks;
  dim3 g1((unsigned)((a.slot_floats + kReduceTile - 1) / kReduceTile), (unsigned)a.nchunks,
          (unsigned)((a.K + kReduceModels - 1) / kReduceModels));
  reduce1_kernel<<<g1, kReduceTile, 0, st>>>(a, chunk);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t n = (int64_t)a.K * a.N * (1 + a.N + a.M);
  reduce2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hmmgb
