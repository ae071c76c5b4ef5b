// fb.cu -- forward-backward adjoint, FP32 SIMT (Sec. 2.7 "Baum-Welch", its
// E-step; Rabiner 1989 eqs. 24-25 backward variable, 37 xi, 38 gamma).
//
// For one (sequence, model) pair with weight w the kernel produces
//   C_pi(i)   += w gamma_1(i)
//   C_A(i,j)  += w sum_{t<T} xi_t(i,j)
//   C_B(j,m)  += w sum_{t: o_t = m} gamma_t(j)
// into a per-pair slot of the workspace (summed later in a fixed order).
//
// Memory: alpha is never stored whole. Phase 1 runs the scaled forward
// recursion and keeps alpha_t (and the power-of-two exponent removed at t)
// every C = ceil(sqrt(max_len)) steps in shared memory. Phase 2 walks the
// segments backwards; while it runs the backward recursion over segment c it
// recomputes alpha over segment c-1 from its checkpoint (the two chains are
// independent, so each step issues both), double-buffering the segments in
// shared memory: O(sqrt(T) N) floats per pair.
//
// Scaling: alpha_t and beta_t each carry an exact power-of-two scale that is
// never divided out. With u_{t+1}(j) = b_j(o_{t+1}) beta_{t+1}(j) and the
// forward exponent e_{t+1} removed at step t+1,
//   Z_t = sum_j (alpha_t A)_j u_{t+1}(j) = 2^{e_{t+1}} D_{t+1},
//   D_{t+1} = sum_j alpha_{t+1}(j) beta_{t+1}(j),
// so with v(j) = u_{t+1}(j) / Z_t
//   xi_t(i,j)      = alpha_t(i) a_ij v(j)          (a_ij applied at the flush)
//   gamma_{t+1}(j) = alpha_{t+1}(j) beta_{t+1}(j) / D_{t+1}
//   beta_t(i)     ~ sum_j a_ij v(j)                (then rescaled),
// and the weight w multiplies only what is accumulated. D_t comes out of the
// same butterfly as the sum that rescales beta_t (one reduction per step).
// Lane ownership: lane r of the pair owns states [rJ, rJ+J) both as columns
// (forward: column slice of A) and as rows (backward: row slice of A, row
// slice of the xi accumulator), so every step needs one broadcast vector.
#include "fb_common.cuh"

namespace hmmgb {

template <int NP, int G>
struct FbLayout {
  static constexpr int J = NP / G;
  static constexpr int PP = 32 / G;
  static constexpr int XS = NP + 4;
  // floats per pair, rounded to 4 (16-byte alignment of every region)
  static __host__ __device__ int per_pair(int C, int NC, int M) {
    const int n = 4 * XS + NC * NP + 2 * C * NP + NC + 2 * C + NP * (M + 1);
    return (n + 3) & ~3;
  }
};

template <int NP, int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
hmm_fb_simt(FbLaunch a) {
  using L = FbLayout<NP, G>;
  constexpr int J = L::J, PP = L::PP, XS = L::XS;
  extern __shared__ __align__(16) float smem[];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / G, r = lane % G, j0 = r * J;
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;
  const int C = a.ckpt, NC = a.nck, MP = M + 1;
  const bool labelled = a.seq.model_of_seq != nullptr;

  const int per = L::per_pair(C, NC, M);
  float* base = smem + (size_t)(warp * PP + p) * per;
  float* xf = base;                                   // [2][XS] forward exchange
  float* xv = xf + 2 * XS;                            // [2][XS] backward exchange
  float* ck = xv + 2 * XS;                            // [NC][NP] checkpoints
  float* seg = ck + NC * NP;                          // [2][C][NP] recomputed segments
  int* cke = reinterpret_cast<int*>(seg + 2 * C * NP);  // [NC]
  int* sege = cke + NC;                               // [2][C]
  float* cb = reinterpret_cast<float*>(sege + 2 * C);   // [NP][MP] emission counts

  for (int e = r; e < NP * MP; e += G) cb[e] = 0.f;
  __syncwarp();

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_items) break;
    const int g = labelled ? item : item / K;
    int k = labelled ? 0 : item % K;
    const int pos = g * PP + p;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    if (labelled && has && T >= 0) k = a.seq.model_of_seq[s];
    const size_t slot = labelled ? (size_t)s : (size_t)s * K + k;
    const int Tn = T < 0 ? 0 : T;
    const float w = (has && a.weight) ? a.weight[slot] : 1.f;

    // A slices of this pair's model
    float2 ac[NP / 2][J];  // ac[i2][jj] = (a_{2i2, j}, a_{2i2+1, j}),  j = j0 + jj
    float2 ar[J][NP / 2];  // ar[ii][j2] = (a_{i, 2j2}, a_{i, 2j2+1}),  i = j0 + ii
    {
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
#pragma unroll
      for (int i2 = 0; i2 < NP / 2; ++i2)
#pragma unroll
        for (int jj = 0; jj < J; ++jj)
          ac[i2][jj] = make_float2(__ldg(Ak + (2 * i2) * NP + j0 + jj),
                                   __ldg(Ak + (2 * i2 + 1) * NP + j0 + jj));
#pragma unroll
      for (int ii = 0; ii < J; ++ii)
#pragma unroll
        for (int j2 = 0; j2 < NP / 2; ++j2)
          ar[ii][j2] = __ldg(reinterpret_cast<const float2*>(Ak + (j0 + ii) * NP) + j2);
    }
    const float* Bk = a.mod.Btp + (size_t)k * M * NP + j0;
    const int32_t* o = a.seq.symbols + ((has && T >= 0) ? a.seq.offsets[s] : 0);

    // ---------------- phase 1: forward with checkpoints ----------------
    float x[J];
    int E = 0;
    bool dead = false, bad = T < 0;
    int err = 0;
    {
      int o0 = Tn > 0 ? __ldg(o) : 0;
      if ((unsigned)o0 >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; o0 = 0; }
      float b[J], pv[J];
      load_vec<J>(b, Bk + (size_t)o0 * NP);
      load_vec<J>(pv, a.mod.pip + (size_t)k * NP + j0);
#pragma unroll
      for (int jj = 0; jj < J; ++jj) x[jj] = pv[jj] * b[jj];
      const float gs = group_sum<G>(tree_sum<J>(x));
      if (Tn > 0 && !bad) {
        if (gs == 0.f) dead = true;
        else if (!(gs > 0.f) || isinf(gs)) { bad = true; err |= HMM_STATUS_PARAM; }
        else {
          const int e = rescale_pow2<J>(x, gs);
          E += e;
          store_vec<J>(ck + j0, x);
          if (r == 0) cke[0] = e;
        }
      }
    }
    const int Tmax = __reduce_max_sync(HMM_FULL_MASK, Tn);
    {
      float bn[J];
      int on = 0;
      if (1 < Tn) {
        on = __ldg(o + 1);
        if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
      }
      load_vec<J>(bn, Bk + (size_t)on * NP);
      int o2 = (2 < Tn) ? __ldg(o + 2) : 0;
      for (int t = 1; t < Tmax; ++t) {
        const bool act = t < Tn && !dead && !bad;
        float* xw = xf + (t & 1) * XS;
        store_vec<J>(xw + j0, x);
        __syncwarp();
        float nx[J];
        matvec_cols<NP, J>(xw, ac, nx);
        float b[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) b[jj] = bn[jj];
        if (t + 1 < Tn) {
          on = o2;
          if ((unsigned)on >= (unsigned)M) { bad = true; err |= HMM_STATUS_SYMBOL; on = 0; }
          load_vec<J>(bn, Bk + (size_t)on * NP);
          if (t + 2 < Tn) o2 = __ldg(o + t + 2);
        }
#pragma unroll
        for (int jj = 0; jj < J; ++jj) nx[jj] *= b[jj];
        const float gs = group_sum<G>(tree_sum<J>(nx));
        if (act) {
          if (gs == 0.f) dead = true;
          else if (!(gs > 0.f) || isinf(gs)) { bad = true; err |= HMM_STATUS_PARAM; }
          else {
            const int e = rescale_pow2<J>(nx, gs);
            E += e;
#pragma unroll
            for (int jj = 0; jj < J; ++jj) x[jj] = nx[jj];
            if (t % C == 0) {
              store_vec<J>(ck + (t / C) * NP + j0, x);
              if (r == 0) cke[t / C] = e;
            }
          }
        }
      }
    }
    const float fs = group_sum<G>(tree_sum<J>(x));
    if (has && r == 0) {
      float out;
      if (bad) { out = __int_as_float(0x7fc00000); if (err) set_status(a.status, err); }
      else if (Tn == 0) out = 0.f;
      else if (dead) out = -INFINITY;
      else out = (float)(log((double)fs) + (double)E * 0.69314718055994530942);
      a.loglik[slot] = out;
    }

    // ---------------- phase 2: backward over segments ----------------
    const bool alive = has && !bad && !dead && Tn > 0;
    const int Tb = alive ? Tn : 0;
    const int TbMax = __reduce_max_sync(HMM_FULL_MASK, Tb);
    auto sym = [&](int t) -> int { return (alive && t >= 0 && t < Tb) ? __ldg(o + t) : 0; };
    float beta[J];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) beta[jj] = 1.f;
    float D = fs;  // D_{T-1} = sum_j alpha_{T-1}(j) * 1
    float2 xa[J][NP / 2];
#pragma unroll
    for (int ii = 0; ii < J; ++ii)
#pragma unroll
      for (int j2 = 0; j2 < NP / 2; ++j2) xa[ii][j2] = make_float2(0.f, 0.f);

    const int nseg = (TbMax + C - 1) / C;
    __syncwarp();
    // prologue: recompute the last segment
    if (nseg > 0) {
      const int c = nseg - 1, t0 = c * C, t1 = TbMax - 1;
      float* sg = seg + (c & 1) * C * NP;
      int* se = sege + (c & 1) * C;
      float xr[J];
      load_vec_smem<J>(xr, ck + c * NP + j0);
      store_vec<J>(sg + j0, xr);
      if (r == 0) se[0] = cke[c];
      for (int t = t0 + 1; t <= t1; ++t) {
        const bool act = alive && t <= Tb - 1;
        float* xw = xf + (t & 1) * XS;
        store_vec<J>(xw + j0, xr);
        __syncwarp();
        float nx[J], b[J];
        matvec_cols<NP, J>(xw, ac, nx);
        load_vec<J>(b, Bk + (size_t)sym(t) * NP);
#pragma unroll
        for (int jj = 0; jj < J; ++jj) nx[jj] *= b[jj];
        const float gs = group_sum<G>(tree_sum<J>(nx));
        if (act) {
          const int e = rescale_pow2<J>(nx, gs);
#pragma unroll
          for (int jj = 0; jj < J; ++jj) xr[jj] = nx[jj];
          store_vec<J>(sg + (t - t0) * NP + j0, xr);
          if (r == 0) se[t - t0] = e;
        }
      }
      __syncwarp();
    }

    for (int c = nseg - 1; c >= 0; --c) {
      const int t0 = c * C;
      const int t1 = min(t0 + C, TbMax) - 1;
      const float* cur = seg + (c & 1) * C * NP;
      const int* cure = sege + (c & 1) * C;
      float* nxt = seg + ((c + 1) & 1) * C * NP;  // segment c-1 (same parity as c+1)
      int* nxte = sege + ((c + 1) & 1) * C;
      const bool rc_on = c >= 1;
      const int r0 = (c - 1) * C;
      float xr[J];
      if (rc_on) {
        load_vec_smem<J>(xr, ck + (c - 1) * NP + j0);
        store_vec<J>(nxt + j0, xr);
        if (r == 0) nxte[0] = cke[c - 1];
      } else {
#pragma unroll
        for (int jj = 0; jj < J; ++jj) xr[jj] = 0.f;
      }
      // symbols and emission rows, one iteration ahead for both chains
      int sb = sym(t1 + 1);
      float bb[J];
      load_vec<J>(bb, Bk + (size_t)sb * NP);
      int sb_next = sym(t1);
      int sr_next = rc_on ? sym(r0 + 1) : 0;
      float br[J];
      load_vec<J>(br, Bk + (size_t)sr_next * NP);
      sr_next = rc_on ? sym(r0 + 2) : 0;

      for (int u = 0; u < C; ++u) {
        const int tb = t1 - u;
        const bool bact = tb >= t0 && alive && tb <= Tb - 2;
        const int tr = r0 + 1 + u;
        const bool ract = rc_on && u <= C - 2 && alive && tr <= Tb - 1;

        // backward: publish v = u_{t+1} / Z_t, count gamma_{t+1} emissions
        float a1[J], a0[J], v[J];
        int e1 = 0;
        if (bact) {
          if (tb + 1 <= t1) {
            load_vec_smem<J>(a1, cur + (tb + 1 - t0) * NP + j0);
            e1 = cure[tb + 1 - t0];
          } else {
            load_vec_smem<J>(a1, ck + (c + 1) * NP + j0);
            e1 = cke[c + 1];
          }
          load_vec_smem<J>(a0, cur + (tb - t0) * NP + j0);
          const float invD = 1.f / D;
          const float wd = w * invD;
#pragma unroll
          for (int jj = 0; jj < J; ++jj) {
            cb[(j0 + jj) * MP + sb] += wd * a1[jj] * beta[jj];
            v[jj] = mul_pow2(bb[jj] * beta[jj], -e1) * invD;
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < J; ++jj) { a0[jj] = 0.f; v[jj] = 0.f; }
        }
        float* vw = xv + (u & 1) * XS;
        float* xw = xf + (u & 1) * XS;
        store_vec<J>(vw + j0, v);
        store_vec<J>(xw + j0, xr);
        // prefetch next iteration's symbols / rows
        const int sb_cur = sb_next;
        sb_next = sym(tb - 1);
        float bbn[J];
        load_vec<J>(bbn, Bk + (size_t)sb_cur * NP);
        const int sr_cur = sr_next;
        sr_next = rc_on ? sym(tr + 2) : 0;
        float brn[J];
        load_vec<J>(brn, Bk + (size_t)sr_cur * NP);
        __syncwarp();

        // recompute step of segment c-1 (independent chain)
        float nx[J];
        matvec_cols<NP, J>(xw, ac, nx);
#pragma unroll
        for (int jj = 0; jj < J; ++jj) nx[jj] *= br[jj];
        const float rs = group_sum<G>(tree_sum<J>(nx));

        // backward step: beta_t and the xi accumulator
        float aw[J], nb[J];
#pragma unroll
        for (int ii = 0; ii < J; ++ii) aw[ii] = w * a0[ii];
        rows_step<NP, J>(vw, ar, aw, xa, nb);
        float ad[J];
#pragma unroll
        for (int ii = 0; ii < J; ++ii) ad[ii] = a0[ii] * nb[ii];
        const float2 red = group_sum2<G>(make_float2(tree_sum<J>(nb), tree_sum<J>(ad)));

        if (ract) {
          const int e = rescale_pow2<J>(nx, rs);
#pragma unroll
          for (int jj = 0; jj < J; ++jj) xr[jj] = nx[jj];
          store_vec<J>(nxt + (u + 1) * NP + j0, xr);
          if (r == 0) nxte[u + 1] = e;
        }
        if (bact && red.x > 0.f && !isinf(red.x)) {
          const int e = rescale_pow2<J>(nb, red.x);
#pragma unroll
          for (int ii = 0; ii < J; ++ii) beta[ii] = nb[ii];
          D = mul_pow2(red.y, -e);
        }
        sb = sb_cur;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) { bb[jj] = bbn[jj]; br[jj] = brn[jj]; }
      }
      __syncwarp();
    }

    // t = 0: gamma_1 for pi and the first emission
    float cpi[J];
    {
      float a0[J];
      if (alive) {
        load_vec_smem<J>(a0, ck + j0);
        const int o0 = __ldg(o);
        const float wd = w / D;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
          cpi[jj] = wd * a0[jj] * beta[jj];
          cb[(j0 + jj) * MP + o0] += cpi[jj];
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < J; ++jj) cpi[jj] = 0.f;
      }
    }
    __syncwarp();
    // ---------------- flush this pair's slot ----------------
    if (has) {
      float* out = a.partial + slot * a.slot_floats;
      store_vec<J>(out + j0, cpi);
#pragma unroll
      for (int ii = 0; ii < J; ++ii) {
        float2* row = reinterpret_cast<float2*>(out + NP + (size_t)(j0 + ii) * NP);
#pragma unroll
        for (int j2 = 0; j2 < NP / 2; ++j2)
          row[j2] = make_float2(ar[ii][j2].x * xa[ii][j2].x, ar[ii][j2].y * xa[ii][j2].y);
      }
      float* ob = out + NP + NP * NP;
#pragma unroll
      for (int jj = 0; jj < J; ++jj) {
        float* crow = cb + (j0 + jj) * MP;
        for (int m = 0; m < M; ++m) {
          ob[(size_t)(j0 + jj) * M + m] = crow[m];
          crow[m] = 0.f;
        }
      }
    }
    __syncwarp();
  }
}

// --------------------------------------------------------------------------
// dispatch
// --------------------------------------------------------------------------
// Shared memory of a block of `warps` warps (the per-pair regions of FbLayout).
size_t fb_smem_bytes(int NP, int G, int C, int NC, int M, int warps) {
  const int PP = 32 / G;
  const int XS = NP + 4;
  int n = 4 * XS + NC * NP + 2 * C * NP + NC + 2 * C + NP * (M + 1);
  n = (n + 3) & ~3;
  return (size_t)warps * PP * n * sizeof(float);
}

template <int NP, int G>
static cudaError_t launch_fb_t(const FbLaunch& a, cudaStream_t st) {
  auto kern = hmm_fb_simt<NP, G>;
  // as many warps per block (up to 4) as the per-pair buffers allow
  int warps = kWarpsPerBlock;
  while (warps > 1 && fb_smem_bytes(NP, G, a.ckpt, a.nck, a.seq.M, warps) > 227 * 1024) warps >>= 1;
  const size_t smem = fb_smem_bytes(NP, G, a.ckpt, a.nck, a.seq.M, warps);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int blocks = num_sms() * per_sm;
  const int need = (a.n_items + warps - 1) / warps;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<blocks, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

#define HMM_FB_CASE(NPV, GV) \
  if (NP == NPV && G == GV) return launch_fb_t<NPV, GV>(a, st);

cudaError_t launch_fb(int NP, int G, const FbLaunch& a, cudaStream_t st) {
  HMM_FB_CASE(4, 2) HMM_FB_CASE(4, 4)
  HMM_FB_CASE(8, 4) HMM_FB_CASE(8, 8)
  HMM_FB_CASE(16, 8) HMM_FB_CASE(16, 16)
  HMM_FB_CASE(32, 32)
  HMM_FB_CASE(64, 32)
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
