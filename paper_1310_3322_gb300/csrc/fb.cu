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
// never divided out, and the scale is applied lazily: a step multiplies its
// result by 2^-f, f the exponent of the sum of its INPUT row, which every lane
// of the pair adds up itself from the row it reads from shared memory for the
// product anyway. The recursion's critical path is then the product alone
// (no cross-lane reduction), and since a power of two commutes with rounding
// the stored values are those of a step-by-step normalisation up to an exact
// power of two. With the forward's f_t stored as e_{t+1} (the exponent applied
// to produce alpha_{t+1}), u_{t+1}(j) = b_j(o_{t+1}) beta_{t+1}(j) 2^-e_{t+1}:
//   Z_t = sum_j (alpha_t A)_j b_j(o_{t+1}) beta_{t+1}(j) = 2^{e_{t+1}} D_{t+1},
//   D_{t+1} = sum_j alpha_{t+1}(j) beta_{t+1}(j),
//   xi_t(i,j)      = alpha_t(i) a_ij u_{t+1}(j) / D_{t+1}   (a_ij applied at the flush)
//   gamma_{t+1}(j) = alpha_{t+1}(j) beta_{t+1}(j) / D_{t+1}
//   beta_t(i)     ~ sum_j a_ij u_{t+1}(j)                  (then scaled),
// and the weight w multiplies only what is accumulated. D_t is the one
// cross-lane reduction per backward step; it feeds only the accumulations of
// the next step, not the beta recursion.
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
    // x = alpha_t 2^-E; step t -> t+1 multiplies by 2^-f_t (f_t the exponent of
    // sum x_t), so E grows by f_t, and e_{t+1} = f_t is kept with checkpoints.
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
      if (Tn > 0) {
        store_vec<J>(ck + j0, x);
        if (r == 0) cke[0] = 0;
      }
    }
    const int Tmax = __reduce_max_sync(HMM_FULL_MASK, Tn);
    {
      // branch-free steps: flags and selects instead of per-pair branches
      float bn[J];
      int on = (1 < Tn) ? __ldg(o + 1) : 0;
      bool symbad = (unsigned)on >= (unsigned)M;
      on = symbad ? 0 : on;
      load_vec<J>(bn, Bk + (size_t)on * NP);
      int o2 = (2 < Tn) ? __ldg(o + 2) : 0;
      int cls = 0;         // OR of sum_class over the active steps
      int cc = 0, ci = 0;  // steps since the last checkpoint, its index
      for (int t = 1; t < Tmax; ++t) {
        const bool act = t < Tn;
        float* xw = xf + (t & 1) * XS;
        store_vec<J>(xw + j0, x);
        __syncwarp();
        float nx[J], sx;
        matvec_cols_sum<NP, J>(xw, ac, nx, sx);
        float b[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) b[jj] = bn[jj];
        {
          const bool nb_ = (unsigned)o2 >= (unsigned)M;
          symbad |= nb_ && t + 1 < Tn;
          on = nb_ ? 0 : o2;
          load_vec<J>(bn, Bk + (size_t)on * NP);
          if (t + 2 < Tn) o2 = __ldg(o + t + 2);
        }
        int f;
        const float sc = pow2_scale(sx, f);
#pragma unroll
        for (int jj = 0; jj < J; ++jj) nx[jj] = (nx[jj] * sc) * b[jj];
        if (++cc == C) { cc = 0; ++ci; }
        // x_{t-1} is checked here, x_{Tn-1} after the loop
        cls |= act ? sum_class(sx) : 0;
        E += act ? f : 0;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) x[jj] = act ? nx[jj] : x[jj];
        if (act && cc == 0) {
          store_vec<J>(ck + ci * NP + j0, x);
          if (r == 0) cke[ci] = f;
        }
      }
      if (symbad) { bad = true; err |= HMM_STATUS_SYMBOL; }
      if (cls & 2) { bad = true; err |= HMM_STATUS_PARAM; }
      else if (cls & 1) dead = true;
    }
    const float fs = group_sum<G>(tree_sum<J>(x));
    if (Tn > 0 && !bad && !dead) {
      if (fs == 0.f) dead = true;
      else if (!(fs > 0.f) || isinf(fs)) { bad = true; err |= HMM_STATUS_PARAM; }
    }
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
        float nx[J], b[J], sx;
        matvec_cols_sum<NP, J>(xw, ac, nx, sx);
        load_vec<J>(b, Bk + (size_t)sym(t) * NP);
        int f;
        const float sc = pow2_scale(sx, f);
#pragma unroll
        for (int jj = 0; jj < J; ++jj) nx[jj] = (nx[jj] * sc) * b[jj];
        if (act) {
#pragma unroll
          for (int jj = 0; jj < J; ++jj) xr[jj] = nx[jj];
          store_vec<J>(sg + (t - t0) * NP + j0, xr);
          if (r == 0) se[t - t0] = f;
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
      // alpha rows and exponents of the backward steps, one iteration ahead:
      // a1 = alpha_{t+1}, e1 = e_{t+1} (the next checkpoint at the segment's
      // end), a0 = alpha_t, e0 = e_t; indices clamped into the buffers (the
      // steps outside a pair's range are masked by bact)
      float a1[J], a0[J];
      load_vec_smem<J>(a1, ck + min(c + 1, NC - 1) * NP + j0);
      int e1 = cke[min(c + 1, NC - 1)];
      load_vec_smem<J>(a0, cur + (t1 - t0) * NP + j0);
      int e0 = cure[t1 - t0];

      for (int u = 0; u < C; ++u) {
        const int tb = t1 - u;
        const bool bact = tb >= t0 && alive && tb <= Tb - 2;
        const int tr = r0 + 1 + u;
        const bool ract = rc_on && u <= C - 2 && alive && tr <= Tb - 1;

        // backward: publish u_{t+1} = b beta_{t+1} 2^-e_{t+1}, count gamma_{t+1}.
        // Branch-free (selects), so that the compiler can interleave the two
        // chains and the accumulations.
        const int nidx = max(tb - 1 - t0, 0);
        float a0n[J];
        load_vec_smem<J>(a0n, cur + nidx * NP + j0);
        const int e0n = cure[nidx];
        float aw[J], v[J];
        const float invD = __frcp_rn(D);
        const float se1 = exp2i(-e1);
        const float wd = w * invD;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
          const float gam = wd * a1[jj] * beta[jj];
          float* cbp = cb + (j0 + jj) * MP + sb;
          if (bact) *cbp += gam;
          v[jj] = bact ? (bb[jj] * beta[jj]) * se1 : 0.f;
          aw[jj] = bact ? (w * a0[jj]) * invD : 0.f;
        }
        float a0s[J], a0m[J];  // alpha_t (kept for the next step), masked copy
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
          a0s[jj] = a0[jj];
          a0m[jj] = bact ? a0[jj] : 0.f;
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
        float nx[J], sx;
        matvec_cols_sum<NP, J>(xw, ac, nx, sx);
        int fr;
        const float scr = pow2_scale(sx, fr);
#pragma unroll
        for (int jj = 0; jj < J; ++jj) nx[jj] = (nx[jj] * scr) * br[jj];

        // backward step: beta_t (scaled by the exponent of sum u) and the xi
        // accumulator, normalised by D_{t+1}
        float nb[J], su;
        rows_step_sum<NP, J>(vw, ar, aw, xa, nb, su);
        int fu;
        const float sg = pow2_scale(su, fu);
        float ad[J];
#pragma unroll
        for (int ii = 0; ii < J; ++ii) {
          nb[ii] *= sg;
          ad[ii] = a0m[ii] * nb[ii];
        }
        const float Dn = group_sum<G>(tree_sum<J>(ad));

        if (ract) {
          store_vec<J>(nxt + (u + 1) * NP + j0, nx);
          if (r == 0) nxte[u + 1] = fr;
        }
#pragma unroll
        for (int jj = 0; jj < J; ++jj) xr[jj] = ract ? nx[jj] : xr[jj];
        const bool bok = bact && su > 0.f && !isinf(su);
#pragma unroll
        for (int ii = 0; ii < J; ++ii) beta[ii] = bok ? nb[ii] : beta[ii];
        D = bok ? Dn : D;
        sb = sb_cur;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
          bb[jj] = bbn[jj];
          br[jj] = brn[jj];
          a1[jj] = a0s[jj];
          a0[jj] = a0n[jj];
        }
        e1 = e0;
        e0 = e0n;
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
