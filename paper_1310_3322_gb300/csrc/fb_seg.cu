// fb_seg.cu -- forward-backward adjoint, FP32 SIMT, with the segments of one
// sequence processed in parallel (Sec. 2.7 "Baum-Welch", its E-step; Rabiner
// 1989 eqs. 19-21 forward, 24-25 backward, 37 xi, 38 gamma).
//
// The single-kernel adjoint (fb.cu) runs three dependent passes per pair --
// forward, then recompute and backward segment by segment -- so its time is
// set by the longest sequence's 2T + C dependent steps. Here:
//
//  * hmm_fb_pass: the forward recursion and the backward recursion of every
//    pair run as independent chains (beta needs no alpha), each on its own
//    group of lanes. The forward keeps alpha_t (and the power-of-two exponent
//    removed at t) every C steps, the log-likelihood and sum_j alpha_{T-1}(j);
//    the backward keeps beta_t every C steps, rescaled by exact powers of two.
//  * hmm_fb_seg: the C-step segments of a pair are split into `spar` ranges
//    of `spg` consecutive segments, each range an independent work item. A
//    range starts from the checkpoints at its end (alpha and beta of the next
//    segment's first step, or beta = 1 at the sequence's end) and walks its
//    segments backwards exactly like fb.cu's second phase (backward over
//    segment c while alpha is recomputed over segment c-1). Its counts go to
//    its own slot; the reduction sums the slots of all ranges in a fixed order.
//
// Per-step normalisation (fb.cu's identity): with u_{t+1} = b(o_{t+1}) beta_{t+1}
// and e_{t+1} the forward exponent removed at t+1,
//   Z_t = sum_j (alpha_t A)_j u_{t+1}(j) = 2^{e_{t+1}} D_{t+1},
//   D_{t+1} = sum_j alpha_{t+1}(j) beta_{t+1}(j),
// so every xi_t and gamma_t is normalised by quantities of steps t and t+1 only,
// whatever scale the stored beta checkpoint carries: the ranges are independent.
// A range counts gamma_t for t in [c_lo C, its end) and xi_t for the same t.
#include "fb_common.cuh"

namespace hmmgb {

template <int NP, int G>
struct FbSegLayout {
  static constexpr int J = NP / G;
  static constexpr int PP = 32 / G;
  static constexpr int XS = NP + 4;
  // floats per pair of the segment kernel, rounded to 4 (16-byte alignment)
  static __host__ __device__ int per_pair(int C, int M) {
    const int n = 4 * XS + 2 * C * NP + 2 * C + NP * (M + 1);
    return (n + 3) & ~3;
  }
};

// ---------------------------------------------------------------------------
// pass kernel: forward (dir 0) or backward (dir 1) recursion of PP pairs
// ---------------------------------------------------------------------------
template <int NP, int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) hmm_fb_pass(FbSegLaunch a) {
  constexpr int J = NP / G, PP = 32 / G, XS = NP + 4;
  __shared__ __align__(16) float xs[kWarpsPerBlock][PP][2][XS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / G, r = lane % G, j0 = r * J;
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;
  const int C = a.ckpt, NC = a.nck;
  const bool labelled = a.seq.model_of_seq != nullptr;

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_items_pass) break;
    const int pi_ = item >> 1, dir = item & 1;
    const int g = labelled ? pi_ : pi_ / K;
    int k = labelled ? 0 : pi_ % K;
    const int pos = g * PP + p;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    if (labelled && has && T >= 0) k = a.seq.model_of_seq[s];
    const size_t slot = labelled ? (size_t)s : (size_t)s * K + k;
    const int Tn = T < 0 ? 0 : T;
    const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
    const float* Bk = a.mod.Btp + (size_t)k * M * NP + j0;
    const int32_t* o = a.seq.symbols + ((has && T >= 0) ? a.seq.offsets[s] : 0);
    const int Tmax = __reduce_max_sync(HMM_FULL_MASK, Tn);
    float* cka = a.ckA + slot * (size_t)NC * NP + j0;
    float* ckb = a.ckB + slot * (size_t)NC * NP + j0;
    int32_t* cke = a.ckE + slot * (size_t)NC;

    if (dir == 0) {
      // ---------------- forward, alpha checkpoints every C steps ----------------
      float2 ac[NP / 2][J];  // ac[i2][jj] = (a_{2i2, j}, a_{2i2+1, j}),  j = j0 + jj
#pragma unroll
      for (int i2 = 0; i2 < NP / 2; ++i2)
#pragma unroll
        for (int jj = 0; jj < J; ++jj)
          ac[i2][jj] = make_float2(__ldg(Ak + (2 * i2) * NP + j0 + jj),
                                   __ldg(Ak + (2 * i2 + 1) * NP + j0 + jj));
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
          store_vec<J>(cka, x);
          if (r == 0) cke[0] = 0;
        }
      }
      // the steps of fb.cu's first phase: each step scales its result by the
      // exponent of its input row's sum (lane-local), e_{t+1} = f_t is kept
      // with the checkpoints, liveness by flags
      float bn[J];
      int on = (1 < Tn) ? __ldg(o + 1) : 0;
      bool symbad = (unsigned)on >= (unsigned)M;
      on = symbad ? 0 : on;
      load_vec<J>(bn, Bk + (size_t)on * NP);
      int o2 = (2 < Tn) ? __ldg(o + 2) : 0;
      int cls = 0;
      int cc = 0, ci = 0;
      for (int t = 1; t < Tmax; ++t) {
        const bool act = t < Tn;
        float* xw = &xs[warp][p][t & 1][0];
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
        cls |= act ? sum_class(sx) : 0;
        E += act ? f : 0;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) x[jj] = act ? nx[jj] : x[jj];
        if (act && cc == 0) {
          store_vec<J>(cka + (size_t)ci * NP, x);
          if (r == 0) cke[ci] = f;
        }
      }
      if (symbad) { bad = true; err |= HMM_STATUS_SYMBOL; }
      if (cls & 2) { bad = true; err |= HMM_STATUS_PARAM; }
      else if (cls & 1) dead = true;
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
        const float w = a.weight ? a.weight[slot] : 1.f;
        a.sig[slot] = fs;
        a.skip[slot] = (bad || dead || Tn == 0 || w == 0.f) ? 1 : 0;
      }
    } else {
      // ---------------- backward, beta checkpoints every C steps ----------------
      float2 ar[J][NP / 2];  // ar[ii][j2] = (a_{i, 2j2}, a_{i, 2j2+1}),  i = j0 + ii
#pragma unroll
      for (int ii = 0; ii < J; ++ii)
#pragma unroll
        for (int j2 = 0; j2 < NP / 2; ++j2)
          ar[ii][j2] = __ldg(reinterpret_cast<const float2*>(Ak + (j0 + ii) * NP) + j2);
      float beta[J];
#pragma unroll
      for (int jj = 0; jj < J; ++jj) beta[jj] = 1.f;
      if (has && Tn > 0 && (Tn - 1) % C == 0) store_vec<J>(ckb + (size_t)((Tn - 1) / C) * NP, beta);
      auto sym = [&](int t) -> int {
        if (t < 0 || t >= Tn) return 0;
        const int v = __ldg(o + t);
        return (unsigned)v < (unsigned)M ? v : 0;
      };
      // step u computes beta_t, t = Tn - 2 - u, from the symbol at t + 1
      int s_cur = sym(Tn - 1), s_nxt = sym(Tn - 2);
      bool live = true;
      for (int u = 0; u + 1 < Tmax; ++u) {
        const int t = Tn - 2 - u;
        const bool act = has && t >= 0 && live;
        float b[J];
        load_vec<J>(b, Bk + (size_t)s_cur * NP);
        s_cur = s_nxt;
        s_nxt = sym(t - 1);
        float v[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) v[jj] = b[jj] * beta[jj];
        float* vw = &xs[warp][p][u & 1][0];
        store_vec<J>(vw + j0, v);
        __syncwarp();
        // beta_t = A v scaled by the exponent of sum v (lane-local)
        float nb[J], su;
        rows_matvec_sum<NP, J>(vw, ar, nb, su);
        int g_;
        const float sg = pow2_scale(su, g_);
        // a zero, infinite or invalid row: the forward marks the pair skipped
        live = live && !(act && (!(su > 0.f) || isinf(su)));
#pragma unroll
        for (int jj = 0; jj < J; ++jj) beta[jj] = (act && live) ? nb[jj] * sg : beta[jj];
        if (act && live && t % C == 0) store_vec<J>(ckb + (size_t)(t / C) * NP, beta);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// segment kernel: one range of segments of PP pairs
// ---------------------------------------------------------------------------
template <int NP, int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) hmm_fb_seg(FbSegLaunch a) {
  using L = FbSegLayout<NP, G>;
  constexpr int J = L::J, PP = L::PP, XS = L::XS;
  extern __shared__ __align__(16) float smem[];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / G, r = lane % G, j0 = r * J;
  const int K = a.seq.K, M = a.seq.M, S = a.seq.S;
  const int C = a.ckpt, NC = a.nck, MP = M + 1;
  const bool labelled = a.seq.model_of_seq != nullptr;

  const int per = L::per_pair(C, M);
  float* base = smem + (size_t)(warp * PP + p) * per;
  float* xf = base;                                   // [2][XS] forward exchange
  float* xv = xf + 2 * XS;                            // [2][XS] backward exchange
  float* seg = xv + 2 * XS;                           // [2][C][NP] recomputed segments
  int* sege = reinterpret_cast<int*>(seg + 2 * C * NP);  // [2][C]
  float* cb = reinterpret_cast<float*>(sege + 2 * C);   // [NP][MP] emission counts

  for (int e = r; e < NP * MP; e += G) cb[e] = 0.f;
  __syncwarp();

  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue + 1, 1);
    item = __shfl_sync(HMM_FULL_MASK, item, 0);
    if (item >= a.n_items_seg) break;
    const int pi_ = item / a.spar, gi = item % a.spar;
    const int g = labelled ? pi_ : pi_ / K;
    int k = labelled ? 0 : pi_ % K;
    const int pos = g * PP + p;
    const bool has = pos < S;
    const int s = has ? a.seq.order[pos] : 0;
    const int T = has ? a.seq.seqlen[s] : 0;
    if (labelled && has && T >= 0) k = a.seq.model_of_seq[s];
    const size_t slot = labelled ? (size_t)s : (size_t)s * K + k;
    const float w = (has && a.weight) ? a.weight[slot] : 1.f;
    const bool alive = has && T > 0 && a.skip[slot] == 0;
    const int Tb = alive ? T : 0;
    const int TbMax = __reduce_max_sync(HMM_FULL_MASK, Tb);
    const int NCs = (Tb + C - 1) / C;
    const int c_lo = gi * a.spg;                        // the same for every pair of the warp
    const int c_hi = min(c_lo + a.spg, NCs) - 1;        // this pair's last segment of the range
    const bool act = alive && c_hi >= c_lo;
    const bool fin = act && c_hi == NCs - 1;            // the range reaches the sequence's end
    const int C_HI = __reduce_max_sync(HMM_FULL_MASK, act ? c_hi : -1);
    const float* cka = a.ckA + slot * (size_t)NC * NP + j0;
    const float* ckb = a.ckB + slot * (size_t)NC * NP + j0;
    const int32_t* cke = a.ckE + slot * (size_t)NC;
    const float* Bk = a.mod.Btp + (size_t)k * M * NP + j0;
    const int32_t* o = a.seq.symbols + ((has && T >= 0) ? a.seq.offsets[s] : 0);
    auto sym = [&](int t) -> int {
      if (!act || t < 0 || t >= Tb) return 0;
      const int v = __ldg(o + t);
      return (unsigned)v < (unsigned)M ? v : 0;
    };

    float2 xa[J][NP / 2];
#pragma unroll
    for (int ii = 0; ii < J; ++ii)
#pragma unroll
      for (int j2 = 0; j2 < NP / 2; ++j2) xa[ii][j2] = make_float2(0.f, 0.f);
    float cpi[J];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) cpi[jj] = 0.f;
    float2 ar[J][NP / 2];
    {
      const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
#pragma unroll
      for (int ii = 0; ii < J; ++ii)
#pragma unroll
        for (int j2 = 0; j2 < NP / 2; ++j2)
          ar[ii][j2] = __ldg(reinterpret_cast<const float2*>(Ak + (j0 + ii) * NP) + j2);
    }

    if (C_HI >= c_lo) {
      float2 ac[NP / 2][J];
      {
        const float* Ak = a.mod.Ap + (size_t)k * NP * NP;
#pragma unroll
        for (int i2 = 0; i2 < NP / 2; ++i2)
#pragma unroll
          for (int jj = 0; jj < J; ++jj)
            ac[i2][jj] = make_float2(__ldg(Ak + (2 * i2) * NP + j0 + jj),
                                     __ldg(Ak + (2 * i2 + 1) * NP + j0 + jj));
      }
      // state at the range's end: beta_{t1} and D_{t1} (or beta = 1, D = sum alpha_{T-1})
      float beta[J];
      float D;
      {
        float a1[J], b1[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) { a1[jj] = 0.f; b1[jj] = 1.f; }
        if (act && !fin) {
          load_vec<J>(a1, cka + (size_t)(c_hi + 1) * NP);
          load_vec<J>(b1, ckb + (size_t)(c_hi + 1) * NP);
        }
        float ad[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) { beta[jj] = b1[jj]; ad[jj] = a1[jj] * b1[jj]; }
        const float dd = group_sum<G>(tree_sum<J>(ad));
        D = fin ? a.sig[slot] : dd;
      }
      // the first step of a non-final range would count gamma of the next range
      const int t_skip = (act && !fin) ? (c_hi + 1) * C - 1 : -1;

      // prologue: recompute the range's last segment
      {
        const int c = C_HI, t0 = c * C, t1 = min(t0 + C, TbMax) - 1;
        float* sg = seg + (c & 1) * C * NP;
        int* se = sege + (c & 1) * C;
        float xr[J];
        load_vec<J>(xr, cka + (size_t)c * NP);
        store_vec<J>(sg + j0, xr);
        if (r == 0) se[0] = act ? cke[c] : 0;
        for (int t = t0 + 1; t <= t1; ++t) {
          const bool ra = act && c <= c_hi && t <= Tb - 1;
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
          if (ra) {
#pragma unroll
            for (int jj = 0; jj < J; ++jj) xr[jj] = nx[jj];
            store_vec<J>(sg + (t - t0) * NP + j0, xr);
            if (r == 0) se[t - t0] = f;
          }
        }
        __syncwarp();
      }

      for (int c = C_HI; c >= c_lo; --c) {
        const int t0 = c * C;
        const int t1 = min(t0 + C, TbMax) - 1;
        const float* cur = seg + (c & 1) * C * NP;
        const int* cure = sege + (c & 1) * C;
        float* nxt = seg + ((c + 1) & 1) * C * NP;  // segment c-1 (same parity as c+1)
        int* nxte = sege + ((c + 1) & 1) * C;
        const bool rc_on = c > c_lo;
        const int r0 = (c - 1) * C;
        float xr[J];
        if (rc_on) {
          load_vec<J>(xr, cka + (size_t)(c - 1) * NP);
          store_vec<J>(nxt + j0, xr);
          if (r == 0) nxte[0] = act ? cke[c - 1] : 0;
        } else {
#pragma unroll
          for (int jj = 0; jj < J; ++jj) xr[jj] = 0.f;
        }
        int sb = sym(t1 + 1);
        float bb[J];
        load_vec<J>(bb, Bk + (size_t)sb * NP);
        int sb_next = sym(t1);
        int sr_next = rc_on ? sym(r0 + 1) : 0;
        float br[J];
        load_vec<J>(br, Bk + (size_t)sr_next * NP);
        sr_next = rc_on ? sym(r0 + 2) : 0;

        // alpha rows and exponents of the backward steps, one iteration ahead
        // (fb.cu's second phase): a1 = alpha_{t+1}, e1 = e_{t+1} (the next
        // segment's checkpoint at the top), a0 = alpha_t, e0 = e_t; indices
        // clamped into the buffers, steps outside a pair's range masked
        float a1[J], a0[J];
        load_vec<J>(a1, cka + (size_t)min(c + 1, NC - 1) * NP);
        int e1 = act ? cke[min(c + 1, NC - 1)] : 0;
        load_vec_smem<J>(a0, cur + (t1 - t0) * NP + j0);
        int e0 = cure[t1 - t0];

        for (int u = 0; u < C; ++u) {
          const int tb = t1 - u;
          const bool bact = act && tb >= t0 && c <= c_hi && tb <= Tb - 2;
          const int tr = r0 + 1 + u;
          const bool ract = rc_on && act && u <= C - 2 && tr <= Tb - 1;

          // backward: publish u_{t+1} = b beta_{t+1} 2^-e_{t+1}, count
          // gamma_{t+1} (not at a range's top); branch-free
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
            if (bact && tb != t_skip) *cbp += gam;
            v[jj] = bact ? (bb[jj] * beta[jj]) * se1 : 0.f;
            aw[jj] = bact ? (w * a0[jj]) * invD : 0.f;
          }
          float a0s[J], a0m[J];
#pragma unroll
          for (int jj = 0; jj < J; ++jj) {
            a0s[jj] = a0[jj];
            a0m[jj] = bact ? a0[jj] : 0.f;
          }
          float* vw = xv + (u & 1) * XS;
          float* xw = xf + (u & 1) * XS;
          store_vec<J>(vw + j0, v);
          store_vec<J>(xw + j0, xr);
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

          // backward step: beta_t scaled by the exponent of sum u, and the xi
          // accumulator normalised by D_{t+1}
          float nb[J], su;
          rows_step_sum<NP, J>(vw, ar, aw, xa, nb, su);
          int fu;
          const float sgu = pow2_scale(su, fu);
          float ad[J];
#pragma unroll
          for (int ii = 0; ii < J; ++ii) {
            nb[ii] *= sgu;
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

      // gamma at the range's first step (and pi when it is t = 0)
      if (act) {
        const int R0 = c_lo * C;
        float a0[J];
        load_vec<J>(a0, cka + (size_t)c_lo * NP);
        const int oR = sym(R0);
        const float wd = w / D;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
          const float gv = wd * a0[jj] * beta[jj];
          cb[(j0 + jj) * MP + oR] += gv;
          if (R0 == 0) cpi[jj] = gv;
        }
      }
      __syncwarp();
    }

    // ---------------- this range's slot ----------------
    if (has) {
      float* out = a.partial + ((size_t)gi * a.npairs + slot) * a.slot_floats;
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

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
size_t fb_seg_smem_bytes(int NP, int G, int C, int M, int warps) {
  const int PP = 32 / G;
  const int XS = NP + 4;
  int n = 4 * XS + 2 * C * NP + 2 * C + NP * (M + 1);
  n = (n + 3) & ~3;
  return (size_t)warps * PP * n * sizeof(float);
}

template <int NP, int G>
static cudaError_t launch_fb_seg_t(const FbSegLaunch& a, int phase, cudaStream_t st) {
  if (phase == 0) {
    auto kern = hmm_fb_pass<NP, G>;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                    kWarpsPerBlock * 32, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int blocks = num_sms() * per_sm;
    const int need = (a.n_items_pass + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks > need) blocks = need > 0 ? need : 1;
    kern<<<blocks, kWarpsPerBlock * 32, 0, st>>>(a);
    return cudaGetLastError();
  }
  auto kern = hmm_fb_seg<NP, G>;
  int warps = kWarpsPerBlock;
  while (warps > 1 && fb_seg_smem_bytes(NP, G, a.ckpt, a.seq.M, warps) > 227 * 1024) warps >>= 1;
  const size_t smem = fb_seg_smem_bytes(NP, G, a.ckpt, a.seq.M, warps);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int blocks = num_sms() * per_sm;
  const int need = (a.n_items_seg + warps - 1) / warps;
  if (blocks > need) blocks = need > 0 ? need : 1;
  kern<<<blocks, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

#define HMM_FBS_CASE(NPV, GV) \
  if (NP == NPV && G == GV) return launch_fb_seg_t<NPV, GV>(a, phase, st);

cudaError_t launch_fb_seg(int NP, int G, const FbSegLaunch& a, int phase, cudaStream_t st) {
  HMM_FBS_CASE(4, 2) HMM_FBS_CASE(4, 4)
  HMM_FBS_CASE(8, 4) HMM_FBS_CASE(8, 8)
  HMM_FBS_CASE(16, 8) HMM_FBS_CASE(16, 16)
  HMM_FBS_CASE(32, 32)
  HMM_FBS_CASE(64, 32)
  return cudaErrorInvalidValue;
}

}  // namespace hmmgb
