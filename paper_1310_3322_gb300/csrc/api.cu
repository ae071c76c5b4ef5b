// api.cu -- the C-ABI of include/hmm.h: host-side argument checks, workspace
// layout, the autotuning table and the launch sequence of every entry point.
// Nothing here allocates device memory or synchronises (except
// hmm_get_device_status, whose job is to read the device status word).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "hmm_internal.cuh"

namespace hmmgb {

static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

static WsLayout make_layout(const hmm_dims_t& d, const hmm_seqs_t& q, int op, bool mma = false,
                            int scan_L = 0, bool tf32 = false);
// Workspace of hmm_forward without HMM_AUTO's parallel-in-time variant (the
// static entry point's scratch is sized for this; hmm_forward falls back to
// the sequential recursion when the scan's storage does not fit).
size_t forward_ws_sequential(const hmm_dims_t& d, const hmm_seqs_t& q) {
  return make_layout(d, q, HMM_OP_FORWARD, false, 0).total;
}

// Records an error message for hmm_last_error() (used by entry points that
// live in other translation units).
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(HMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static std::atomic<uint32_t> g_wait_limit{kDrainPolls};

uint32_t wait_limit_polls() { return g_wait_limit.load(std::memory_order_relaxed); }

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

// ---------------------------------------------------------------------------
// padded state counts and the tuning table
// ---------------------------------------------------------------------------
static const int kNPs[] = {4, 8, 16, 32, 64};
static int np_index(int NP) {
  for (int i = 0; i < 5; ++i)
    if (kNPs[i] == NP) return i;
  return -1;
}
// 4..64 for the SIMT kernels, 128 for the tensor-core forward and adjoint,
// 256 and 512 for the wide tensor-core forward
static int pad_states(int N) {
  for (int i = 0; i < 5; ++i)
    if (N <= kNPs[i]) return kNPs[i];
  if (N <= 128) return 128;
  if (N <= 256) return 256;
  return N <= 512 ? 512 : -1;
}

// candidate lanes-per-pair (ops 0-3) or segment ranges per pair of the SIMT
// adjoint (op 4, 1 = the single-kernel adjoint), default first; 0 terminates
constexpr int kTuneOps = 5;
static const int kCand[kTuneOps][5][5] = {
    /* forward */ {{1, 2, 4, 0}, {1, 2, 4, 8, 0}, {2, 4, 8, 16, 0}, {8, 16, 32, 0}, {32, 0}},
    /* viterbi scores */ {{1, 2, 4, 0}, {1, 2, 4, 8, 0}, {2, 4, 8, 16, 0}, {8, 16, 32, 0}, {32, 0}},
    /* fb      */ {{4, 2, 0}, {8, 4, 0}, {8, 16, 0}, {32, 0}, {32, 0}},
    /* viterbi paths */ {{4, 2, 1, 0}, {8, 4, 2, 0}, {8, 16, 4, 0}, {16, 32, 8, 0}, {32, 0}},
    /* fb ranges */ {{1, 2, 4, 8, 16}, {1, 2, 4, 8, 16}, {1, 2, 4, 8, 16}, {1, 2, 4, 8, 16},
                     {1, 2, 4, 8, 16}},
};
static int g_tuning[kTuneOps][5] = {{0}};
static std::mutex g_tuning_mu;

int candidates(int op, int NP, int* out, int cap) {
  const int ni = np_index(NP);
  if (op < 0 || op >= kTuneOps || ni < 0) return -1;
  int n = 0;
  for (int i = 0; i < 5 && kCand[op][ni][i]; ++i) {
    if (n < cap && out) out[n] = kCand[op][ni][i];
    ++n;
  }
  return n;
}

static int lanes_for(int op, int NP) {
  const int ni = np_index(NP);
  if (ni < 0) return 1;  // no SIMT kernel at this state count
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  const int v = g_tuning[op][ni];
  return v ? v : kCand[op][ni][0];
}

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int first_chunks(int S) {
  int n = (S + kReduceChunk - 1) / kReduceChunk;
  if (n > 1024) n = 1024;
  return n < 1 ? 1 : n;
}

static int ckpt_stride(int max_len) {
  int C = (int)ceil(sqrt((double)(max_len > 0 ? max_len : 1)));
  return C < 1 ? 1 : C;
}

// Checkpoint images per CTA of the tensor-core adjoint for tiles up to max_len.
static int fb_mma_nsmax(int max_len) {
  const int l1 = max_len < 8192 ? max_len : 8192;
  int ns = l1 > 0 ? (l1 + fb_mma_segment(l1) - 1) / fb_mma_segment(l1) : 1;
  const int big = (int)ceil(sqrt((double)(max_len > 0 ? max_len : 1))) + 1;
  if (max_len > 8192 && big > ns) ns = big;
  return ns < 1 ? 1 : ns;
}

// Checkpoint segments per range item of the tensor-core adjoint: enough
// items (about 12 per SM for the tiles the batch can have) that the ranges of
// the longest tiles spread over the GPU, at least two segments each so an
// item's fixed costs (its restart step, loading its model, writing its count
// slot) stay small against its steps.
static int fb_mma_spr(int nsmax, int tiles) {
  const int64_t want = (int64_t)12 * num_sms();
  int spr = (int)(((int64_t)nsmax * tiles + want - 1) / want);
  if (spr < 2) spr = 2;
  return spr > nsmax ? (nsmax > 0 ? nsmax : 1) : spr;
}

static int fb_mma_tile_cap(const hmm_dims_t& d, const hmm_seqs_t& q) {
  const int64_t chunks = ((int64_t)(q.S > 0 ? q.S : 0) + 127) / 128;
  const int64_t cap = q.model_of_seq ? chunks + d.K : chunks * d.K;
  return (int)(cap < 1 ? 1 : cap);
}

static int fb_mma_grid(const hmm_dims_t& d, int NP) {
  return num_sms() * fb_mma_ctas_per_sm(NP, d.M);
}

// Steps per chunk of the parallel-in-time forward (0 = automatic).
static int scan_chunk_len(int chunk, int max_len) {
  if (chunk > 0) return chunk;
  int L = (int)ceil(sqrt(2.0 * (max_len > 1 ? max_len : 1)));
  L = (L + 15) / 16 * 16;
  return L < kScanMaxChunk ? L : kScanMaxChunk;
}

// Chunk slots per model slot: enough for every sequence at max_len and for
// non-overlapping sequences within total_obs, whichever is fewer.
static int64_t scan_cap(const hmm_seqs_t& q, int L) {
  const int64_t S = q.S > 0 ? q.S : 0;
  const int64_t per = q.max_len > 1 ? ((int64_t)q.max_len - 1 + L - 1) / L : 0;
  const int64_t a1 = S * per;
  const int64_t a2 = (q.total_obs > 0 ? q.total_obs : 0) / L + S;
  const int64_t c = a1 < a2 ? a1 : a2;
  return c > 1 ? c : 1;
}

// HMM_AUTO's choice of the parallel-in-time forward: a batch whose pairs
// leave the GPU mostly idle, long enough that the T-step chain dominates, and
// small enough that the scan's N_pad^3 work per step stays below the chain's
// time (pairs * N_pad^3 <= 2^21: e.g. 64 pairs at 32 states, 512 at 16).
static bool scan_preferred(const hmm_dims_t& d, const hmm_seqs_t& q) {
  if (d.N > 32 || q.max_len < 4096 || q.S <= 0) return false;
  const int64_t span = q.model_of_seq ? 1 : (q.model_base ? q.model_span : d.K);
  const int64_t pairs = (int64_t)q.S * span;
  const int64_t NP = pad_states(d.N);
  return pairs * NP * NP * NP <= ((int64_t)1 << 21) && pairs <= (int64_t)num_sms() * 32;
}

// The TF32 adjoint's symbol range: the M <= 256 of the tensor-core adjoint
// (its passes' shared memory would take a few more).
static bool tf32_adjoint_m_ok(int NP, int M) { return M <= 256 && fb_tf32_supported(NP, M); }

// Emission-count buffers of the adjoint from per-step rows (fb_wide.cu).
static void emis_layout(WsLayout& L, size_t& off, const hmm_dims_t& d, int NP, int64_t nrows) {
  const FbwEmisSizes z = fbw_emis_sizes(d.K, d.M, NP, nrows);
  L.w_ech = z.ech;
  L.w_ncc = (int)z.ncc;
  L.w_ecb = off; off = align256(off + ((size_t)d.K + 1) * 4);
  L.w_eh = off; off = align256(off + (size_t)z.ehist * 4);
  L.w_eb = off; off = align256(off + (size_t)z.ebase * 4);
  L.w_epb = off; off = align256(off + (size_t)z.ebase * 4);
  L.w_el = off; off = align256(off + (size_t)z.elist * 4);
  L.w_ep = off; off = align256(off + (size_t)z.epart * 4);
}

static WsLayout make_layout(const hmm_dims_t& d, const hmm_seqs_t& q, int op, bool mma,
                            int scan_L, bool tf32) {
  WsLayout L;
  memset(&L, 0, sizeof(L));
  const int NP = pad_states(d.N);
  L.NP = NP;
  const size_t S = (size_t)(q.S > 0 ? q.S : 0);
  size_t off = sizeof(WsHeader);
  L.order = off; off = align256(off + S * 4);
  L.seqlen = off; off = align256(off + S * 4);
  L.done = off; off = align256(off + S * 4);
  {
    const size_t nb = (size_t)plan_blocks((int)S);
    L.phist = off; off = align256(off + nb * kLenBuckets * 4);
    L.punits = off; off = align256(off + 2 * nb * 8);
  }
  if (op == HMM_OP_VITERBI) {
    L.bpoff = off; off = align256(off + S * 8);
    L.best = off; off = align256(off + S * 4);
    if (NP > 64) {  // paths grouped by decoded model, segments padded to 4
      L.vgorder = off; off = align256(off + (S + 4 * ((size_t)d.K + 1)) * 4);
      L.vgcount = off; off = align256(off + 4);
    }
  }
  L.pip = off; off = align256(off + (size_t)d.K * NP * 4);
  L.Ap = off; off = align256(off + (size_t)d.K * NP * NP * 4);
  L.Btp = off; off = align256(off + (size_t)d.K * d.M * NP * 4);
  L.Btp16 = off; off = align256(off + (size_t)d.K * d.M * NP * 2);
  if (op == HMM_OP_VITERBI) {
    L.bp_cap = (q.total_obs > 0 ? q.total_obs : 0) * (int64_t)NP;
    L.bp = off; off = align256(off + (size_t)L.bp_cap);
  }
  if (op == HMM_OP_FORWARD && NP >= 256) {
    L.wimg = off; off = align256(off + (size_t)d.K * NP * NP * 2);
  }
  if (op == HMM_OP_FORWARD_SCAN) {
    const int64_t slots = (q.model_of_seq ? 1 : (q.model_base ? q.model_span : d.K));
    L.sc_cap = scan_cap(q, scan_L);
    L.sc_coff = off; off = align256(off + (S + 1) * 8);
    L.sc_P = off; off = align256(off + (size_t)(slots * L.sc_cap) * NP * NP * 4);
    L.sc_E = off; off = align256(off + (size_t)(slots * L.sc_cap) * NP * 4);
  }
  if (op == HMM_OP_FORWARD_BACKWARD && !mma) {
    L.slot_floats = (int64_t)NP + (int64_t)NP * NP + (int64_t)NP * d.M;
    L.slots = q.model_of_seq ? (int64_t)S : (int64_t)S * d.K;
    // segment ranges: checkpoints of alpha and beta, one slot per range
    const int C = ckpt_stride(q.max_len);
    const int NC = (q.max_len > 0 ? (q.max_len - 1) / C : 0) + 1;
    const int want = lanes_for(HMM_TUNE_FB_RANGES, NP);  // the current tuning
    L.s_planes = NC < want ? NC : want;
    L.nchunks = first_chunks((int)(S * L.s_planes));
    L.s_ckA = off; off = align256(off + (size_t)L.slots * NC * NP * 4);
    L.s_ckB = off; off = align256(off + (size_t)L.slots * NC * NP * 4);
    L.s_ckE = off; off = align256(off + (size_t)L.slots * NC * 4);
    L.s_sig = off; off = align256(off + (size_t)L.slots * 4);
    L.s_skip = off; off = align256(off + (size_t)L.slots * 4);
    L.partial = off; off = align256(off + (size_t)(L.slots * L.s_planes * L.slot_floats * 4));
    L.red1 = off; off = align256(off + (size_t)L.nchunks * d.K * L.slot_floats * 4);
  }
  if (op == HMM_OP_FORWARD_BACKWARD && mma && NP >= 256) {
    // adjoint above 128 states: per-step rows of both passes, count partials
    const int64_t rtot = q.total_obs > 0 ? q.total_obs : 1;
    const int64_t slots = d.K;
    L.w_rtot = rtot;
    L.bpoff = off; off = align256(off + S * 8);
    const size_t rowb = (size_t)(slots * rtot) * NP * 4;
    L.w_X = off; off = align256(off + rowb);
    L.w_Bh = off; off = align256(off + rowb);
    L.w_V = off; off = align256(off + rowb);
    L.w_G = off; off = align256(off + rowb);
    L.w_xe = off; off = align256(off + (size_t)(slots * rtot) * 4);
    L.w_sym = off; off = align256(off + (size_t)(slots * rtot) * 4);
    const int tiles = (NP / 128) * (NP / 256);  // output tiles of the count contraction
    int ns = (2 * num_sms() + tiles * d.K - 1) / (tiles * d.K);
    L.w_nsplit = ns < 1 ? 1 : (ns > 64 ? 64 : ns);
    L.w_Cp = off; off = align256(off + (size_t)slots * L.w_nsplit * NP * NP * 4);
    emis_layout(L, off, d, NP, slots * rtot);
  } else if (op == HMM_OP_FORWARD_BACKWARD && mma && tf32) {
    // TF32 adjoint (N_pad = 128): the tile plan with one tile per pass group,
    // then every step's rows (model blocks of rtot rows unless labelled), row
    // offsets and the count partials of fb_wide.cu
    const int cap = fb_mma_tile_cap(d, q);
    const int max_len = q.max_len > 0 ? q.max_len : 1;
    const int nsmax = fb_mma_nsmax(max_len);
    const int64_t rtot = q.total_obs > 0 ? q.total_obs : 1;
    const int64_t nrows = q.model_of_seq ? rtot : rtot * d.K;
    L.m_group = 1;
    L.m_spr = fb_mma_spr(nsmax, cap);
    L.m_pass_cap = cap;
    L.m_rng_cap = cap * ((nsmax + L.m_spr - 1) / L.m_spr);
    L.w_rtot = rtot;
    L.m_sorted = off; off = align256(off + S * 4);
    L.m_tmp = off; off = align256(off + S * 4);
    L.m_keys = off; off = align256(off + 2 * (size_t)std::max<int64_t>(S, cap) * 4);
    L.m_tiles = off; off = align256(off + ((size_t)cap * 6 + (size_t)d.K * 2) * 4);
    L.m_ntiles = off; off = align256(off + 4);
    L.m_pscr = off; off = align256(off + mma_plan_scratch_bytes((int64_t)S));
    L.m_pass = off; off = align256(off + (size_t)cap * 4);
    L.m_ptmp = off; off = align256(off + (size_t)cap * 2 * 4);
    L.m_npass = off; off = align256(off + 4);
    L.m_rtile = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_rseg = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_rmodel = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_rlen = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_nrng = off; off = align256(off + 4);
    const size_t rowb = (size_t)nrows * NP * 4;
    L.w_X = off; off = align256(off + rowb);
    L.w_Bh = off; off = align256(off + rowb);
    L.w_V = off; off = align256(off + rowb);
    L.w_G = off; off = align256(off + rowb);
    L.w_xe = off; off = align256(off + (size_t)nrows * 4);
    L.w_sym = off; off = align256(off + (size_t)nrows * 4);
    L.bpoff = off; off = align256(off + S * 8);                    // rp: first row per sequence
    L.t_pos = off; off = align256(off + S * 8);                    // first row per plan position
    L.t_mrow = off; off = align256(off + 2 * ((size_t)d.K + 1) * 8);  // model row ranges
    L.t_rpos = off; off = align256(off + (size_t)rtot * 4);           // position of each row
    int ns = (num_sms() + d.K - 1) / d.K;  // the contraction runs one CTA per SM
    L.w_nsplit = ns < 1 ? 1 : (ns > 64 ? 64 : ns);
    L.w_Cp = off; off = align256(off + (size_t)d.K * L.w_nsplit * NP * NP * 4);
    emis_layout(L, off, d, NP, nrows);
  } else if (op == HMM_OP_FORWARD_BACKWARD && mma) {
    // tensor-core adjoint: tile plan and work lists; per tile the pass
    // kernel's checkpoints (alpha and Y images, exponents, last row sums);
    // per range item a count slot; per CTA of the range kernel its buffers
    const int cap = fb_mma_tile_cap(d, q);
    const size_t img = (size_t)128 * NP * 2;
    const int max_len = q.max_len > 0 ? q.max_len : 1;
    const int nsmax = fb_mma_nsmax(max_len);
    L.m_group = fb_pass_tiles_per_cta(NP, cap);
    L.m_spr = fb_mma_spr(nsmax, cap);
    L.m_pass_cap = cap;
    L.m_rng_cap = cap * ((nsmax + L.m_spr - 1) / L.m_spr);
    L.slot_floats = (int64_t)NP + (int64_t)NP * NP + (int64_t)NP * d.M;
    L.slots = L.m_rng_cap;
    L.nchunks = first_chunks(L.m_rng_cap);
    L.m_sorted = off; off = align256(off + S * 4);
    L.m_tmp = off; off = align256(off + S * 4);
    L.m_keys = off; off = align256(off + 2 * (size_t)std::max<int64_t>(S, cap) * 4);
    L.m_tiles = off; off = align256(off + ((size_t)cap * 6 + (size_t)d.K * 2) * 4);
    L.m_ntiles = off; off = align256(off + 4);
    L.m_pscr = off; off = align256(off + mma_plan_scratch_bytes((int64_t)S));
    L.m_pass = off; off = align256(off + (size_t)cap * L.m_group * 4);
    L.m_ptmp = off; off = align256(off + (size_t)cap * 2 * 4);
    L.m_npass = off; off = align256(off + 4);
    L.m_rtile = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_rseg = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_rmodel = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_rlen = off; off = align256(off + (size_t)L.m_rng_cap * 4);
    L.m_nrng = off; off = align256(off + 4);
    L.partial = off; off = align256(off + (size_t)(L.slots * L.slot_floats * 4));
    L.red1 = off; off = align256(off + (size_t)L.nchunks * d.K * L.slot_floats * 4);
    L.m_ckpt_bytes = (int64_t)nsmax * img;
    L.m_gexp_bytes = (int64_t)align256((size_t)max_len * 128);
    L.m_ckpt = off; off = align256(off + (size_t)cap * L.m_ckpt_bytes);
    L.m_cky = off; off = align256(off + (size_t)cap * L.m_ckpt_bytes);
    L.m_gexp = off; off = align256(off + (size_t)cap * L.m_gexp_bytes);
    L.m_slast = off; off = align256(off + (size_t)cap * 128 * 4);
    const int grid = fb_mma_grid(d, NP);
    L.m_grid = grid;
    L.m_scr_bytes = (int64_t)fb_mma_segment(max_len) * img;
    L.m_scr = off; off = align256(off + (size_t)grid * L.m_scr_bytes);
    L.m_gbuf = off; off = align256(off + (size_t)grid * 128 * NP * 4);
    L.m_psum = off; off = align256(off + (size_t)grid * 2 * 4 * 128 * 4);
  }
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static bool al(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

static int check_dims(const hmm_dims_t& d, int max_n) {
  if (d.K < 1 || d.N < 1 || d.M < 1)
    return fail(HMM_ERR_ARG, "dims must be positive (K=%d N=%d M=%d)", d.K, d.N, d.M);
  if (d.N > max_n)
    return fail(HMM_ERR_UNSUPPORTED, "N=%d above the largest supported state count %d", d.N, max_n);
  if (d.M > (1 << 24)) return fail(HMM_ERR_ARG, "M=%d too large", d.M);
  if ((int64_t)d.K * d.M * 64 > ((int64_t)1 << 31))
    return fail(HMM_ERR_ARG, "K*M too large (K=%d M=%d)", d.K, d.M);
  return HMM_OK;
}

static int check_seqs(const hmm_seqs_t* q, const hmm_dims_t& d) {
  if (!q) return fail(HMM_ERR_ARG, "seqs is NULL");
  if (q->S < 0 || q->max_len < 0 || q->total_obs < 0)
    return fail(HMM_ERR_ARG, "negative S, max_len or total_obs");
  if ((int64_t)q->S * d.K > ((int64_t)1 << 30))
    return fail(HMM_ERR_ARG, "S*K too large (S=%d K=%d)", q->S, d.K);
  if (q->S > 0) {
    if (!q->offsets || !q->lengths) return fail(HMM_ERR_ARG, "offsets/lengths NULL");
    if (!al(q->offsets, 8) || !al(q->lengths, 4) || (q->model_of_seq && !al(q->model_of_seq, 4)))
      return fail(HMM_ERR_ARG, "misaligned offsets/lengths/model_of_seq");
    if (q->total_obs > 0 && (!q->symbols || !al(q->symbols, 4)))
      return fail(HMM_ERR_ARG, "symbols NULL or misaligned");
  }
  if (q->model_base) {
    if (q->model_of_seq) return fail(HMM_ERR_ARG, "model_of_seq and model_base both set");
    if (q->model_span < 1 || q->model_span > d.K)
      return fail(HMM_ERR_ARG, "model_span %d outside [1, K=%d]", q->model_span, d.K);
    if (!al(q->model_base, 4)) return fail(HMM_ERR_ARG, "misaligned model_base");
  }
  return HMM_OK;
}

// Models each sequence is scored against in all-models mode.
static int span_of(const hmm_seqs_t& q, const hmm_dims_t& d) {
  return q.model_base ? q.model_span : d.K;
}

static int check_params(const float* pi, const float* A, const float* B) {
  if (!pi || !A || !B) return fail(HMM_ERR_ARG, "pi/A/B NULL");
  if (!al(pi, 4) || !al(A, 4) || !al(B, 4)) return fail(HMM_ERR_ARG, "pi/A/B misaligned");
  return HMM_OK;
}

static int check_ws(void* ws, size_t bytes, const WsLayout& L) {
  if (!ws) return fail(HMM_ERR_WORKSPACE, "workspace is NULL");
  if (!al(ws, 256)) return fail(HMM_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (bytes < L.total)
    return fail(HMM_ERR_WORKSPACE, "workspace %zu bytes, need %zu", bytes, L.total);
  return HMM_OK;
}

template <typename T>
static T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(reinterpret_cast<char*>(ws) + off);
}

static SetupArgs setup_args(const hmm_dims_t& d, const hmm_seqs_t& q, const WsLayout& L,
                            void* ws, const float* pi, const float* A, const float* B,
                            int log_mode) {
  SetupArgs s;
  memset(&s, 0, sizeof(s));
  s.phist = at<int32_t>(ws, L.phist);
  s.punits = at<int64_t>(ws, L.punits);
  s.K = d.K; s.N = d.N; s.M = d.M; s.NP = L.NP; s.S = q.S;
  s.total_obs = q.total_obs;
  s.max_len = q.max_len;
  s.log_mode = log_mode;
  s.pi = pi; s.A = A; s.B = B;
  s.lengths = q.lengths; s.offsets = q.offsets; s.model_of_seq = q.model_of_seq;
  s.model_base = q.model_base; s.span = span_of(q, d);
  s.pip = at<float>(ws, L.pip); s.Ap = at<float>(ws, L.Ap); s.Btp = at<float>(ws, L.Btp);
  s.Btp16 = at<uint16_t>(ws, L.Btp16);
  s.seqlen = at<int32_t>(ws, L.seqlen);
  s.order = at<int32_t>(ws, L.order);
  s.done = at<int32_t>(ws, L.done);
  s.status = &at<WsHeader>(ws, 0)->status;
  return s;
}

static SeqArgs seq_args(const hmm_dims_t& d, const hmm_seqs_t& q, const WsLayout& L, void* ws) {
  SeqArgs a;
  a.symbols = q.symbols;
  a.offsets = q.offsets;
  a.model_of_seq = q.model_of_seq;
  a.model_base = q.model_base;
  a.span = span_of(q, d);
  a.seqlen = at<int32_t>(ws, L.seqlen);
  a.order = at<int32_t>(ws, L.order);
  a.S = q.S; a.K = d.K; a.M = d.M; a.N = d.N;
  return a;
}

static ModelArgs model_args(const WsLayout& L, void* ws) {
  ModelArgs m;
  m.pip = at<float>(ws, L.pip);
  m.Ap = at<float>(ws, L.Ap);
  m.Btp = at<float>(ws, L.Btp);
  m.Btp16 = at<uint16_t>(ws, L.Btp16);
  return m;
}

static int max_states(int op, int precision) {
  if (op == HMM_OP_VITERBI) return (precision == HMM_FP32 || precision == HMM_AUTO) ? 128 : 0;
  if (op == HMM_OP_FORWARD_BACKWARD && (precision == HMM_BF16_MMA || precision == HMM_AUTO))
    return 512;
  if (op == HMM_OP_FORWARD_SCAN) return (precision == HMM_FP32 || precision == HMM_AUTO) ? 32 : 0;
  if (op == HMM_OP_FORWARD && (precision == HMM_BF16_MMA || precision == HMM_AUTO)) return 512;
  if ((op == HMM_OP_FORWARD || op == HMM_OP_FORWARD_BACKWARD) && precision == HMM_TF32_MMA) return 128;
  if (precision != HMM_FP32 && precision != HMM_AUTO) return 0;
  return 64;
}

static int check_precision(int precision, int op) {
  if (precision == HMM_FP32 || precision == HMM_AUTO) return HMM_OK;
  if (precision == HMM_BF16_MMA && (op == HMM_OP_FORWARD || op == HMM_OP_FORWARD_BACKWARD))
    return HMM_OK;
  if (precision == HMM_TF32_MMA && (op == HMM_OP_FORWARD || op == HMM_OP_FORWARD_BACKWARD))
    return HMM_OK;
  if (precision == HMM_BF16_MMA || precision == HMM_TF32_MMA)
    return fail(HMM_ERR_UNSUPPORTED, "tensor-core precision %d not available for op %d in this build",
                precision, op);
  return fail(HMM_ERR_ARG, "unknown precision %d", precision);
}

// Tensor-core forward: N in (32, 128], every sequence against every model.
static bool use_mma_forward(const hmm_dims_t& d, int precision) {
  return precision == HMM_BF16_MMA || precision == HMM_TF32_MMA ||
         (precision == HMM_AUTO && d.N > 64);
}

// Tensor-core adjoint: N in (32, 128]; the library's choice above N = 32
// (the FP32 SIMT adjoint holds a whole N = 64 pair in one warp's registers
// and spills there).
static bool use_mma_fb(const hmm_dims_t& d, int precision) {
  return precision == HMM_BF16_MMA || (precision == HMM_AUTO && d.N > 32);
}

// ---------------------------------------------------------------------------
// kernel timing (host-side tracing with CUDA events)
// ---------------------------------------------------------------------------
enum {
  T_SETUP = 0, T_FORWARD, T_VSCORES, T_VPATHS, T_FB, T_REDUCE, T_SOFTMAX, T_SGRAD, T_ADAM, T_MSTEP,
  T_SCAN_CHUNKS, T_SCAN_COMBINE, T_FB_PASS
};

struct EventPair {
  cudaEvent_t a, b;
};

static struct {
  bool on = false;
  std::vector<EventPair> rec[HMM_TIMING_KINDS];
  std::vector<EventPair> pool;
  std::mutex mu;
} g_timing;

// Records the start event of a timed launch (no-op while timing is off).
struct Timed {
  int kind;
  cudaStream_t st;
  EventPair ev{nullptr, nullptr};
  Timed(int k, cudaStream_t s) : kind(k), st(s) {
    if (!g_timing.on) return;
    std::lock_guard<std::mutex> lk(g_timing.mu);
    if (!g_timing.pool.empty()) {
      ev = g_timing.pool.back();
      g_timing.pool.pop_back();
    } else if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) {
      ev = EventPair{nullptr, nullptr};
      return;
    }
    cudaEventRecord(ev.a, st);
  }
  void stop() {
    if (!ev.a) return;
    cudaEventRecord(ev.b, st);
    std::lock_guard<std::mutex> lk(g_timing.mu);
    g_timing.rec[kind].push_back(ev);
    ev = EventPair{nullptr, nullptr};
  }
};

static int zero_counts(const hmm_dims_t& d, float* cnt_pi, float* cnt_A, float* cnt_B,
                       cudaStream_t st) {
  const size_t n = (size_t)d.K * d.N;
  cudaError_t e;
  if ((e = cudaMemsetAsync(cnt_pi, 0, n * 4, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(cnt_A, 0, n * d.N * 4, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(cnt_B, 0, n * d.M * 4, st)) != cudaSuccess)
    return cuda_fail(e, "memset");
  return HMM_OK;
}

static void emis_args(FbWideArgs& c, const WsLayout& L, void* ws) {
  c.cbase = at<int32_t>(ws, L.w_ecb);
  c.ehist = at<int32_t>(ws, L.w_eh);
  c.ebase = at<int32_t>(ws, L.w_eb);
  c.epbase = at<int32_t>(ws, L.w_epb);
  c.elist = at<int32_t>(ws, L.w_el);
  c.epart = at<float>(ws, L.w_ep);
  c.ncc = L.w_ncc;
  c.ech = L.w_ech;
}

// hmm_forward_backward above 128 states (arguments already checked except the
// workspace): setup, the tensor-core forward and backward passes keeping their
// per-step rows, then the count kernels of fb_wide.cu.
static int fb_wide(const hmm_dims_t& dims, const hmm_seqs_t* seqs, const float* weight,
                   float* loglik, float* cnt_pi, float* cnt_A, float* cnt_B, void* ws,
                   size_t ws_bytes, hmm_stream_t stream, const float* pi, const float* A,
                   const float* B) {
  const bool labelled = seqs->model_of_seq != nullptr;
  if (labelled && dims.K != 1)
    return fail(HMM_ERR_UNSUPPORTED,
                "above 128 states the adjoint scores every sequence against every model "
                "(model_of_seq only with K = 1)");
  const int NP = pad_states(dims.N);
  if (!forward_cluster_fits(NP, dims.M))
    return fail(HMM_ERR_UNSUPPORTED, "adjoint above 128 states: M=%d too large", dims.M);
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_FORWARD_BACKWARD, true);
  int rc = check_ws(ws, ws_bytes, L);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (seqs->S == 0) return zero_counts(dims, cnt_pi, cnt_A, cnt_B, st);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
  s.bf16_b = 1;  // BF16 path: B rounded to BF16 like A
  s.want_bpoff = 1;
  s.bpoff = at<int64_t>(ws, L.bpoff);
  s.bp_cap_rows = L.w_rtot;
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");
  const int rows = cluster_tile_rows(NP, seqs->S, dims.K, 2);
  const int n_tiles = (seqs->S + rows - 1) / rows;
  MmaWideLaunch f;
  memset(&f, 0, sizeof(f));
  f.seq = seq_args(dims, *seqs, L, ws);
  f.mod = model_args(L, ws);
  f.loglik = loglik;
  f.done = at<int32_t>(ws, L.done);
  f.queue = &at<WsHeader>(ws, 0)->queue[0];
  f.status = &at<WsHeader>(ws, 0)->status;
  f.n_tiles = n_tiles;
  f.rows = rows;
  f.n_items = n_tiles * dims.K;
  f.xs = at<float>(ws, L.w_X);
  f.roff = at<int64_t>(ws, L.bpoff);
  f.rtot = L.w_rtot;
  f.wait_limit = wait_limit_polls();
  // the backward pass: own row buffers
  MmaWideLaunch b = f;
  b.xs = at<float>(ws, L.w_Bh);
  b.xe = at<int32_t>(ws, L.w_xe);
  b.loglik = nullptr;
  {
    Timed tm(T_FB, st);
    e = launch_cluster_passes(NP, f, b, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core forward/backward launch");
  FbWideArgs c;
  memset(&c, 0, sizeof(c));
  c.K = dims.K; c.N = dims.N; c.M = dims.M; c.NP = NP; c.S = seqs->S;
  c.labelled = labelled ? 1 : 0;
  c.rtot = L.w_rtot;
  c.X = at<float>(ws, L.w_X);
  c.Bh = at<float>(ws, L.w_Bh);
  c.V = at<float>(ws, L.w_V);
  c.G = at<float>(ws, L.w_G);
  c.xe = at<int32_t>(ws, L.w_xe);
  c.sym = at<int32_t>(ws, L.w_sym);
  c.roff = at<int64_t>(ws, L.bpoff);
  c.seqlen = at<int32_t>(ws, L.seqlen);
  c.offsets = seqs->offsets;
  c.symbols = seqs->symbols;
  c.Btp = at<float>(ws, L.Btp);
  c.weight = weight;
  c.A = A;
  c.Cp = at<float>(ws, L.w_Cp);
  c.nsplit = L.w_nsplit;
  emis_args(c, L, ws);
  c.nrows = (int64_t)dims.K * L.w_rtot;
  c.u_in_x = 1;  // rows of invalid sequences are never written: U replaces X
  c.cnt_pi = cnt_pi;
  c.cnt_A = cnt_A;
  c.cnt_B = cnt_B;
  c.status = &at<WsHeader>(ws, 0)->status;
  {
    Timed tm(T_REDUCE, st);
    e = launch_fbw_counts(c, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint count launch");
  return HMM_OK;
}

// hmm_forward_backward on the tensor cores (arguments already checked except
// the workspace): setup, tile plan, adjoint, fixed-order reduction.
static int fb_mma(const hmm_dims_t& dims, const hmm_seqs_t* seqs, const float* weight,
                  float* loglik, float* cnt_pi, float* cnt_A, float* cnt_B, void* ws,
                  size_t ws_bytes, hmm_stream_t stream, const float* pi, const float* A,
                  const float* B) {
  const int NP = pad_states(dims.N);
  if (!fb_mma_supported(NP, dims.M))
    return fail(HMM_ERR_UNSUPPORTED, "tensor-core adjoint supports M <= 256 (M=%d)", dims.M);
  if (seqs->model_of_seq && dims.K > 65536)
    return fail(HMM_ERR_UNSUPPORTED, "tensor-core adjoint supports K <= 65536 labelled models");
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_FORWARD_BACKWARD, true);
  int rc;
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (seqs->S == 0) return zero_counts(dims, cnt_pi, cnt_A, cnt_B, st);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
  s.bf16_b = 1;      // BF16 path: B rounded to BF16 like A
  s.skip_order = 1;  // the tile plan orders the sequences itself
  const bool labelled = seqs->model_of_seq != nullptr;
  const int cap = L.m_pass_cap;  // tiles the plan can form
  int32_t* tiles = at<int32_t>(ws, L.m_tiles);
  MmaPlanArgs p;
  memset(&p, 0, sizeof(p));
  p.S = seqs->S; p.K = dims.K; p.labelled = labelled ? 1 : 0;
  p.seqlen = at<int32_t>(ws, L.seqlen);
  p.model_of_seq = seqs->model_of_seq;
  p.loglik = loglik;
  p.sorted = at<int32_t>(ws, L.m_sorted);
  p.tmp = at<int32_t>(ws, L.m_tmp);
  p.key = at<uint32_t>(ws, L.m_keys);
  p.key_tmp = p.key + std::max<int64_t>(seqs->S, (int64_t)cap);
  p.tile_start = tiles; p.tile_rows = tiles + cap; p.tile_model = tiles + 2 * cap;
  p.tile_len = tiles + 3 * cap; p.tile_order = tiles + 4 * cap; p.tile_tmp = tiles + 5 * cap;
  p.group_start = tiles + 6 * cap; p.group_end = p.group_start + dims.K;
  p.n_tiles_cap = cap;
  p.n_tiles = at<int32_t>(ws, L.m_ntiles);
  p.group = L.m_group;
  p.spr = L.m_spr;
  p.pass_tiles = at<int32_t>(ws, L.m_pass);
  p.pass_tmp = at<int32_t>(ws, L.m_ptmp);
  p.n_pass = at<int32_t>(ws, L.m_npass);
  p.pass_cap = L.m_pass_cap;
  p.rng_tile = at<int32_t>(ws, L.m_rtile);
  p.rng_seg = at<int32_t>(ws, L.m_rseg);
  p.rng_model = at<int32_t>(ws, L.m_rmodel);
  p.rng_len = at<int32_t>(ws, L.m_rlen);
  p.n_rng = at<int32_t>(ws, L.m_nrng);
  p.rng_cap = L.m_rng_cap;
  {
    const int nb = (int)((seqs->S + 4095) / 4096 > 0 ? (seqs->S + 4095) / 4096 : 1);
    p.bcnt = at<int32_t>(ws, L.m_pscr);
    p.hist = p.bcnt + nb;
    p.n_valid = p.hist + 256 * nb;
  }
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    if (e == cudaSuccess) e = launch_mma_plan(p, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");

  MmaPassLaunch pa;
  memset(&pa, 0, sizeof(pa));
  pa.seq = seq_args(dims, *seqs, L, ws);
  pa.mod = model_args(L, ws);
  pa.sorted = p.sorted;
  pa.tile_start = p.tile_start; pa.tile_rows = p.tile_rows; pa.tile_model = p.tile_model;
  pa.tile_len = p.tile_len;
  pa.pass_tiles = p.pass_tiles;
  pa.n_pass = p.n_pass;
  pa.labelled = p.labelled;
  pa.loglik = loglik;
  pa.ckx = at<uint8_t>(ws, L.m_ckpt);
  pa.cky = at<uint8_t>(ws, L.m_cky);
  pa.ck_stride = L.m_ckpt_bytes;
  pa.gexp = at<int8_t>(ws, L.m_gexp);
  pa.gexp_stride = L.m_gexp_bytes;
  pa.s_last = at<float>(ws, L.m_slast);
  pa.queue = &at<WsHeader>(ws, 0)->queue[5];
  pa.status = &at<WsHeader>(ws, 0)->status;
  pa.wait_limit = wait_limit_polls();
  {
    Timed tm(T_FB_PASS, st);
    e = launch_fb_pass(NP, L.m_group, pa, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core adjoint pass launch");

  MmaFbLaunch f;
  memset(&f, 0, sizeof(f));
  f.seq = pa.seq;
  f.mod = pa.mod;
  f.weight = weight;
  f.sorted = p.sorted;
  f.tile_start = p.tile_start; f.tile_rows = p.tile_rows; f.tile_model = p.tile_model;
  f.tile_len = p.tile_len;
  f.rng_tile = p.rng_tile; f.rng_seg = p.rng_seg; f.n_rng = p.n_rng;
  f.labelled = p.labelled;
  f.slots = at<float>(ws, L.partial);
  f.slot_floats = L.slot_floats;
  f.ckx = pa.ckx; f.cky = pa.cky; f.ck_stride = pa.ck_stride;
  f.gexp = pa.gexp; f.gexp_stride = pa.gexp_stride;
  f.s_last = pa.s_last;
  f.scr = at<uint8_t>(ws, L.m_scr);
  f.gbuf = at<float>(ws, L.m_gbuf);
  f.psum = at<float>(ws, L.m_psum);
  f.scr_bytes = L.m_scr_bytes;
  f.queue = &at<WsHeader>(ws, 0)->queue[3];
  f.status = &at<WsHeader>(ws, 0)->status;
  f.wait_limit = wait_limit_polls();
  {
    Timed tm(T_FB, st);
    e = launch_fb_mma(NP, dims.M, L.m_grid, f, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core adjoint launch");

  ReduceLaunch r;
  r.partial = f.slots;
  r.red1 = at<float>(ws, L.red1);
  r.model_of_seq = p.rng_model;   // every slot is one range of one tile of one model
  r.seqlen = p.rng_len;           // -1 marks unused slots
  r.S = L.m_rng_cap; r.K = dims.K; r.N = dims.N; r.M = dims.M; r.NP = NP;
  r.planes = 1;
  r.slot_floats = L.slot_floats;
  r.nchunks = L.nchunks;
  r.cnt_pi = cnt_pi; r.cnt_A = cnt_A; r.cnt_B = cnt_B;
  {
    Timed tm(T_REDUCE, st);
    e = launch_reduce(r, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
  return HMM_OK;
}

}  // namespace hmmgb

using namespace hmmgb;

extern "C" {

const char* hmm_last_error(void) { return g_err; }

int hmm_max_states(hmm_op_t op, hmm_precision_t precision) {
  if (op < HMM_OP_FORWARD || op > HMM_OP_FORWARD_SCAN) return fail(HMM_ERR_ARG, "bad op");
  return max_states(op, precision);
}

int hmm_workspace_size(hmm_dims_t dims, const hmm_seqs_t* seqs, hmm_op_t op, size_t* bytes) {
  g_err[0] = 0;
  if (!bytes) return fail(HMM_ERR_ARG, "bytes is NULL");
  if (op < HMM_OP_FORWARD || op > HMM_OP_FORWARD_SCAN) return fail(HMM_ERR_ARG, "bad op %d", op);
  if (op == HMM_OP_FORWARD_SCAN) return hmm_forward_scan_workspace_size(dims, seqs, 0, bytes);
  int rc = check_dims(dims, max_states(op, HMM_AUTO));
  if (rc) return rc;
  if (!seqs) return fail(HMM_ERR_ARG, "seqs is NULL");
  if (seqs->S < 0 || seqs->total_obs < 0) return fail(HMM_ERR_ARG, "negative S or total_obs");
  size_t need = 0;
  if (op != HMM_OP_FORWARD_BACKWARD || dims.N <= 64) need = make_layout(dims, *seqs, op).total;
  if (op == HMM_OP_FORWARD && scan_preferred(dims, *seqs)) {  // room for HMM_AUTO's scan
    const size_t sc = make_layout(dims, *seqs, HMM_OP_FORWARD_SCAN, false,
                                  scan_chunk_len(0, seqs->max_len)).total;
    if (sc > need) need = sc;
  }
  if (op == HMM_OP_FORWARD_BACKWARD && dims.N > 32) {
    if (pad_states(dims.N) >= 256) {
      if (!forward_cluster_fits(pad_states(dims.N), dims.M))
        return fail(HMM_ERR_UNSUPPORTED, "adjoint above 128 states: M=%d too large", dims.M);
    } else if (!fb_mma_supported(pad_states(dims.N), dims.M))
      return fail(HMM_ERR_UNSUPPORTED, "tensor-core adjoint supports M <= 256 (M=%d)", dims.M);
    const size_t m = make_layout(dims, *seqs, op, true).total;
    if (m > need) need = m;
  }
  *bytes = need;
  return HMM_OK;
}

int hmm_forward_backward_workspace_size(hmm_dims_t dims, const hmm_seqs_t* seqs,
                                        hmm_precision_t precision, size_t* bytes) {
  g_err[0] = 0;
  if (precision != HMM_TF32_MMA)
    return hmm_workspace_size(dims, seqs, HMM_OP_FORWARD_BACKWARD, bytes);
  if (!bytes) return fail(HMM_ERR_ARG, "bytes is NULL");
  int rc = check_dims(dims, max_states(HMM_OP_FORWARD_BACKWARD, HMM_TF32_MMA));
  if (rc) return rc;
  if (!seqs) return fail(HMM_ERR_ARG, "seqs is NULL");
  if (seqs->S < 0 || seqs->total_obs < 0) return fail(HMM_ERR_ARG, "negative S or total_obs");
  if (pad_states(dims.N) != 128)
    return fail(HMM_ERR_UNSUPPORTED, "TF32 adjoint needs 64 < N <= 128 (N=%d)", dims.N);
  if (!tf32_adjoint_m_ok(128, dims.M))
    return fail(HMM_ERR_UNSUPPORTED, "TF32 adjoint: M=%d too large", dims.M);
  *bytes = make_layout(dims, *seqs, HMM_OP_FORWARD_BACKWARD, true, 0, true).total;
  return HMM_OK;
}

int hmm_set_tuning(int32_t op, int32_t n_pad, int32_t lanes) {
  g_err[0] = 0;
  const int ni = np_index(n_pad);
  if (op < 0 || op >= kTuneOps || ni < 0) return fail(HMM_ERR_ARG, "bad op %d or n_pad %d", op, n_pad);
  if (lanes != 0) {
    bool ok = false;
    for (int i = 0; i < 5 && kCand[op][ni][i]; ++i) ok |= kCand[op][ni][i] == lanes;
    if (!ok) return fail(HMM_ERR_ARG, "lanes %d not instantiated for op %d n_pad %d", lanes, op, n_pad);
  }
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  g_tuning[op][ni] = lanes;
  return HMM_OK;
}

int hmm_get_tuning(int32_t op, int32_t n_pad, int32_t* lanes) {
  g_err[0] = 0;
  const int ni = np_index(n_pad);
  if (op < 0 || op >= kTuneOps || ni < 0 || !lanes) return fail(HMM_ERR_ARG, "bad op, n_pad or pointer");
  if (!kCand[op][ni][0]) return fail(HMM_ERR_UNSUPPORTED, "no kernel for op %d n_pad %d", op, n_pad);
  *lanes = lanes_for(op, n_pad);
  return HMM_OK;
}

int hmm_tuning_candidates(int32_t op, int32_t n_pad, int32_t* out, int32_t cap) {
  g_err[0] = 0;
  const int n = candidates(op, n_pad, out, cap);
  if (n < 0) return fail(HMM_ERR_ARG, "bad op %d or n_pad %d", op, n_pad);
  return n;
}

int hmm_forward(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                const hmm_seqs_t* seqs, hmm_precision_t precision, float* loglik,
                int32_t* argmax, void* ws, size_t ws_bytes, hmm_stream_t stream) {
  g_err[0] = 0;
  int rc = check_precision(precision, HMM_OP_FORWARD);
  if (rc) return rc;
  if ((rc = check_dims(dims, max_states(HMM_OP_FORWARD, precision)))) return rc;
  if ((rc = check_seqs(seqs, dims))) return rc;
  if ((rc = check_params(pi, A, B))) return rc;
  if (seqs->S > 0 && (!loglik || !al(loglik, 4))) return fail(HMM_ERR_ARG, "loglik NULL or misaligned");
  if (argmax && !al(argmax, 4)) return fail(HMM_ERR_ARG, "argmax misaligned");
  const bool mma = use_mma_forward(dims, precision);
  // HMM_AUTO takes the parallel-in-time forward for batches of few long
  // sequences, when the workspace holds its chunk products
  if (precision == HMM_AUTO && !mma && scan_preferred(dims, *seqs) && ws && al(ws, 256) &&
      ws_bytes >= make_layout(dims, *seqs, HMM_OP_FORWARD_SCAN, false,
                              scan_chunk_len(0, seqs->max_len)).total)
    return hmm_forward_scan(dims, pi, A, B, seqs, 0, loglik, argmax, ws, ws_bytes, stream);
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_FORWARD);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  const bool all = seqs->model_of_seq == nullptr;
  if (mma && dims.N <= 32)
    return fail(HMM_ERR_UNSUPPORTED, "tensor-core forward needs N > 32 (N=%d: use HMM_FP32)", dims.N);
  if (mma && (!all || seqs->model_base))
    return fail(HMM_ERR_UNSUPPORTED,
                "tensor-core forward scores every sequence against every model "
                "(model_of_seq and model_base must be NULL)");
  if (seqs->S == 0) return HMM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (mma && L.NP >= 256) {
    // wide state counts: each tile on a cluster of CTAs where its slices fit,
    // else one 128-row tile per CTA with A^T streamed
    const bool cluster = forward_cluster_fits(L.NP, dims.M);
    const int rows = cluster ? cluster_tile_rows(L.NP, seqs->S, dims.K, 1) : 128;
    const int n_tiles = (seqs->S + rows - 1) / rows;
    if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
    SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
    s.bf16_b = 1;  // BF16 path: B rounded to BF16 like A
    s.ndone = argmax ? n_tiles : 0;
    {
      Timed tm(T_SETUP, st);
      e = launch_setup(s, st);
      tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(e, "setup launch");
    MmaWideLaunch f;
    memset(&f, 0, sizeof(f));
    f.seq = seq_args(dims, *seqs, L, ws);
    f.mod = model_args(L, ws);
    f.img = at<uint8_t>(ws, L.wimg);
    f.loglik = loglik;
    f.argmax = argmax;
    f.done = at<int32_t>(ws, L.done);
    f.queue = &at<WsHeader>(ws, 0)->queue[0];
    f.status = &at<WsHeader>(ws, 0)->status;
    f.n_tiles = n_tiles;
    f.rows = rows;
    f.n_items = n_tiles * dims.K;
    f.wait_limit = wait_limit_polls();
    {
      Timed tm(T_FORWARD, st);
      e = cluster ? launch_forward_cluster(L.NP, f, st) : launch_forward_wide(L.NP, f, st);
      tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core forward launch");
    return HMM_OK;
  }
  if (mma) {
    const int n_tiles = (seqs->S + 127) / 128;
    const int nt = mma_tiles_per_cta(L.NP);
    const int n_pairs = (n_tiles + nt - 1) / nt;  // tile groups of one CTA
    if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
    SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
    s.bf16_b = precision != HMM_TF32_MMA;  // BF16 path: B rounded to BF16 like A
    s.ndone = argmax ? n_pairs : 0;
    {
      Timed tm(T_SETUP, st);
      e = launch_setup(s, st);
      tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(e, "setup launch");
    MmaFwdLaunch f;
    f.seq = seq_args(dims, *seqs, L, ws);
    f.mod = model_args(L, ws);
    f.loglik = loglik;
    f.argmax = argmax;
    f.done = at<int32_t>(ws, L.done);
    f.queue = &at<WsHeader>(ws, 0)->queue[0];
    f.status = &at<WsHeader>(ws, 0)->status;
    f.n_tiles = n_tiles;
    f.n_items = n_pairs * dims.K;
    f.wait_limit = wait_limit_polls();
    {
      Timed tm(T_FORWARD, st);
      e = launch_forward_mma(L.NP, precision == HMM_TF32_MMA, f, st);
      tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core forward launch");
    return HMM_OK;
  }
  const int G = lanes_for(HMM_OP_FORWARD, L.NP);
  const int PP = 32 / G;
  const int ngroups = (seqs->S + PP - 1) / PP;

  e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
  s.ndone = (all && argmax) ? ngroups : 0;
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");

  FwdLaunch f;
  f.seq = seq_args(dims, *seqs, L, ws);
  f.mod = model_args(L, ws);
  f.loglik = loglik;
  f.argmax = all ? argmax : nullptr;
  f.done = at<int32_t>(ws, L.done);
  f.queue = &at<WsHeader>(ws, 0)->queue[0];
  f.status = &at<WsHeader>(ws, 0)->status;
  f.n_items = all ? ngroups * span_of(*seqs, dims) : ngroups;
  {
    Timed tm(T_FORWARD, st);
    e = launch_forward(L.NP, G, f, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  return HMM_OK;
}

int hmm_forward_scan_workspace_size(hmm_dims_t dims, const hmm_seqs_t* seqs, int32_t chunk,
                                    size_t* bytes) {
  g_err[0] = 0;
  if (!bytes) return fail(HMM_ERR_ARG, "bytes is NULL");
  int rc = check_dims(dims, max_states(HMM_OP_FORWARD_SCAN, HMM_FP32));
  if (rc) return rc;
  if (!seqs) return fail(HMM_ERR_ARG, "seqs is NULL");
  if (seqs->S < 0 || seqs->total_obs < 0 || seqs->max_len < 0)
    return fail(HMM_ERR_ARG, "negative S, max_len or total_obs");
  if (chunk < 0 || chunk > kScanMaxChunk)
    return fail(HMM_ERR_ARG, "chunk %d outside [0, %d]", chunk, kScanMaxChunk);
  *bytes = make_layout(dims, *seqs, HMM_OP_FORWARD_SCAN, false,
                       scan_chunk_len(chunk, seqs->max_len)).total;
  return HMM_OK;
}

int hmm_forward_scan(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                     const hmm_seqs_t* seqs, int32_t chunk, float* loglik, int32_t* argmax,
                     void* ws, size_t ws_bytes, hmm_stream_t stream) {
  g_err[0] = 0;
  int rc;
  if ((rc = check_dims(dims, max_states(HMM_OP_FORWARD_SCAN, HMM_FP32)))) return rc;
  if ((rc = check_seqs(seqs, dims))) return rc;
  if ((rc = check_params(pi, A, B))) return rc;
  if (chunk < 0 || chunk > kScanMaxChunk)
    return fail(HMM_ERR_ARG, "chunk %d outside [0, %d]", chunk, kScanMaxChunk);
  if (seqs->S > 0 && (!loglik || !al(loglik, 4))) return fail(HMM_ERR_ARG, "loglik NULL or misaligned");
  if (argmax && !al(argmax, 4)) return fail(HMM_ERR_ARG, "argmax misaligned");
  const int Lc = scan_chunk_len(chunk, seqs->max_len);
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_FORWARD_SCAN, false, Lc);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  if (seqs->S == 0) return HMM_OK;
  const bool all = seqs->model_of_seq == nullptr;
  const int span = all ? span_of(*seqs, dims) : 1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
  s.ndone = (all && argmax) ? seqs->S : 0;
  s.scan_chunk = Lc;
  s.coff = at<int64_t>(ws, L.sc_coff);
  s.coff_cap = L.sc_cap;
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");
  ScanLaunch a;
  a.seq = seq_args(dims, *seqs, L, ws);
  a.mod = model_args(L, ws);
  a.coff = at<int64_t>(ws, L.sc_coff);
  a.P = at<float>(ws, L.sc_P);
  a.E = at<int32_t>(ws, L.sc_E);
  a.cap = L.sc_cap;
  a.L = Lc;
  a.loglik = loglik;
  a.argmax = all ? argmax : nullptr;
  a.done = at<int32_t>(ws, L.done);
  a.queue = &at<WsHeader>(ws, 0)->queue[0];
  a.status = &at<WsHeader>(ws, 0)->status;
  const int rpw = 32 / L.NP;
  a.n_pair_items = (int)(((int64_t)seqs->S * span + rpw - 1) / rpw);
  {
    Timed tm(T_SCAN_CHUNKS, st);
    e = launch_scan(L.NP, a, L.sc_cap * span, 0, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "scan chunk launch");
  {
    Timed tm(T_SCAN_COMBINE, st);
    e = launch_scan(L.NP, a, L.sc_cap * span, 1, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "scan combine launch");
  return HMM_OK;
}

int hmm_viterbi(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                const hmm_seqs_t* seqs, float* score, int32_t* best_model, int32_t* path,
                void* ws, size_t ws_bytes, hmm_stream_t stream) {
  g_err[0] = 0;
  int rc;
  if ((rc = check_dims(dims, max_states(HMM_OP_VITERBI, HMM_FP32)))) return rc;
  if ((rc = check_seqs(seqs, dims))) return rc;
  if ((rc = check_params(pi, A, B))) return rc;
  if (seqs->S > 0 && (!score || !al(score, 4))) return fail(HMM_ERR_ARG, "score NULL or misaligned");
  if ((best_model && !al(best_model, 4)) || (path && !al(path, 4)))
    return fail(HMM_ERR_ARG, "best_model/path misaligned");
  if (path && seqs->total_obs > 0 && !seqs->symbols) return fail(HMM_ERR_ARG, "symbols NULL");
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_VITERBI);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  if (seqs->S == 0) return HMM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool all = seqs->model_of_seq == nullptr;
  // above 64 states: one warp per pair (four in all-models score blocks),
  // the log matrix in shared memory; an all-models score item is a group of
  // 16 sequences sharing the block's matrix
  const bool wide = L.NP > 64;
  const int G = wide ? 32 : lanes_for(HMM_OP_VITERBI, L.NP);
  const int PP = wide ? ((all && !seqs->model_base) ? 16 : 1) : 32 / G;
  const int ngroups = (seqs->S + PP - 1) / PP;
  const int Gp = wide ? 32 : lanes_for(HMM_TUNE_VITERBI_PATHS, L.NP);
  const int PPp = 32 / Gp;
  int32_t* best = best_model ? best_model : at<int32_t>(ws, L.best);
  const bool need_best = all && (best_model || path);

  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 1);
  s.ndone = need_best ? ngroups : 0;
  s.want_bpoff = path ? 1 : 0;
  s.bpoff = at<int64_t>(ws, L.bpoff);
  s.bp_cap_rows = seqs->total_obs;
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");

  VitLaunch v;
  v.seq = seq_args(dims, *seqs, L, ws);
  v.mod = model_args(L, ws);
  v.score = score;
  v.path = path;
  v.done = at<int32_t>(ws, L.done);
  v.queue = &at<WsHeader>(ws, 0)->queue[0];
  v.status = &at<WsHeader>(ws, 0)->status;
  v.bpoff = at<int64_t>(ws, L.bpoff);
  v.bp = at<uint8_t>(ws, L.bp);
  v.gorder = wide ? at<int32_t>(ws, L.vgorder) : nullptr;
  v.gcount = wide ? at<int32_t>(ws, L.vgcount) : nullptr;
  v.n_items_score = all ? ngroups * span_of(*seqs, dims) : ngroups;
  v.n_items_path = (seqs->S + PPp - 1) / PPp;
  auto scores = [&]() {
    Timed tm(T_VSCORES, st);
    cudaError_t r = wide ? launch_viterbi_scores_wide(v, st) : launch_viterbi_scores(L.NP, G, v, st);
    tm.stop();
    return r;
  };
  auto paths = [&]() {
    Timed tm(T_VPATHS, st);
    cudaError_t r = wide ? launch_viterbi_paths_wide(v, st) : launch_viterbi_paths(L.NP, Gp, v, st);
    tm.stop();
    return r;
  };
  if (all) {
    v.best = need_best ? best : nullptr;
    if ((e = scores()) != cudaSuccess) return cuda_fail(e, "viterbi scores");
    if (path) {
      v.best = best;
      if ((e = paths()) != cudaSuccess) return cuda_fail(e, "viterbi paths");
    }
  } else {
    v.best = best_model;
    if (path) {
      if ((e = paths()) != cudaSuccess) return cuda_fail(e, "viterbi paths");
    } else {
      if ((e = scores()) != cudaSuccess) return cuda_fail(e, "viterbi scores");
    }
  }
  return HMM_OK;
}

// hmm_forward_backward with TF32 operands (64 < N <= 128): the tile plan,
// the TF32 passes keeping every step's rows (mma_pass_tf32.cu), then the
// count kernels of fb_wide.cu over the rows of each model.
static int fb_tf32(const hmm_dims_t& dims, const hmm_seqs_t* seqs, const float* weight,
                   float* loglik, float* cnt_pi, float* cnt_A, float* cnt_B, void* ws,
                   size_t ws_bytes, hmm_stream_t stream, const float* pi, const float* A,
                   const float* B) {
  const int NP = pad_states(dims.N);
  if (NP != 128)
    return fail(HMM_ERR_UNSUPPORTED, "TF32 adjoint needs 64 < N <= 128 (N=%d: use HMM_FP32)", dims.N);
  if (!tf32_adjoint_m_ok(NP, dims.M))
    return fail(HMM_ERR_UNSUPPORTED, "TF32 adjoint: M=%d too large", dims.M);
  if (seqs->model_of_seq && dims.K > 65536)
    return fail(HMM_ERR_UNSUPPORTED, "tensor-core adjoint supports K <= 65536 labelled models");
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_FORWARD_BACKWARD, true, 0, true);
  int rc;
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (seqs->S == 0) return zero_counts(dims, cnt_pi, cnt_A, cnt_B, st);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
  s.skip_order = 1;  // the tile plan orders the sequences itself
  const bool labelled = seqs->model_of_seq != nullptr;
  const int cap = L.m_pass_cap;
  int32_t* tiles = at<int32_t>(ws, L.m_tiles);
  MmaPlanArgs p;
  memset(&p, 0, sizeof(p));
  p.S = seqs->S; p.K = dims.K; p.labelled = labelled ? 1 : 0;
  p.seqlen = at<int32_t>(ws, L.seqlen);
  p.model_of_seq = seqs->model_of_seq;
  p.loglik = loglik;
  p.sorted = at<int32_t>(ws, L.m_sorted);
  p.tmp = at<int32_t>(ws, L.m_tmp);
  p.key = at<uint32_t>(ws, L.m_keys);
  p.key_tmp = p.key + std::max<int64_t>(seqs->S, (int64_t)cap);
  p.tile_start = tiles; p.tile_rows = tiles + cap; p.tile_model = tiles + 2 * cap;
  p.tile_len = tiles + 3 * cap; p.tile_order = tiles + 4 * cap; p.tile_tmp = tiles + 5 * cap;
  p.group_start = tiles + 6 * cap; p.group_end = p.group_start + dims.K;
  p.n_tiles_cap = cap;
  p.n_tiles = at<int32_t>(ws, L.m_ntiles);
  p.group = 1;
  p.spr = L.m_spr;
  p.pass_tiles = at<int32_t>(ws, L.m_pass);
  p.pass_tmp = at<int32_t>(ws, L.m_ptmp);
  p.n_pass = at<int32_t>(ws, L.m_npass);
  p.pass_cap = L.m_pass_cap;
  p.rng_tile = at<int32_t>(ws, L.m_rtile);
  p.rng_seg = at<int32_t>(ws, L.m_rseg);
  p.rng_model = at<int32_t>(ws, L.m_rmodel);
  p.rng_len = at<int32_t>(ws, L.m_rlen);
  p.n_rng = at<int32_t>(ws, L.m_nrng);
  p.rng_cap = L.m_rng_cap;
  {
    const int nb = (int)((seqs->S + 4095) / 4096 > 0 ? (seqs->S + 4095) / 4096 : 1);
    p.bcnt = at<int32_t>(ws, L.m_pscr);
    p.hist = p.bcnt + nb;
    p.n_valid = p.hist + 256 * nb;
  }
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    if (e == cudaSuccess) e = launch_mma_plan(p, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");

  MmaPassLaunch pa;
  memset(&pa, 0, sizeof(pa));
  pa.seq = seq_args(dims, *seqs, L, ws);
  pa.mod = model_args(L, ws);
  pa.sorted = p.sorted;
  pa.tile_start = p.tile_start; pa.tile_rows = p.tile_rows; pa.tile_model = p.tile_model;
  pa.tile_len = p.tile_len;
  pa.pass_tiles = p.pass_tiles;
  pa.n_pass = p.n_pass;
  pa.labelled = p.labelled;
  pa.loglik = loglik;
  pa.queue = &at<WsHeader>(ws, 0)->queue[5];
  pa.status = &at<WsHeader>(ws, 0)->status;
  pa.wait_limit = wait_limit_polls();
  pa.xs = at<float>(ws, L.w_X);
  pa.bhs = at<float>(ws, L.w_Bh);
  pa.xe = at<int32_t>(ws, L.w_xe);
  pa.rp = at<int64_t>(ws, L.bpoff);
  pa.rtot = L.w_rtot;
  int64_t* pos_row = at<int64_t>(ws, L.t_pos);
  int64_t* mrow = at<int64_t>(ws, L.t_mrow);
  {
    Timed tm(T_FB_PASS, st);
    e = launch_fb_pass_tf32(NP, pa, p.n_valid, pos_row, mrow, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "TF32 adjoint pass launch");

  FbWideArgs c;
  memset(&c, 0, sizeof(c));
  c.K = dims.K; c.N = dims.N; c.M = dims.M; c.NP = NP; c.S = seqs->S;
  c.labelled = labelled ? 1 : 0;
  c.rtot = L.w_rtot;
  c.nrows = labelled ? L.w_rtot : (int64_t)dims.K * L.w_rtot;
  c.u_in_x = 0;  // the passes store every row the contraction reads (zeros where dead)
  c.X = pa.xs;
  c.Bh = pa.bhs;
  c.V = at<float>(ws, L.w_V);
  c.G = at<float>(ws, L.w_G);
  c.xe = pa.xe;
  c.sym = at<int32_t>(ws, L.w_sym);
  c.seqlen = at<int32_t>(ws, L.seqlen);
  c.offsets = seqs->offsets;
  c.symbols = seqs->symbols;
  c.Btp = at<float>(ws, L.Btp);
  c.weight = weight;
  c.A = A;
  c.Cp = at<float>(ws, L.w_Cp);
  c.nsplit = L.w_nsplit;
  emis_args(c, L, ws);
  c.cnt_pi = cnt_pi;
  c.cnt_A = cnt_A;
  c.cnt_B = cnt_B;
  c.status = &at<WsHeader>(ws, 0)->status;
  c.pos_row = pos_row;
  c.row_pos = at<int32_t>(ws, L.t_rpos);
  c.sorted = p.sorted;
  c.n_valid = p.n_valid;
  c.model_of_seq = seqs->model_of_seq;
  c.mrow = mrow;
  {
    Timed tm(T_FB, st);
    e = launch_fbw_counts(c, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint count launch");
  return HMM_OK;
}

int hmm_forward_backward(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                         const hmm_seqs_t* seqs, const float* weight, hmm_precision_t precision,
                         float* loglik, float* cnt_pi, float* cnt_A, float* cnt_B, void* ws,
                         size_t ws_bytes, hmm_stream_t stream) {
  g_err[0] = 0;
  int rc = check_precision(precision, HMM_OP_FORWARD_BACKWARD);
  if (rc) return rc;
  if ((rc = check_dims(dims, max_states(HMM_OP_FORWARD_BACKWARD, precision)))) return rc;
  if ((rc = check_seqs(seqs, dims))) return rc;
  if ((rc = check_params(pi, A, B))) return rc;
  if (!cnt_pi || !cnt_A || !cnt_B || !al(cnt_pi, 4) || !al(cnt_A, 4) || !al(cnt_B, 4))
    return fail(HMM_ERR_ARG, "count outputs NULL or misaligned");
  if (seqs->S > 0 && (!loglik || !al(loglik, 4))) return fail(HMM_ERR_ARG, "loglik NULL or misaligned");
  if (weight && !al(weight, 4)) return fail(HMM_ERR_ARG, "weight misaligned");
  if (seqs->model_base)
    return fail(HMM_ERR_UNSUPPORTED, "model sets apply to recognition; the adjoint takes model_of_seq");
  if (precision == HMM_TF32_MMA)
    return fb_tf32(dims, seqs, weight, loglik, cnt_pi, cnt_A, cnt_B, ws, ws_bytes, stream, pi, A, B);
  if (use_mma_fb(dims, precision)) {
    if (dims.N <= 32)
      return fail(HMM_ERR_UNSUPPORTED, "tensor-core adjoint needs N > 32 (N=%d: use HMM_FP32)", dims.N);
    if (pad_states(dims.N) >= 256)
      return fb_wide(dims, seqs, weight, loglik, cnt_pi, cnt_A, cnt_B, ws, ws_bytes, stream, pi, A, B);
    return fb_mma(dims, seqs, weight, loglik, cnt_pi, cnt_A, cnt_B, ws, ws_bytes, stream, pi, A, B);
  }
  const WsLayout L = make_layout(dims, *seqs, HMM_OP_FORWARD_BACKWARD);
  if ((rc = check_ws(ws, ws_bytes, L))) return rc;
  const int G = lanes_for(HMM_OP_FORWARD_BACKWARD, L.NP);
  const int C = ckpt_stride(seqs->max_len);
  const int NC = (seqs->max_len > 0 ? (seqs->max_len - 1) / C : 0) + 1;
  // segment ranges per pair (1 = the single-kernel adjoint)
  int spar = lanes_for(HMM_TUNE_FB_RANGES, L.NP);
  if (spar > L.s_planes) spar = L.s_planes;
  const int spg = (NC + (spar > 0 ? spar : 1) - 1) / (spar > 0 ? spar : 1);
  if (spar > 1) spar = (NC + spg - 1) / spg;  // no empty ranges
  const size_t smem = spar > 1 ? fb_seg_smem_bytes(L.NP, G, C, dims.M, 1)
                               : fb_smem_bytes(L.NP, G, C, NC, dims.M, 1);  // one warp per block
  if (smem > 227 * 1024)
    return fail(HMM_ERR_UNSUPPORTED,
                "adjoint shared memory %zu bytes above 227 KB (N=%d M=%d max_len=%d)", smem,
                dims.N, dims.M, seqs->max_len);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (seqs->S == 0) {
    const size_t n = (size_t)dims.K * dims.N;
    if ((e = cudaMemsetAsync(cnt_pi, 0, n * 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(cnt_A, 0, n * dims.N * 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(cnt_B, 0, n * dims.M * 4, st)) != cudaSuccess)
      return cuda_fail(e, "memset");
    return HMM_OK;
  }
  const bool labelled = seqs->model_of_seq != nullptr;
  const int PP = 32 / G;
  const int ngroups = (seqs->S + PP - 1) / PP;

  if ((e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st)) != cudaSuccess) return cuda_fail(e, "memset");
  SetupArgs s = setup_args(dims, *seqs, L, ws, pi, A, B, 0);
  {
    Timed tm(T_SETUP, st);
    e = launch_setup(s, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "setup launch");

  const int items = labelled ? ngroups : ngroups * dims.K;
  if (spar > 1) {
    FbSegLaunch f;
    f.seq = seq_args(dims, *seqs, L, ws);
    f.mod = model_args(L, ws);
    f.weight = weight;
    f.loglik = loglik;
    f.partial = at<float>(ws, L.partial);
    f.slot_floats = L.slot_floats;
    f.ckA = at<float>(ws, L.s_ckA);
    f.ckB = at<float>(ws, L.s_ckB);
    f.ckE = at<int32_t>(ws, L.s_ckE);
    f.sig = at<float>(ws, L.s_sig);
    f.skip = at<int32_t>(ws, L.s_skip);
    f.queue = &at<WsHeader>(ws, 0)->queue[4];
    f.status = &at<WsHeader>(ws, 0)->status;
    f.npairs = (int)L.slots;
    f.n_items_pass = 2 * items;
    f.n_items_seg = items * spar;
    f.ckpt = C;
    f.nck = NC;
    f.spar = spar;
    f.spg = spg;
    {
      Timed tm(T_FB_PASS, st);
      e = launch_fb_seg(L.NP, G, f, 0, st);
      tm.stop();
    }
    if (e == cudaSuccess) {
      Timed tm(T_FB, st);
      e = launch_fb_seg(L.NP, G, f, 1, st);
      tm.stop();
    }
  } else {
    FbLaunch f;
    f.seq = seq_args(dims, *seqs, L, ws);
    f.mod = model_args(L, ws);
    f.weight = weight;
    f.loglik = loglik;
    f.partial = at<float>(ws, L.partial);
    f.slot_floats = L.slot_floats;
    f.queue = &at<WsHeader>(ws, 0)->queue[2];
    f.status = &at<WsHeader>(ws, 0)->status;
    f.n_items = items;
    f.ckpt = C;
    f.nck = NC;
    Timed tm(T_FB, st);
    e = launch_fb(L.NP, G, f, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");

  ReduceLaunch r;
  r.partial = at<float>(ws, L.partial);
  r.red1 = at<float>(ws, L.red1);
  r.model_of_seq = seqs->model_of_seq;
  r.seqlen = at<int32_t>(ws, L.seqlen);
  r.S = seqs->S; r.K = dims.K; r.N = dims.N; r.M = dims.M; r.NP = L.NP;
  r.planes = spar > 1 ? spar : 1;
  r.slot_floats = L.slot_floats;
  r.nchunks = first_chunks(seqs->S * r.planes);
  r.cnt_pi = cnt_pi; r.cnt_A = cnt_A; r.cnt_B = cnt_B;
  {
    Timed tm(T_REDUCE, st);
    e = launch_reduce(r, st);
    tm.stop();
  }
  if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
  return HMM_OK;
}

int hmm_softmax_rows(hmm_dims_t dims, const float* lpi, const float* lA, const float* lB,
                     float* pi, float* A, float* B, hmm_stream_t stream) {
  g_err[0] = 0;
  if (dims.K < 1 || dims.N < 1 || dims.M < 1) return fail(HMM_ERR_ARG, "dims must be positive");
  if (!lpi || !lA || !lB || !pi || !A || !B) return fail(HMM_ERR_ARG, "NULL table");
  Timed tm(T_SOFTMAX, reinterpret_cast<cudaStream_t>(stream));
  cudaError_t e = launch_softmax_rows(dims.K, dims.N, dims.M, lpi, lA, lB, pi, A, B,
                                      reinterpret_cast<cudaStream_t>(stream));
  tm.stop();
  return e == cudaSuccess ? HMM_OK : cuda_fail(e, "softmax launch");
}

int hmm_softmax_grad(hmm_dims_t dims, const float* pi, const float* A, const float* B,
                     const float* cpi, const float* cA, const float* cB, float* gpi, float* gA,
                     float* gB, hmm_stream_t stream) {
  g_err[0] = 0;
  if (dims.K < 1 || dims.N < 1 || dims.M < 1) return fail(HMM_ERR_ARG, "dims must be positive");
  if (!pi || !A || !B || !cpi || !cA || !cB || !gpi || !gA || !gB) return fail(HMM_ERR_ARG, "NULL table");
  Timed tm(T_SGRAD, reinterpret_cast<cudaStream_t>(stream));
  cudaError_t e = launch_softmax_grad(dims.K, dims.N, dims.M, pi, A, B, cpi, cA, cB, gpi, gA, gB,
                                      reinterpret_cast<cudaStream_t>(stream));
  tm.stop();
  return e == cudaSuccess ? HMM_OK : cuda_fail(e, "softmax grad launch");
}

int hmm_mstep(hmm_dims_t dims, const float* pi, const float* A, const float* B,
              const float* cnt_pi, const float* cnt_A, const float* cnt_B, float* pi_out,
              float* A_out, float* B_out, hmm_stream_t stream) {
  g_err[0] = 0;
  if (dims.K < 1 || dims.N < 1 || dims.M < 1) return fail(HMM_ERR_ARG, "dims must be positive");
  if (!pi || !A || !B || !cnt_pi || !cnt_A || !cnt_B || !pi_out || !A_out || !B_out)
    return fail(HMM_ERR_ARG, "NULL table");
  Timed tm(T_MSTEP, reinterpret_cast<cudaStream_t>(stream));
  cudaError_t e = launch_mstep(dims.K, dims.N, dims.M, pi, A, B, cnt_pi, cnt_A, cnt_B, pi_out,
                               A_out, B_out, reinterpret_cast<cudaStream_t>(stream));
  tm.stop();
  return e == cudaSuccess ? HMM_OK : cuda_fail(e, "mstep launch");
}

int hmm_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, float grad_scale, int32_t* step,
                  hmm_stream_t stream) {
  g_err[0] = 0;
  if (n < 0 || !step) return fail(HMM_ERR_ARG, "n < 0 or step counter NULL");
  if (n == 0) return HMM_OK;
  if (!param || !grad || !m || !v) return fail(HMM_ERR_ARG, "NULL buffer");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f))
    return fail(HMM_ERR_ARG, "betas must lie in [0, 1)");
  Timed tm(T_ADAM, reinterpret_cast<cudaStream_t>(stream));
  cudaError_t e = launch_adam(n, param, grad, m, v, lr, beta1, beta2, eps, grad_scale, step,
                              reinterpret_cast<cudaStream_t>(stream));
  tm.stop();
  return e == cudaSuccess ? HMM_OK : cuda_fail(e, "adam launch");
}

int hmm_get_device_status(const void* ws, hmm_stream_t stream, int32_t* status) {
  g_err[0] = 0;
  if (!ws || !status) return fail(HMM_ERR_ARG, "NULL workspace or status");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  *status = h;
  if (h) return fail(HMM_ERR_DEVICE, "device status 0x%x%s%s%s", h,
                     (h & HMM_STATUS_SYMBOL) ? " symbol-out-of-range" : "",
                     (h & HMM_STATUS_PARAM) ? " bad-parameter" : "",
                     (h & HMM_STATUS_SEQ) ? " bad-sequence" : "");
  return HMM_OK;
}

int hmm_set_wait_limit(int64_t polls) {
  g_err[0] = 0;
  const uint32_t v = polls < 0 ? kDrainPolls
                               : (polls > (int64_t)0xffffffff ? 0xffffffffu : (uint32_t)polls);
  g_wait_limit.store(v, std::memory_order_relaxed);
  return HMM_OK;
}

uint32_t hmm_get_wait_limit(void) { return wait_limit_polls(); }

int hmm_timing_enable(int on) {
  g_err[0] = 0;
  std::lock_guard<std::mutex> lk(g_timing.mu);
  g_timing.on = on != 0;
  return HMM_OK;
}

int hmm_timing_reset(void) {
  g_err[0] = 0;
  std::lock_guard<std::mutex> lk(g_timing.mu);
  for (auto& r : g_timing.rec) {
    for (auto& p : r) g_timing.pool.push_back(p);
    r.clear();
  }
  return HMM_OK;
}

int hmm_timing_read(int32_t kind, int64_t* launches, double* total_ms) {
  g_err[0] = 0;
  if (kind < 0 || kind >= HMM_TIMING_KINDS || !launches || !total_ms)
    return fail(HMM_ERR_ARG, "bad timing kind or NULL output");
  std::lock_guard<std::mutex> lk(g_timing.mu);
  double tot = 0.0;
  for (auto& p : g_timing.rec[kind]) {
    cudaError_t e = cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return cuda_fail(e, "timing read");
    tot += ms;
  }
  *launches = (int64_t)g_timing.rec[kind].size();
  *total_ms = tot;
  return HMM_OK;
}

}  // extern "C"
