// noalloc.cu -- hmm_forward_static: the forward/recognition call for callers
// that cannot hand the library a device workspace.
//
// Some integrations cannot allocate device memory at the point where they
// score sequences: real-time or embedded hosts that forbid cudaMalloc after
// start-up (allocation can block, fragment memory or fail mid-run), plug-in
// hosts that own every device allocation and expose none to plug-ins, and
// code that must not touch an allocator at all on its recognition path.
// They still own their inputs and outputs; only the scratch space is the
// problem. This entry point takes its scratch from a fixed array compiled
// into the library instead of from a caller-owned workspace, and otherwise
// runs exactly the hmm_forward launch sequence on it.
//
// The array lives in device memory of every GPU that loads the library, for
// the life of the process. Its size is fixed at build time
// (HMM_STATIC_SCRATCH_BYTES); calls whose scratch need is larger are refused.
// Host code cannot use the array's name as a device address (it names a host
// shadow), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <stdio.h>

#include <mutex>

#include "hmm_internal.cuh"

namespace hmmgb {
int report_error(int code, const char* msg);
}

static __device__ __align__(256) unsigned char g_static_scratch[HMM_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_static_scratch on the current device (looked up on the
// first call per device). Returns HMM_OK or an error code with the message set.
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hmmgb::report_error(HMM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return hmmgb::report_error(HMM_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return hmmgb::report_error(HMM_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                : "static scratch has no address");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HMM_OK;
}
}  // namespace

extern "C" int hmm_forward_static(hmm_dims_t dims, const float* pi, const float* A,
                                  const float* B, const hmm_seqs_t* seqs,
                                  hmm_precision_t precision, float* loglik, int32_t* argmax,
                                  hmm_stream_t stream) {
  size_t need = 0;
  int rc = hmm_workspace_size(dims, seqs, HMM_OP_FORWARD, &need);
  if (rc != HMM_OK) return rc;
  // the sequential recursion's need (HMM_AUTO's parallel-in-time variant is
  // only taken when its storage fits the scratch)
  need = hmmgb::forward_ws_sequential(dims, *seqs);
  if (need > (size_t)HMM_STATIC_SCRATCH_BYTES) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "hmm_forward_static needs %zu bytes of scratch, above its fixed %d; "
             "use hmm_forward with a workspace",
             need, HMM_STATIC_SCRATCH_BYTES);
    return hmmgb::report_error(HMM_ERR_WORKSPACE, msg);
  }
  void* scratch = nullptr;
  if ((rc = scratch_address(&scratch)) != HMM_OK) return rc;
  // hmm_forward clears the header (status word and work counter) and the
  // argmax counters it uses before its kernels run; nothing else in the
  // scratch has to start at zero.
  return hmm_forward(dims, pi, A, B, seqs, precision, loglik, argmax, scratch,
                     (size_t)HMM_STATIC_SCRATCH_BYTES, stream);
}
