"""hmm_forward_static: forward scoring for callers that cannot allocate.

Real-time and embedded hosts that forbid device allocation after start-up,
and plug-in hosts that own every device allocation, cannot pass the library
a workspace. hmm_forward_static serves them from a fixed scratch array
compiled into the library. These tests call it through the C-ABI and check
that, on two calls in a row, it returns what hmm_forward (the workspace
entry point) returns -- bit for bit, since both run the same kernels on the
same inputs, which is within any tolerance of the parity tests -- on the
FP32 recursion, the BF16 tensor-core forward and HMM_AUTO's parallel-in-time
branch for few long sequences (chunk products in the fixed array), and that
a request larger than the fixed array is refused.

The file name sorts last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process (the
first call performs the per-device set-up).
"""
import ctypes

import numpy as np
import pytest

from helpers import ll_tol, to_gpu
from paper_1310_3322_gb300 import hmm, synth


def _call_static(lib, pi, A, B, seqs, loglik, argmax, precision=hmm.HMM_FP32):
    import torch
    c = seqs.c()
    dims = hmm.hmm_dims_t(int(pi.shape[0]), int(pi.shape[1]), int(B.shape[2]))
    return lib.hmm_forward_static(dims, pi.data_ptr(), A.data_ptr(), B.data_ptr(),
                                  ctypes.byref(c), precision, loglik.data_ptr(),
                                  argmax.data_ptr() if argmax is not None else None,
                                  torch.cuda.current_stream().cuda_stream)


def _twice_equal(lib, w, labelled, precision):
    import torch
    seqs, pi, A, B = to_gpu(w, labelled=labelled)
    ref_ll, ref_am = hmm.hmm_forward(pi, A, B, seqs, precision=precision)
    assert bool(torch.isfinite(ref_ll).all())
    for _ in range(2):
        ll = torch.full_like(ref_ll, float("nan"))
        am = None if labelled else torch.full_like(ref_am, -7)
        assert _call_static(lib, pi, A, B, seqs, ll, am, precision) == hmm.HMM_OK, \
            hmm.hmm_last_error()
        torch.cuda.synchronize()
        # the same kernels on the same inputs: bit for bit (NaN-free above)
        assert torch.equal(ll, ref_ll)
        if not labelled:
            assert torch.equal(am, ref_am)
    # and within the parity tolerance of the log-likelihood, a fortiori
    tol = torch.from_numpy(ll_tol(w.lengths)).float().cuda()
    assert bool(((ll - ref_ll).abs() <= (tol if labelled else tol[:, None])).all())


@pytest.mark.gpu
@pytest.mark.parametrize("labelled", [False, True])
@pytest.mark.parametrize("n_seqs", [300, 6000])  # 6000: the setup plan over many blocks
def test_static_scratch_matches_workspace_entry_point(labelled, n_seqs):
    w = synth.make_workload("batched", n_seqs=n_seqs, lengths=("uniform", 0, 300))
    _twice_equal(hmm.lib(), w, labelled, hmm.HMM_FP32)


@pytest.mark.gpu
def test_static_scratch_tensor_core_forward():
    """N = 128, M = 256 on the BF16 tensor cores (every sequence against every
    model; the padded tables take the scratch)."""
    w = synth.make_workload("large", n_seqs=300, lengths=("uniform", 1, 400), K=4)
    _twice_equal(hmm.lib(), w, False, hmm.HMM_BF16_MMA)


@pytest.mark.gpu
def test_static_scratch_parallel_in_time_branch():
    """Two long sequences, N = 32: HMM_AUTO takes the parallel-in-time
    forward, whose chunk products (about 1 MB here) fit the fixed array."""
    w = synth.make_workload("longseq", n_seqs=2, lengths=("uniform", 8000, 8192), K=2)
    seqs, _, _, _ = to_gpu(w)
    c = seqs.c()
    dims = hmm.hmm_dims_t(w.K, w.N, w.M)
    need_scan = ctypes.c_size_t()
    assert hmm.lib().hmm_forward_scan_workspace_size(dims, ctypes.byref(c), 0,
                                                     ctypes.byref(need_scan)) == 0
    assert need_scan.value <= hmm_static_bytes()
    assert hmm.hmm_workspace_size(dims, seqs, hmm.HMM_OP_FORWARD) >= need_scan.value
    _twice_equal(hmm.lib(), w, False, hmm.HMM_AUTO)


@pytest.mark.gpu
def test_static_scratch_refuses_oversized_requests():
    import torch
    lib = hmm.lib()
    rng = np.random.default_rng(0)
    pi, A, B = (torch.from_numpy(x).cuda() for x in synth.random_model(rng, 4, 8, 16))
    # 2^21 sequences need about 24 MiB of scratch: refused before any launch
    S = 1 << 21
    c = hmm.hmm_seqs_t(0x10000, 0x20000, 0x30000, None, S, 10, 10 * S)
    dims = hmm.hmm_dims_t(4, 8, 16)
    out = ctypes.c_size_t()
    assert lib.hmm_workspace_size(dims, ctypes.byref(c), hmm.HMM_OP_FORWARD, ctypes.byref(out)) == 0
    assert out.value > hmm_static_bytes()
    rc = lib.hmm_forward_static(dims, pi.data_ptr(), A.data_ptr(), B.data_ptr(), ctypes.byref(c),
                                hmm.HMM_FP32, 0x40000, None, None)
    assert rc == hmm.HMM_ERR_WORKSPACE and "scratch" in hmm.hmm_last_error()


def hmm_static_bytes():
    with open(hmm.HEADER) as f:
        for line in f:
            if line.startswith("#define HMM_STATIC_SCRATCH_BYTES"):
                return eval(line.split(None, 2)[2])
    raise AssertionError("HMM_STATIC_SCRATCH_BYTES not declared")
