"""Failure detection of the tensor-core kernels: bounded waits that give up.

Every per-step mbarrier wait of the tensor-core forward (N <= 128 and the
wide one above), and of the tensor-core adjoint, polls at most
hmm_set_wait_limit() times. A limit of zero polls makes every such wait give
up at once, while the matrix products it waits for are still in flight. The kernel must then set HMM_STATUS_TIMEOUT, wait for the matrix
products and copies it already started, free its tensor memory and return:
the call's outputs are invalid (NaN log-likelihoods for the rows it did not
finish), the device stays usable, and the next call with the default limit on
the same workspace returns exactly what a clean call returns.

Nothing here faults or hangs the GPU: a give-up is an ordinary return path.
"""
import numpy as np
import pytest

from helpers import to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

CASES = {
    # op, precision, workload overrides (small: a few tiles, a few hundred steps)
    "forward-bf16-n128": ("forward", hmm.HMM_BF16_MMA, ("large", 200, ("uniform", 20, 200), {"K": 2})),
    "forward-tf32-n64": ("forward", hmm.HMM_TF32_MMA, ("training", 300, ("uniform", 20, 200), {"K": 2})),
    "forward-bf16-n256": ("forward", hmm.HMM_BF16_MMA,
                          ("large", 130, ("uniform", 10, 60), {"K": 1, "N": 256, "M": 64})),
    "forward-bf16-n512": ("forward", hmm.HMM_BF16_MMA,
                          ("large", 130, ("uniform", 10, 60), {"K": 2, "N": 512, "M": 64})),
    "forward-bf16-n512-m200": ("forward", hmm.HMM_BF16_MMA,
                               ("large", 40, ("uniform", 10, 40), {"K": 1, "N": 512, "M": 200})),
    "adjoint-bf16-n64": ("adjoint", hmm.HMM_BF16_MMA, ("training", 300, ("uniform", 20, 200), {"K": 2})),
    "adjoint-bf16-n128": ("adjoint", hmm.HMM_BF16_MMA, ("large", 200, ("uniform", 20, 200), {"K": 2})),
    "adjoint-tf32-n128": ("adjoint", hmm.HMM_TF32_MMA, ("large", 200, ("uniform", 20, 200), {"K": 2})),
    "adjoint-bf16-n512": ("adjoint", hmm.HMM_BF16_MMA,
                          ("cuhmm", 130, ("uniform", 10, 60), {"K": 1, "M": 64})),
}


def _run(op, prec, seqs, lab, pi, A, B, ws):
    if op == "forward":
        ll, am = hmm.hmm_forward(pi, A, B, seqs, precision=prec, workspace=ws)
        return [ll]
    return list(hmm.hmm_forward_backward(pi, A, B, lab, precision=prec, workspace=ws))


@pytest.mark.parametrize("name", list(CASES))
def test_wait_limit_gives_up_then_next_call_is_exact(name):
    import torch
    op, prec, (wl, S, lengths, over) = CASES[name]
    w = synth.make_workload(wl, n_seqs=S, lengths=lengths, **over)
    seqs, pi, A, B = to_gpu(w)
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    ws = hmm.Workspace()
    ref = [t.cpu().numpy() for t in _run(op, prec, seqs, lab, pi, A, B, ws)]
    assert hmm.hmm_get_device_status(ws) == 0
    assert hmm.hmm_get_wait_limit() == 1 << 24
    try:
        hmm.hmm_set_wait_limit(0)
        assert hmm.hmm_get_wait_limit() == 0
        out = [t.cpu().numpy() for t in _run(op, prec, seqs, lab, pi, A, B, ws)]
        status = hmm.hmm_get_device_status(ws)
    finally:
        hmm.hmm_set_wait_limit(-1)
    assert hmm.hmm_get_wait_limit() == 1 << 24
    assert status & hmm.HMM_STATUS_TIMEOUT, f"status {status:#x}"
    # rows the kernel gave up on report NaN (rows it had finished keep their
    # value; tiles it never started keep whatever the buffer held)
    assert np.isnan(out[0]).any()
    # the device is still usable, and the same workspace gives the clean result
    again = [t.cpu().numpy() for t in _run(op, prec, seqs, lab, pi, A, B, ws)]
    assert hmm.hmm_get_device_status(ws) == 0
    for a, b in zip(again, ref):
        np.testing.assert_array_equal(a, b)
