"""Learning path on the GPU: row softmax, the autograd adjoint against the
oracle's gradient, the Adam kernel, and a short training loop."""
import numpy as np
import pytest

import oracle
from helpers import COUNT_RTOL, oparams, rel_l2
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu


def _logits(w):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda().requires_grad_(True) for x in w.logits]


def test_softmax_rows_matches_fp64():
    import torch
    w = synth.make_workload("gradient", n_seqs=4)
    lp = [torch.from_numpy(x).cuda() for x in w.logits]
    pi, A, B = hmm.hmm_softmax_rows(*lp)
    for got, x in zip((pi, A, B), w.logits):
        ref = oracle.softmax_rows(x)
        np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=2e-6, atol=1e-9)


def test_autograd_gradient_matches_oracle():
    from paper_1310_3322_gb300.autograd import loglik
    import torch
    w = synth.make_workload("gradient", n_seqs=120, lengths=("uniform", 20, 200))
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, model_of_seq=w.labels)
    lpi, lA, lB = _logits(w)
    ll = loglik(lpi, lA, lB, seqs)
    wts = torch.linspace(0.5, 1.5, w.S, device="cuda")
    (ll * wts).sum().backward()
    P = oracle.params(*(oracle.softmax_rows(x) for x in w.logits))
    _, cpi, cA, cB, _ = oracle.forward_backward(P, w.symbols, w.offsets, w.lengths, w.labels,
                                                wts.cpu().numpy().astype(np.float64), nthreads=8)
    gpi, gA, gB = oracle.softmax_grad(P, cpi, cA, cB)
    for got, ref in zip((lpi.grad, lA.grad, lB.grad), (gpi, gA, gB)):
        assert rel_l2(got.cpu().numpy(), ref) <= 10 * COUNT_RTOL
        np.testing.assert_allclose(got.sum(-1).cpu().numpy(), 0.0, atol=1e-3)


def test_adam_kernel_matches_reference():
    import torch
    rng = np.random.default_rng(0)
    n = 10007
    p0, g = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    p, gt = torch.from_numpy(p0.copy()).cuda(), torch.from_numpy(g).cuda()
    m, v = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    mr, vr, pr = np.zeros(n), np.zeros(n), p0.astype(np.float64)
    lr, b1, b2, eps, gs = 1e-2, 0.9, 0.999, 1e-8, -0.5
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    for step in (1, 2, 3):
        hmm.hmm_adam_step(p, gt, m, v, lr, b1, b2, eps, gs, counter)
        gg = gs * g.astype(np.float64)
        mr = b1 * mr + (1 - b1) * gg
        vr = b2 * vr + (1 - b2) * gg * gg
        pr = pr - lr * (mr / (1 - b1 ** step)) / (np.sqrt(vr / (1 - b2 ** step)) + eps)
    np.testing.assert_allclose(p.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    assert int(counter.item()) == 3


def test_training_steps_raise_likelihood():
    import torch
    w = synth.make_workload("gradient", n_seqs=256, lengths=("uniform", 50, 150))
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, model_of_seq=w.labels)
    # start from perturbed logits so there is something to learn
    rng = np.random.default_rng(1)
    lg = [torch.from_numpy((x + rng.standard_normal(x.shape).astype(np.float32))).cuda()
          for x in w.logits]
    state = [(torch.zeros_like(x), torch.zeros_like(x), torch.zeros(1, dtype=torch.int32,
                                                                     device="cuda")) for x in lg]
    first = None
    for step in range(1, 21):
        pi, A, B = hmm.hmm_softmax_rows(*lg)
        ll, cpi, cA, cB = hmm.hmm_forward_backward(pi, A, B, seqs)
        tot = float(ll.sum())
        first = tot if first is None else first
        grads = hmm.hmm_softmax_grad(pi, A, B, cpi, cA, cB)
        for x, gx, (m, v, c) in zip(lg, grads, state):
            hmm.hmm_adam_step(x, gx, m, v, 5e-2, grad_scale=-1.0 / float(w.lengths.sum()),
                              step_counter=c)
    assert tot > first + 1.0
