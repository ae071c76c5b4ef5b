"""Differentiable log-likelihood of the HMM recognition path.

``HMMLogLik.apply(logit_pi, logit_A, logit_B, seqs)`` returns log P(O_s | lambda)
with pi, A, B the row softmax of the logits. Its backward is the hand-written
forward-backward adjoint of the library: the weighted expected counts of the
E-step of Baum-Welch (Sec. 2.7) are exactly d(sum_s w_s log P)/d(log p), and
the softmax chain rule g = C - p * rowsum(C) maps them to the logits. Every
step runs in the CUDA library; torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import hmm


class HMMLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logit_pi, logit_A, logit_B, seqs: "hmm.Sequences"):
        pi, A, B = hmm.hmm_softmax_rows(logit_pi.contiguous(), logit_A.contiguous(),
                                        logit_B.contiguous())
        ll, _ = hmm.hmm_forward(pi, A, B, seqs, want_argmax=False)
        ctx.save_for_backward(pi, A, B)
        ctx.seqs = seqs
        return ll

    @staticmethod
    def backward(ctx, grad_ll):
        pi, A, B = ctx.saved_tensors
        _, cpi, cA, cB = hmm.hmm_forward_backward(pi, A, B, ctx.seqs,
                                                  weight=grad_ll.contiguous().float())
        g_pi, g_A, g_B = hmm.hmm_softmax_grad(pi, A, B, cpi, cA, cB)
        return g_pi, g_A, g_B, None


def loglik(logit_pi, logit_A, logit_B, seqs):
    return HMMLogLik.apply(logit_pi, logit_A, logit_B, seqs)
