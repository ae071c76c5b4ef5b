"""Shared test helpers: moving seeded workloads to the GPU, running the
oracle on the same inputs, and the tolerances of the parity checks.

Tolerances (written here once, used by every parity test):
  * log-likelihoods and Viterbi scores: |delta| <= 1e-4 * max(T, 1) nats
    (the FP32 bound stated for the method);
  * expected counts and logit gradients: relative L2 error per tensor
    <= 1e-4, elementwise |delta| <= 1e-4 * (1 + |ref|) * scale for sampled
    entries;
  * Viterbi paths: bit-exact on inputs whose best path beats the second best
    by more than 1e-3 nats.
"""
import numpy as np

import oracle
from paper_1310_3322_gb300 import synth

LL_TOL = 1e-4
COUNT_RTOL = 1e-4
PATH_MARGIN = 1e-3


def ll_tol(lengths):
    return LL_TOL * np.maximum(np.asarray(lengths, np.float64), 1.0)


def to_gpu(w, device="cuda", labelled=False):
    import torch
    from paper_1310_3322_gb300 import hmm
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths,
                                    model_of_seq=w.labels if labelled else None, device=device)
    pi, A, B = (torch.from_numpy(np.ascontiguousarray(x)).to(device) for x in (w.pi, w.A, w.B))
    return seqs, pi, A, B


def oparams(w):
    return oracle.params(w.pi, w.A, w.B)


def rel_l2(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def margin_filtered(w, labelled=False, rounds=8, nthreads=8):
    """Redraws sequences whose decoded path is not unique by more than
    PATH_MARGIN nats (or, in all-models mode, whose best model is not ahead of
    the runner-up by more than the score tolerance), until none is left."""
    for rnd in range(rounds):
        P = oparams(w)
        mos = w.labels if labelled else None
        score, best, _, margin, _ = oracle.viterbi(P, w.symbols, w.offsets, w.lengths, mos,
                                                   want_path=False, nthreads=nthreads)
        bad = ~(margin > PATH_MARGIN)
        if not labelled and w.K > 1:
            srt = np.sort(score, axis=1)
            gap = srt[:, -1] - srt[:, -2]
            bad |= ~(gap > 2 * ll_tol(w.lengths))
        bad &= w.lengths > 0
        idx = np.nonzero(bad)[0]
        if idx.size == 0:
            return w
        w = synth.resample(w, idx, rnd)
    raise AssertionError(f"{idx.size} sequences still within the path margin")
