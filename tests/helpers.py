"""Shared test helpers: moving seeded workloads to the GPU, running the
oracle on the same inputs, and the tolerances of the parity checks.

Tolerances (written here once, used by every parity test):
  * log-likelihoods and Viterbi scores: |delta| <= 1e-4 * max(T, 1) nats
    (the FP32 bound stated for the method);
  * expected counts: every entry |delta| <= 1e-4 * (1 + |ref|) -- an
    expected count is a number of visits, so 1 is its natural absolute unit
    and large counts are held to 1e-4 relative -- and the relative L2 error
    per tensor <= 1e-4 (for signed weights |ref| is replaced by the count
    under |weights|, the scale the cancelling terms came from); logit
    gradients g = C - p rowsum(C) inherit the bound of the counts they are
    built from (check_grads);
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


def check_counts(got, ref, rtol=COUNT_RTOL, scale=None, what=""):
    """Element-wise and relative-L2 comparison of (cnt_pi, cnt_A, cnt_B).
    `scale`: the same counts under unsigned weights (signed-weight runs).
    Returns the worst |delta| / (1 + |scale|) per tensor."""
    worst = []
    scale = ref if scale is None else scale
    for g, r, u, name in zip(got, ref, scale, ("pi", "A", "B")):
        g = np.asarray(g.cpu().numpy() if hasattr(g, "cpu") else g, np.float64)
        r = np.asarray(r, np.float64)
        ratio = np.abs(g - r) / (1.0 + np.abs(np.asarray(u, np.float64)))
        i = np.unravel_index(np.argmax(ratio), ratio.shape)
        assert ratio[i] <= rtol, (f"{what} cnt_{name}{list(i)}: got {g[i]} ref {r[i]} "
                                  f"(|d|/(1+|ref|) = {ratio[i]:.3e} > {rtol:.3e})")
        if scale is ref:
            e = rel_l2(g, r)
            assert e <= rtol, f"{what} cnt_{name}: rel L2 {e:.3e} > {rtol:.3e}"
        worst.append(float(ratio[i]))
    return worst


def check_grads(grads, ref_grads, counts, probs, rtol=COUNT_RTOL, what=""):
    """Logit gradients g = C - p * rowsum(C) against the oracle's: with every
    count within rtol (1 + |C|), |dg_ij| <= rtol ((1 + |C_ij|) + p_ij sum_j (1 + |C_ij|))."""
    for g, rg, c, p, name in zip(grads, ref_grads, counts, probs, ("pi", "A", "B")):
        g = np.asarray(g.cpu().numpy() if hasattr(g, "cpu") else g, np.float64)
        c = np.abs(np.asarray(c, np.float64))
        p = np.asarray(p, np.float64)
        row = (1.0 + c).sum(axis=-1, keepdims=True)
        bound = rtol * ((1.0 + c) + p * row)
        err = np.abs(g - np.asarray(rg, np.float64))
        i = np.unravel_index(np.argmax(err / bound), err.shape)
        assert err[i] <= bound[i], f"{what} g_{name}{list(i)}: |d| {err[i]:.3e} > {bound[i]:.3e}"


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
