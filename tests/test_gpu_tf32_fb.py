"""TF32 tensor-core forward-backward adjoint (64 < N <= 128) vs the FP64 oracle.

The TF32 adjoint runs the forward and the backward recursion of every tile
with TF32 operands (A rounded to TF32 once per call, round to nearest, unit
roundoff u = 2^-11; the rows rounded to TF32 as MMA operands; B in FP32;
FP32 accumulation) and keeps every step's rows; the counts are formed from
the rows (gamma per row, xi as one contraction over all rows whose operands
are rounded to TF32). Checks:

* log-likelihoods: the forward is the TF32 tensor-core recursion, so the
  forward tests' hard bound |delta log P| <= 2 u T (+ the FP32 bound) holds
  against the exact model, and the mean error per observation against the
  oracle on A rounded to TF32 stays below u / 8;
* counts against the oracle on the model as the kernel holds it (A rounded):
  every entry within 2^-8 (1 + |ref|) and the relative L2 error of each count
  tensor within 2^-8 (each count term is a product of two normalised
  messages, each with O(u) relative error per step, and, for xi, two TF32
  roundings); the count sums are invariant per model;
* labelled sequences of several models (the rows of each model contiguous),
  every sequence against every model, weights, degenerate sequences, bitwise
  reproducibility, and the cases the path refuses.
"""
import numpy as np
import pytest

import oracle
from helpers import check_counts, ll_tol, oparams, rel_l2, to_gpu
from test_gpu_mma import tf32_round
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

U_TF32 = 2.0 ** -11
CNT_TOL = 2.0 ** -8

CASES = [
    # name, n_seqs, lengths, overrides: N = 128 / M = 256, padded N and odd M,
    # tiles with ragged tails, sequences over a thousand steps
    ("large", 150, ("uniform", 1, 300), {"K": 2}),
    ("large", 90, ("uniform", 1, 200), {"K": 3, "N": 100, "M": 200}),
    ("training", 120, ("uniform", 1, 400), {"K": 3, "N": 65, "M": 40}),
    ("large", 40, ("uniform", 600, 1200), {"K": 2}),
    # four symbols: every symbol's rows span many pieces of the emission sums
    ("large", 60, ("uniform", 200, 600), {"K": 2, "N": 128, "M": 4}),
]


def _workload(case):
    name, S, lengths, over = case
    return synth.make_workload(name, n_seqs=S, lengths=lengths, **over)


def held(w):
    return oracle.params(w.pi, tf32_round(w.A), w.B)


def _run(w, labelled=True, weights=None):
    import torch
    seqs, pi, A, B = to_gpu(w, labelled=labelled)
    wt = None if weights is None else torch.from_numpy(weights).cuda()
    out = hmm.hmm_forward_backward(pi, A, B, seqs, weight=wt, precision=hmm.HMM_TF32_MMA)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_tf32_adjoint_labelled_matches_oracle(case):
    w = _workload(case)
    wts = np.random.default_rng(15).uniform(0.5, 2.0, size=w.S).astype(np.float32)
    ll, cpi, cA, cB = _run(w, True, wts)
    rll_r, rpi, rA, rB, _ = oracle.forward_backward(held(w), w.symbols, w.offsets, w.lengths,
                                                    w.labels, wts.astype(np.float64), nthreads=8)
    rll, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths, w.labels, nthreads=8)
    T = np.maximum(w.lengths, 1).astype(np.float64)
    err = np.abs(ll - rll)
    assert np.all(err <= 2 * U_TF32 * T + ll_tol(w.lengths)), (err / T).max()
    mean_r = np.mean(np.abs(ll - rll_r) / T)
    assert mean_r <= U_TF32 / 8 + 1e-5, mean_r
    errs = [rel_l2(g, r) for g, r in zip((cpi, cA, cB), (rpi, rA, rB))]
    worst = check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=CNT_TOL, what=case[0])
    print(f"{case[0]} N={w.N} M={w.M} K={w.K}: loglik max|d|/T {np.max(err / T):.2e} "
          f"(mean vs rounded model {mean_r:.2e}); count rel L2 pi {errs[0]:.2e} A {errs[1]:.2e} "
          f"B {errs[2]:.2e}; worst |d|/(1+|ref|) {max(worst):.2e}")
    assert max(errs) <= CNT_TOL, errs
    for k in range(w.K):
        sel = w.labels == k
        wk = wts[sel].astype(np.float64)
        Tk = w.lengths[sel].astype(np.float64)
        live = Tk > 0
        tot = max(1.0, (wk * Tk).sum())
        assert abs(cpi[k].sum() - wk[live].sum()) <= CNT_TOL * max(1.0, wk.sum())
        assert abs(cA[k].sum() - (wk * np.maximum(Tk - 1, 0)).sum()) <= CNT_TOL * tot
        assert abs(cB[k].sum() - (wk * Tk).sum()) <= CNT_TOL * tot


def test_tf32_adjoint_all_models_weighted():
    w = _workload(CASES[1])
    wts = np.random.default_rng(16).uniform(0.5, 2.0, size=(w.S, w.K)).astype(np.float32)
    ll, cpi, cA, cB = _run(w, False, wts)
    assert ll.shape == (w.S, w.K)
    rll, rpi, rA, rB, _ = oracle.forward_backward(held(w), w.symbols, w.offsets, w.lengths, None,
                                                  wts.astype(np.float64), nthreads=8)
    T = np.maximum(w.lengths, 1).astype(np.float64)[:, None]
    assert np.all(np.abs(ll - rll) <= 2 * U_TF32 * T + ll_tol(w.lengths)[:, None])
    check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=CNT_TOL, what="all models")
    errs = [rel_l2(g, r) for g, r in zip((cpi, cA, cB), (rpi, rA, rB))]
    assert max(errs) <= CNT_TOL, errs


@pytest.mark.parametrize("labelled", [False, True])
def test_tf32_adjoint_degenerate_and_deterministic(labelled):
    import torch
    rng = np.random.default_rng(17)
    K, N, M = 2, 100, 16
    pi, A, B = synth.random_model(rng, K, N, M, alpha=0.5)
    B[1, :, 15] = 0.0  # model 1 never emits symbol 15
    B /= B.sum(axis=2, keepdims=True)
    lengths = np.array([0, 1, 2, 45, 3, 70, 30, 2], np.int32)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    sym = rng.integers(0, 15, size=int(lengths.sum())).astype(np.int32)
    sym[offsets[5] + 33] = 15          # impossible under model 1 only
    sym[offsets[6] + 7] = M + 3        # invalid symbol in sequence 6
    labels = np.array([0, 1, 0, 1, 1, 1, 0, 0], np.int32)
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths,
                                    model_of_seq=labels if labelled else None, device="cuda")

    def run():
        out = hmm.hmm_forward_backward(*t, seqs, precision=hmm.HMM_TF32_MMA)
        return [x.cpu().numpy() for x in out], hmm.hmm_get_device_status(hmm.default_workspace())

    (a1, st1), (a2, _) = run(), run()
    for x, y in zip(a1, a2):
        assert np.array_equal(x, y, equal_nan=True)
    assert st1 & hmm.HMM_STATUS_SYMBOL
    ll, cpi, cA, cB = a1
    ok = np.array([True, True, True, True, True, True, False, True])
    Pm = oracle.params(pi, tf32_round(A), B)
    keep = np.flatnonzero(ok)
    rll, rpi, rA, rB, _ = oracle.forward_backward(Pm, sym, offsets[keep], lengths[keep],
                                                  labels[keep] if labelled else None, None,
                                                  nthreads=8)
    if labelled:
        assert np.isnan(ll[6])
        assert np.isneginf(ll[5]) and np.isneginf(rll[keep.tolist().index(5)])
        fin = np.isfinite(rll)
        assert np.all(np.abs(ll[keep][fin] - rll[fin]) <= 2 * U_TF32 * np.maximum(lengths[keep][fin], 1) + 1e-3)
    else:
        assert np.all(np.isnan(ll[6]))
        assert np.isneginf(ll[5, 1]) and np.isfinite(ll[5, 0])
        fin = np.isfinite(rll)
        d = np.abs(ll[keep] - rll)
        cap = np.broadcast_to(2 * U_TF32 * np.maximum(lengths[keep], 1)[:, None] + 1e-3, d.shape)
        assert np.all(d[fin] <= cap[fin])
    # the invalid sequence contributes nothing; the rest as the oracle
    errs = [rel_l2(g, r) for g, r in zip((cpi, cA, cB), (rpi, rA, rB))]
    assert max(errs) <= CNT_TOL, errs


def test_tf32_adjoint_refusals():
    import torch
    rng = np.random.default_rng(18)
    small = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 2, 40, 8)]
    seqs = hmm.Sequences.from_numpy(np.zeros(10, np.int32), np.array([0, 5], np.int64),
                                    np.array([5, 5], np.int32), device="cuda")
    with pytest.raises(hmm.HmmError):  # N <= 64: the FP32 SIMT adjoint serves it
        hmm.hmm_forward_backward(*small, seqs, precision=hmm.HMM_TF32_MMA)
    wide = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 1, 200, 8)]
    with pytest.raises(hmm.HmmError):  # above 128 states: BF16 only
        hmm.hmm_forward_backward(*wide, seqs, precision=hmm.HMM_TF32_MMA)
    many = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 1, 100, 257)]
    with pytest.raises(hmm.HmmError):  # M <= 256, as the tensor-core adjoint
        hmm.hmm_forward_backward(*many, seqs, precision=hmm.HMM_TF32_MMA)


def test_tf32_adjoint_empty_model_single_symbol_zero_weights():
    """Emission sums over the symbol sort: a model no sequence is labelled
    with (no rows, no chunks), a model whose sequences all carry weight 0
    (rows but no entries), and one symbol (every row of a model in one
    bucket, spread over many pieces)."""
    import torch
    rng = np.random.default_rng(19)
    K, N, M, S = 3, 90, 1, 70
    pi, A, _ = synth.random_model(rng, K, N, 2)
    B = np.ones((K, N, M), np.float32)
    lengths = rng.integers(1, 260, size=S).astype(np.int32)
    lengths[:3] = (0, 1, 2)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    sym = np.zeros(int(lengths.sum()), np.int32)
    labels = np.where(rng.random(S) < 0.5, 0, 2).astype(np.int32)
    wts = rng.uniform(0.5, 2.0, size=S).astype(np.float32)
    wts[labels == 2] = 0.0
    wts[rng.random(S) < 0.2] = 0.0
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths, model_of_seq=labels, device="cuda")
    out = hmm.hmm_forward_backward(*t, seqs, weight=torch.from_numpy(wts).cuda(),
                                   precision=hmm.HMM_TF32_MMA)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    ll, cpi, cA, cB = [x.cpu().numpy() for x in out]
    Pm = oracle.params(pi, tf32_round(A), B)
    rll, rpi, rA, rB, _ = oracle.forward_backward(Pm, sym, offsets, lengths, labels,
                                                  wts.astype(np.float64), nthreads=8)
    # one symbol of probability 1: log P is 0 up to the rounding of A
    T = np.maximum(lengths, 1).astype(np.float64)
    assert np.all(np.abs(ll - rll) <= 2 * U_TF32 * T + ll_tol(lengths))
    assert np.all(np.abs(ll) <= 2 * U_TF32 * T + ll_tol(lengths))
    for k in (1, 2):  # no sequence; only zero weights
        assert not cpi[k].any() and not cA[k].any() and not cB[k].any()
    live = (labels == 0) & (lengths > 0) & (wts != 0)
    Tl = lengths.astype(np.float64)
    assert abs(cpi[0].sum() - wts[live].sum()) <= CNT_TOL * wts[live].sum()
    assert abs(cB[0].sum() - (wts[live] * Tl[live]).sum()) <= CNT_TOL * (wts[live] * Tl[live]).sum()
    check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=CNT_TOL, what="empty model")
    errs = [rel_l2(g, r) for g, r in zip((cpi, cA, cB), (rpi, rA, rB))]
    assert max(errs) <= CNT_TOL, errs
