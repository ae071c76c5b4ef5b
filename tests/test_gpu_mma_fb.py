"""Tensor-core (BF16 tcgen05) forward-backward adjoint vs the FP64 oracle.

The tensor-core adjoint rounds A and B (once per call), the rescaled forward
variable, the backward messages Y and gamma to BF16 (unit roundoff u = 2^-8)
and accumulates every product in FP32. Checks:

* log-likelihoods: phase 1 is the tensor-core forward recursion, so the same
  hard bound |delta log P| <= 3 u T (+ the FP32 bound) holds against the exact
  model;
* log-likelihoods also within the per-sequence cap (u / 4) T + 2 u of the
  forward tests, and their mean error per observation against the oracle run
  on A and B rounded to BF16 below u / 8 (the forward's check);
* counts (against the oracle on the model as the kernel holds it, A and B
  rounded, so that the bound covers the per-step rounding of the messages):
  every count term is a product of a normalised forward and backward
  message and, for xi, one BF16 transition; the normalisation is re-measured
  every step, so the per-term relative error stays O(u) instead of growing
  with T: every entry within u (1 + |ref|) (an expected count is a number of
  visits: 1 is its absolute unit) and the relative L2 error of each count
  tensor within u (measured values are printed); the sums over the counts are invariant
  (sum C_A = sum_s w_s (T_s - 1), sum C_B = sum_s w_s T_s, sum C_pi =
  sum_s w_s per model) to within u relative;
* bitwise reproducibility across calls (fixed tile composition and order).
"""
import numpy as np
import pytest

import oracle
from helpers import check_counts, ll_tol, oparams, rel_l2, to_gpu
from test_gpu_mma import held_model, seq_cap
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8

CASES = [
    # name, n_seqs, lengths, overrides: N=128/M=256, N=64/M=128, padded N, odd M,
    # tiles with ragged tails, sequences crossing several checkpoint segments
    ("large", 150, ("uniform", 1, 300), {"K": 2}),
    ("training", 300, ("uniform", 1, 400), {"K": 3}),
    ("training", 140, ("uniform", 50, 1000), {"K": 2}),
    ("large", 90, ("uniform", 1, 200), {"K": 3, "N": 100, "M": 200}),
    ("gradient", 200, ("uniform", 1, 150), {"K": 4, "N": 40, "M": 70}),
]


def _workload(case):
    name, S, lengths, over = case
    return synth.make_workload(name, n_seqs=S, lengths=lengths, **over)


def _run(w, labelled=True, weights=None):
    import torch
    seqs, pi, A, B = to_gpu(w, labelled=labelled)
    wt = None if weights is None else torch.from_numpy(weights).cuda()
    out = hmm.hmm_forward_backward(pi, A, B, seqs, weight=wt, precision=hmm.HMM_BF16_MMA)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_bf16_adjoint_labelled_matches_oracle(case):
    w = _workload(case)
    wts = np.random.default_rng(5).uniform(0.5, 2.0, size=w.S).astype(np.float32)
    ll, cpi, cA, cB = _run(w, True, wts)
    # counts against the model the kernel holds (A and B rounded to BF16):
    # the per-step rounding of the messages is what they must bound
    rll_r, rpi, rA, rB, _ = oracle.forward_backward(held_model(w, "bf16"), w.symbols, w.offsets,
                                                    w.lengths, w.labels, wts.astype(np.float64),
                                                    nthreads=8)
    # log-likelihoods against the exact model
    rll, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths, w.labels, nthreads=8)
    T = np.maximum(w.lengths, 1).astype(np.float64)
    err = np.abs(ll - rll)
    assert np.all(err <= 3 * U_BF16 * T + ll_tol(w.lengths)), (err / T).max()
    assert np.all(err <= seq_cap(U_BF16, w.lengths)), (err / seq_cap(U_BF16, w.lengths)).max()
    mean_r = np.mean(np.abs(ll - rll_r) / T)
    assert mean_r <= U_BF16 / 8 + 1e-5, mean_r
    errs = [rel_l2(g, r) for g, r in zip((cpi, cA, cB), (rpi, rA, rB))]
    worst = check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=U_BF16, what=case[0])
    print(f"{case[0]} N={w.N} M={w.M}: loglik max|d|/T {np.max(err / T):.2e} "
          f"(mean vs rounded model {mean_r:.2e}); count rel L2 pi {errs[0]:.2e} A {errs[1]:.2e} "
          f"B {errs[2]:.2e}; worst |d|/(1+|ref|) {max(worst):.2e}")
    # invariants per model
    for k in range(w.K):
        sel = w.labels == k
        wk = wts[sel].astype(np.float64)
        Tk = w.lengths[sel].astype(np.float64)
        live = Tk > 0
        assert abs(cpi[k].sum() - wk[live].sum()) <= U_BF16 * max(1.0, wk.sum())
        assert abs(cA[k].sum() - (wk * np.maximum(Tk - 1, 0)).sum()) <= U_BF16 * max(1.0, (wk * Tk).sum())
        assert abs(cB[k].sum() - (wk * Tk).sum()) <= U_BF16 * max(1.0, (wk * Tk).sum())
    # the logit gradient built from the counts: g = C - p rowsum(C) cancels,
    # so its error is bounded on the scale of the counts,
    # |dg| <= |dC| + |p| |d rowsum C| <= 2 |dC|
    import torch
    t = [torch.from_numpy(x).cuda() for x in (w.pi, w.A, w.B)]
    g = hmm.hmm_softmax_grad(*t, *(torch.from_numpy(x).cuda() for x in (cpi, cA, cB)))
    rg = oracle.softmax_grad(oparams(w), rpi, rA, rB)
    for a, b, r, e in zip(g, rg, (rpi, rA, rB), errs):
        assert np.linalg.norm(a.cpu().numpy() - b) <= 2 * max(e, U_BF16 / 16) * np.linalg.norm(r)


@pytest.mark.parametrize("case", CASES[:2], ids=lambda c: f"{c[0]}-{c[1]}")
def test_bf16_adjoint_all_models_signed_weights(case):
    w = _workload(case)
    rng = np.random.default_rng(6)
    wts = rng.uniform(-1.0, 1.0, size=(w.S, w.K)).astype(np.float32)
    wts[rng.random(size=wts.shape) < 0.1] = 0.0  # zero weights drop out
    ll, cpi, cA, cB = _run(w, False, wts)
    hm = held_model(w, "bf16")
    rll, rpi, rA, rB, _ = oracle.forward_backward(hm, w.symbols, w.offsets, w.lengths,
                                                  None, wts.astype(np.float64), nthreads=8)
    T = np.maximum(w.lengths, 1).astype(np.float64)[:, None]
    assert np.all(np.abs(ll - rll) <= 2 * U_BF16 * T + ll_tol(w.lengths)[:, None])
    # signed weights: compare on the scale of the unsigned totals
    _, upi, uA, uB, _ = oracle.forward_backward(hm, w.symbols, w.offsets, w.lengths,
                                                None, np.abs(wts).astype(np.float64), nthreads=8)
    for g, r, u in zip((cpi, cA, cB), (rpi, rA, rB), (upi, uA, uB)):
        assert np.linalg.norm(g - r) <= U_BF16 * np.linalg.norm(u), np.linalg.norm(g - r) / np.linalg.norm(u)
    check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=U_BF16, scale=(upi, uA, uB), what="signed")


def test_bf16_adjoint_rows_longer_than_the_first_row_of_their_tile():
    """Lengths 256..263 share one scheduler length bucket, so rows within a
    tile are not in exact length order: every row must still run to its end."""
    w = synth.make_workload("training", n_seqs=300, lengths=("uniform", 256, 263), K=1)
    ll, cpi, cA, cB = _run(w, True)
    rll, rpi, rA, rB, _ = oracle.forward_backward(held_model(w, "bf16"), w.symbols, w.offsets,
                                                  w.lengths, w.labels, nthreads=8)
    T = w.lengths.astype(np.float64)
    assert np.all(np.abs(ll - rll) <= 2 * U_BF16 * T + ll_tol(w.lengths))
    assert np.all(np.abs(ll - rll) <= seq_cap(U_BF16, w.lengths))
    check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=U_BF16, what="same-bucket rows")


def test_bf16_adjoint_deterministic_repeat():
    w = synth.make_workload("training", n_seqs=700, lengths=("uniform", 1, 300), K=4)
    a = _run(w, True)
    b = _run(w, True)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_bf16_adjoint_degenerate_and_errors():
    import torch
    rng = np.random.default_rng(8)
    K, N, M = 2, 70, 6
    pi, A, B = synth.random_model(rng, K, N, M)
    # an impossible symbol for model 1: state emissions of symbol 5 all zero
    B[1, :, 5] = 0.0
    B[1] /= B[1].sum(axis=1, keepdims=True)
    seqs_l = [rng.integers(0, 5, size=T).tolist() for T in (0, 1, 2, 129, 3, 17, 40)]
    seqs_l[2] = [0, 9]          # bad symbol
    seqs_l[5][3] = 5            # impossible under model 1
    labels = np.array([0, 1, 0, 1, 0, 1, 0], np.int32)
    lengths = np.array([len(x) for x in seqs_l], np.int32)
    offsets = np.zeros(len(seqs_l), np.int64)
    offsets[1:] = np.cumsum(lengths)[:-1]
    sym = np.array([x for q in seqs_l for x in q], np.int32)
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths, model_of_seq=labels)
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    ll, cpi, cA, cB = hmm.hmm_forward_backward(*t, seqs, precision=hmm.HMM_BF16_MMA)
    ll = ll.cpu().numpy()
    assert hmm.hmm_get_device_status(hmm.default_workspace()) & hmm.HMM_STATUS_SYMBOL
    assert ll[0] == 0.0 and np.isnan(ll[2]) and ll[5] == -np.inf
    ok = np.array([0, 1, 3, 4, 6])
    rll, rpi, rA, rB, _ = oracle.forward_backward(oracle.params(pi, A, B), sym, offsets[ok],
                                                  lengths[ok], labels[ok], nthreads=4)
    assert np.all(np.abs(ll[ok] - rll) <= 3 * U_BF16 * np.maximum(lengths[ok], 1) + 1e-3)
    check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=U_BF16, what="degenerate")
    # small N is not served by the tensor-core adjoint; M above 256 neither
    small = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 2, 16, 5)]
    with pytest.raises(hmm.HmmError):
        hmm.hmm_forward_backward(*small, seqs, precision=hmm.HMM_BF16_MMA)
    wide = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 2, 70, 300)]
    with pytest.raises(hmm.HmmError):
        hmm.hmm_forward_backward(*wide, seqs, precision=hmm.HMM_BF16_MMA)


def test_bf16_adjoint_full_training_size_invariants():
    """The training configuration at full size (65536 sequences, K=20, N=64,
    M=128) in the launch configuration the bench times: sampled
    log-likelihoods against the oracle and the count invariants."""
    w = synth.make_workload("training")
    ll, cpi, cA, cB = _run(w, True)
    assert np.all(np.isfinite(ll))
    idx = np.random.default_rng(9).choice(w.S, size=48, replace=False)
    rll, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets[idx], w.lengths[idx],
                               w.labels[idx], nthreads=8)
    T = np.maximum(w.lengths[idx], 1).astype(np.float64)
    assert np.all(np.abs(ll[idx] - rll) <= 3 * U_BF16 * T + ll_tol(w.lengths[idx]))
    for k in range(w.K):
        Tk = w.lengths[w.labels == k].astype(np.float64)
        assert abs(cpi[k].sum() - (Tk > 0).sum()) <= U_BF16 * max(1.0, Tk.size)
        assert abs(cA[k].sum() - np.maximum(Tk - 1, 0).sum()) <= U_BF16 * Tk.sum()
        assert abs(cB[k].sum() - Tk.sum()) <= U_BF16 * Tk.sum()
        assert np.all(cA[k] >= 0) and np.all(cB[k] >= 0)
