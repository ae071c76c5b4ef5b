"""Adjoint (Baum-Welch E-step) above 128 states vs the FP64 oracle.

Above 128 states the forward and the backward recursions run on the tensor
cores (BF16 operands and BF16-rounded A and B, u = 2^-8, FP32 accumulation)
and keep every step's
rescaled rows; gamma and xi are formed from them with a per-step
normalisation and summed by a fixed-order contraction over all steps. As for
the adjoint up to 128 states: |delta log P| <= 3 u T, relative L2 error of
each count tensor <= u, count totals invariant to within u, bitwise
reproducible. Plus the degenerate cases (T = 0, 1, 2, an invalid symbol, an
impossible sequence) and the argument checks of the path.
"""
import numpy as np
import pytest

import oracle
from helpers import check_counts, ll_tol, oparams, rel_l2, to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8

CASES = [
    # name, n_seqs, lengths, overrides: 512 padded states (K = 1, the 512-state
    # shape), 300 states (padding inside the last 256-column block), 200
    # states (256 padded), several models
    ("cuhmm", 24, ("uniform", 1, 90), {}),
    ("cuhmm", 30, ("uniform", 1, 60), {"K": 2, "N": 300, "M": 32}),
    ("cuhmm", 50, ("uniform", 1, 120), {"K": 3, "N": 200, "M": 48}),
    # many short sequences: 64- and 128-row tiles of the cluster passes
    ("cuhmm", 700, ("uniform", 1, 10), {"K": 1, "N": 256, "M": 32}),
    ("cuhmm", 1300, ("uniform", 1, 8), {"K": 1, "N": 256, "M": 32}),
    # 512 padded states with more symbols than a state-by-symbol table in
    # shared memory would hold; three symbols: buckets of several pieces
    ("cuhmm", 40, ("uniform", 1, 50), {"K": 2, "N": 400, "M": 160}),
    ("cuhmm", 40, ("uniform", 50, 150), {"K": 1, "N": 256, "M": 3}),
]


def _workload(case):
    name, S, lengths, over = case
    return synth.make_workload(name, n_seqs=S, lengths=lengths, **over)


def _run(w, labelled, weights):
    import torch
    seqs, pi, A, B = to_gpu(w, labelled=labelled)
    wt = None if weights is None else torch.from_numpy(weights).cuda()
    out = hmm.hmm_forward_backward(pi, A, B, seqs, weight=wt, precision=hmm.HMM_BF16_MMA)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_wide_adjoint_all_models_matches_oracle(case):
    w = _workload(case)
    rng = np.random.default_rng(7)
    wts = rng.uniform(0.5, 2.0, size=(w.S, w.K)).astype(np.float32)
    ll, cpi, cA, cB = _run(w, False, wts)
    rll, rpi, rA, rB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets, w.lengths,
                                                  None, wts.astype(np.float64), nthreads=16)
    T = np.maximum(w.lengths, 1).astype(np.float64)[:, None]
    err = np.abs(ll - rll)
    assert np.all(err <= 3 * U_BF16 * T + ll_tol(w.lengths)[:, None]), (err / T).max()
    errs = [rel_l2(g, r) for g, r in zip((cpi, cA, cB), (rpi, rA, rB))]
    print(f"N={w.N} M={w.M} K={w.K}: loglik max|d|/T {np.max(err / T):.2e}; "
          f"count rel L2 pi {errs[0]:.2e} A {errs[1]:.2e} B {errs[2]:.2e}")
    assert max(errs) <= U_BF16, errs
    # totals per model: sum C_pi = sum w, sum C_A = sum w (T - 1), sum C_B = sum w T
    Tl = w.lengths.astype(np.float64)
    live = Tl > 0
    for k in range(w.K):
        wk = wts[:, k].astype(np.float64)
        tot = max(1.0, (wk * Tl).sum())
        assert abs(cpi[k].sum() - wk[live].sum()) <= U_BF16 * max(1.0, wk.sum())
        assert abs(cA[k].sum() - (wk * np.maximum(Tl - 1, 0)).sum()) <= U_BF16 * tot
        assert abs(cB[k].sum() - (wk * Tl).sum()) <= U_BF16 * tot


def test_wide_adjoint_labelled_single_model_and_signed_weights():
    w = _workload(CASES[0])
    rng = np.random.default_rng(8)
    wts = rng.uniform(-1.0, 1.0, size=w.S).astype(np.float32)
    wts[rng.random(w.S) < 0.15] = 0.0  # zero weights drop out
    ll, cpi, cA, cB = _run(w, True, wts)
    rll, rpi, rA, rB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets, w.lengths,
                                                  w.labels, wts.astype(np.float64), nthreads=16)
    assert ll.shape == (w.S,)
    assert np.all(np.abs(ll - rll) <= 3 * U_BF16 * np.maximum(w.lengths, 1) + ll_tol(w.lengths))
    _, upi, uA, uB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets, w.lengths,
                                                w.labels, np.abs(wts).astype(np.float64),
                                                nthreads=16)
    for g, r, u in zip((cpi, cA, cB), (rpi, rA, rB), (upi, uA, uB)):
        assert np.linalg.norm(g - r) <= U_BF16 * np.linalg.norm(u)


def test_wide_adjoint_deterministic_and_degenerate():
    import torch
    rng = np.random.default_rng(9)
    K, N, M = 2, 260, 16
    pi, A, B = synth.random_model(rng, K, N, M, alpha=0.5)
    B[1, :, 15] = 0.0  # model 1 never emits symbol 15
    B /= B.sum(axis=2, keepdims=True)
    lengths = np.array([0, 1, 2, 45, 3, 70, 30], np.int32)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    sym = rng.integers(0, 15, size=int(lengths.sum())).astype(np.int32)
    sym[offsets[5] + 33] = 15          # impossible under model 1 only
    bad = sym.copy()
    bad[offsets[3] + 20] = M + 2       # invalid symbol in sequence 3
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]

    def run(symbols):
        seqs = hmm.Sequences.from_numpy(symbols, offsets, lengths, device="cuda")
        return [x.cpu().numpy() for x in hmm.hmm_forward_backward(*t, seqs,
                                                                  precision=hmm.HMM_BF16_MMA)]

    a1, a2 = run(sym), run(sym)
    for x, y in zip(a1, a2):
        assert np.array_equal(x, y, equal_nan=True)
    ll, cpi, cA, cB = a1
    P = oracle.params(pi, A, B)
    rll, rpi, rA, rB, _ = oracle.forward_backward(P, sym, offsets, lengths, None, None,
                                                  nthreads=16)
    assert np.isneginf(ll[5, 1]) and np.isneginf(rll[5, 1])
    fin = np.isfinite(rll)
    assert np.array_equal(fin, np.isfinite(ll))
    Tm = np.broadcast_to(np.maximum(lengths, 1)[:, None], ll.shape)
    assert np.all(np.abs(ll[fin] - rll[fin]) <= 3 * U_BF16 * Tm[fin] + 1e-3)
    for g, r in zip((cpi, cA, cB), (rpi, rA, rB)):
        assert rel_l2(g, r) <= U_BF16
    # an invalid symbol: NaN log-likelihoods and no counts from that sequence
    ll_b, cpi_b, cA_b, cB_b = run(bad)
    st = hmm.hmm_get_device_status(hmm.default_workspace())
    assert st & hmm.HMM_STATUS_SYMBOL
    assert np.isnan(ll_b[3]).all()
    keep = np.array([0, 1, 2, 4, 5, 6])
    _, kpi, kA, kB, _ = oracle.forward_backward(P, sym, offsets[keep], lengths[keep], None, None,
                                                nthreads=16)
    for g, r in zip((cpi_b, cA_b, cB_b), (kpi, kA, kB)):
        assert rel_l2(g, r) <= U_BF16


def test_wide_adjoint_argument_checks():
    import torch
    rng = np.random.default_rng(10)
    lengths = np.array([5, 9], np.int32)
    offsets = np.array([0, 5], np.int64)
    sym = rng.integers(0, 8, size=14).astype(np.int32)
    labels = np.array([0, 1], np.int32)
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths, model_of_seq=labels, device="cuda")
    two = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 2, 300, 8)]
    with pytest.raises(hmm.HmmError):  # labelled pairs with K > 1 above 128 states
        hmm.hmm_forward_backward(*two, seqs, precision=hmm.HMM_BF16_MMA)
    big_m = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 1, 300, 200)]
    with pytest.raises(hmm.HmmError):  # emission slice beyond the cluster forward's shared memory
        hmm.hmm_forward_backward(*big_m, seqs.all_models(), precision=hmm.HMM_BF16_MMA)


def test_wide_adjoint_single_symbol_and_zero_weights():
    """One symbol (a model's rows all in one bucket of many pieces) and
    weights of zero (rows without entries), above 128 states."""
    import torch
    rng = np.random.default_rng(11)
    K, N, M, S = 1, 200, 1, 40
    pi, A, _ = synth.random_model(rng, K, N, 2)
    B = np.ones((K, N, M), np.float32)
    lengths = rng.integers(1, 120, size=S).astype(np.int32)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    sym = np.zeros(int(lengths.sum()), np.int32)
    wts = rng.uniform(0.5, 2.0, size=(S, K)).astype(np.float32)
    wts[rng.random(S) < 0.3] = 0.0
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths, device="cuda")
    out = hmm.hmm_forward_backward(*t, seqs, weight=torch.from_numpy(wts).cuda(),
                                   precision=hmm.HMM_BF16_MMA)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    ll, cpi, cA, cB = [x.cpu().numpy() for x in out]
    rll, rpi, rA, rB, _ = oracle.forward_backward(oracle.params(pi, A, B), sym, offsets, lengths,
                                                  None, wts.astype(np.float64), nthreads=16)
    # one symbol of probability 1: log P is 0 up to the rounding of A
    T = np.maximum(lengths, 1).astype(np.float64)[:, None]
    assert np.all(np.abs(ll - rll) <= 3 * U_BF16 * T + ll_tol(lengths)[:, None])
    assert np.all(np.abs(rll) <= 1e-4)
    w0 = wts[:, 0].astype(np.float64)
    assert abs(cB[0].sum() - (w0 * lengths).sum()) <= U_BF16 * (w0 * lengths).sum()
    for g, r in zip((cpi, cA, cB), (rpi, rA, rB)):
        assert rel_l2(g, r) <= U_BF16
    zero = np.zeros_like(wts)
    out0 = hmm.hmm_forward_backward(*t, seqs, weight=torch.from_numpy(zero).cuda(),
                                    precision=hmm.HMM_BF16_MMA)
    for x in out0[1:]:
        assert not x.cpu().numpy().any()


def test_wide_adjoint_full_cuhmm_shape():
    """The 512-state x 512-sequence workload the Baum-Welch bench times
    (K = 1, N = 512, M = 64, T ~ U{100..500}): the E-step on the whole batch
    (sampled log-likelihoods against the oracle, count identities), and on a
    weighted subset holding the 12 longest sequences, element by element
    against the oracle's expected counts on the model the kernel holds (A and
    B rounded to BF16)."""
    import torch
    from test_gpu_mma import held_model, seq_cap
    w = synth.make_workload("cuhmm")
    seqs, pi, A, B = to_gpu(w)
    ll, cpi, cA, cB = (t.cpu().numpy() for t in
                       hmm.hmm_forward_backward(pi, A, B, seqs, precision=hmm.HMM_BF16_MMA))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    assert np.all(np.isfinite(ll))
    idx = np.random.default_rng(20).choice(w.S, size=8, replace=False)
    ref, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets[idx], w.lengths[idx], nthreads=16)
    T = w.lengths[idx].astype(np.float64)[:, None]
    assert np.all(np.abs(ll[idx] - ref) <= 3 * U_BF16 * T + ll_tol(w.lengths[idx])[:, None])
    Tl = w.lengths.astype(np.float64)
    assert abs(cpi[0].sum() - w.S) <= U_BF16 * w.S
    assert abs(cA[0].sum() - (Tl - 1).sum()) <= U_BF16 * Tl.sum()
    assert abs(cB[0].sum() - Tl.sum()) <= U_BF16 * Tl.sum()
    assert np.all(cA >= 0) and np.all(cB >= 0) and np.all(cpi >= 0)

    order = np.argsort(-w.lengths, kind="stable")
    sub = np.sort(np.concatenate([order[:12], np.random.default_rng(21).choice(
        order[12:], size=12, replace=False)]))
    wts = np.random.default_rng(22).uniform(0.5, 2.0, size=(sub.size, 1)).astype(np.float32)
    s2 = hmm.Sequences.from_numpy(w.symbols, w.offsets[sub], w.lengths[sub], device="cuda")
    ll2, spi, sA, sB = (t.cpu().numpy() for t in hmm.hmm_forward_backward(
        pi, A, B, s2, weight=torch.from_numpy(wts).cuda(), precision=hmm.HMM_BF16_MMA))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    rll, rpi, rA, rB, _ = oracle.forward_backward(held_model(w, "bf16"), w.symbols, w.offsets[sub],
                                                  w.lengths[sub], None, wts.astype(np.float64),
                                                  nthreads=16)
    assert np.all(np.abs(ll2 - rll) <= seq_cap(U_BF16, w.lengths[sub])[:, None])
    worst = check_counts((spi, sA, sB), (rpi, rA, rB), rtol=U_BF16, what="512 states")
    print(f"512 states, longest subset: worst |d|/(1+|ref|) pi {worst[0]:.2e} "
          f"A {worst[1]:.2e} B {worst[2]:.2e}")
