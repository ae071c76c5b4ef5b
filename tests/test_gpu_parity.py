"""GPU path vs the FP64 oracle, element by element, through the C-ABI.

Sizes are ones the oracle finishes in seconds while still spanning many warps
and work items with ragged tails; every instantiated lane count (the tuning
candidates) is exercised, and padded state counts (N not a power of two) are
covered. Tolerances are in tests/helpers.py.
"""
import numpy as np
import pytest

import oracle
from helpers import check_counts, check_grads, ll_tol, margin_filtered, oparams, to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

CASES = [
    # name, n_seqs, lengths, K/N/M overrides
    ("plain", 64, None, {}),
    ("plain", 300, ("uniform", 0, 90), {"N": 3, "M": 5}),
    ("batched", 160, ("uniform", 30, 300), {}),
    ("batched", 150, ("uniform", 1, 200), {"N": 13, "K": 3}),
    ("gradient", 70, ("uniform", 50, 500), {}),
    ("gradient", 90, ("uniform", 1, 120), {"N": 27, "M": 11}),
    ("training", 40, ("uniform", 20, 200), {"K": 5}),
    ("plain", 200, ("uniform", 1, 64), {"N": 7, "K": 4, "M": 3}),
    # above 32 states the FP32 SIMT kernels hold 64 padded states per pair
    ("gradient", 60, ("uniform", 1, 150), {"N": 40, "M": 20, "K": 3}),
    ("training", 48, ("uniform", 1, 200), {"K": 3}),
]


def _workload(case):
    name, S, lengths, over = case
    return synth.make_workload(name, n_seqs=S, lengths=lengths, **over)


def _npad(N):
    for p in (4, 8, 16, 32, 64):
        if N <= p:
            return p


@pytest.fixture(autouse=True)
def _reset_tuning():
    yield
    for op in (0, 1, 2, 3, hmm.HMM_TUNE_FB_RANGES):
        for n in (4, 8, 16, 32, 64):
            hmm.hmm_set_tuning(op, n, 0)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_forward_all_models(case):
    w = _workload(case)
    seqs, pi, A, B = to_gpu(w)
    ref, ref_am, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths, nthreads=8)
    tol = ll_tol(w.lengths)[:, None]
    for G in hmm.hmm_tuning_candidates(hmm.HMM_OP_FORWARD, _npad(w.N)):
        hmm.hmm_set_tuning(hmm.HMM_OP_FORWARD, _npad(w.N), G)
        ll, am = hmm.hmm_forward(pi, A, B, seqs)
        ll, am = ll.cpu().numpy(), am.cpu().numpy()
        err = np.abs(ll - ref)
        assert np.all(err <= tol), f"G={G}: max err {err.max()} at {np.unravel_index(err.argmax(), err.shape)}"
        # the argmax must agree wherever the top two models are separated
        srt = np.sort(ref, axis=1)
        clear = (srt[:, -1] - srt[:, -2] > 2 * tol[:, 0]) if w.K > 1 else np.ones(w.S, bool)
        np.testing.assert_array_equal(am[clear], ref_am[clear])
        assert np.all((am >= 0) & (am < w.K))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_forward_labelled(case):
    w = _workload(case)
    seqs, pi, A, B = to_gpu(w, labelled=True)
    ref, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths, w.labels)
    ll, am = hmm.hmm_forward(pi, A, B, seqs)
    assert am is None
    assert np.all(np.abs(ll.cpu().numpy() - ref) <= ll_tol(w.lengths))


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_viterbi_scores_and_paths(case):
    w = margin_filtered(_workload(case))
    seqs, pi, A, B = to_gpu(w)
    rs, rbest, rpath, _, _ = oracle.viterbi(oparams(w), w.symbols, w.offsets, w.lengths,
                                            nthreads=8)
    tol = ll_tol(w.lengths)[:, None]
    gs = hmm.hmm_tuning_candidates(hmm.HMM_OP_VITERBI, _npad(w.N))
    gp = hmm.hmm_tuning_candidates(hmm.HMM_TUNE_VITERBI_PATHS, _npad(w.N))
    for i in range(max(len(gs), len(gp))):
        G = gs[i % len(gs)]
        hmm.hmm_set_tuning(hmm.HMM_OP_VITERBI, _npad(w.N), G)
        hmm.hmm_set_tuning(hmm.HMM_TUNE_VITERBI_PATHS, _npad(w.N), gp[i % len(gp)])
        sc, best, path = hmm.hmm_viterbi(pi, A, B, seqs)
        sc, best, path = sc.cpu().numpy(), best.cpu().numpy(), path.cpu().numpy()
        err = np.abs(sc - rs)
        assert np.all(err <= tol), f"G={G}: max err {err.max()}"
        np.testing.assert_array_equal(best, rbest)
        np.testing.assert_array_equal(path, rpath)


@pytest.mark.parametrize("case", CASES[:6], ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_viterbi_labelled(case):
    w = margin_filtered(_workload(case), labelled=True)
    seqs, pi, A, B = to_gpu(w, labelled=True)
    rs, rbest, rpath, _, _ = oracle.viterbi(oparams(w), w.symbols, w.offsets, w.lengths, w.labels)
    for Gp in hmm.hmm_tuning_candidates(hmm.HMM_TUNE_VITERBI_PATHS, _npad(w.N)):
        hmm.hmm_set_tuning(hmm.HMM_TUNE_VITERBI_PATHS, _npad(w.N), Gp)
        sc, best, path = hmm.hmm_viterbi(pi, A, B, seqs)
        assert np.all(np.abs(sc.cpu().numpy() - rs) <= ll_tol(w.lengths))
        np.testing.assert_array_equal(best.cpu().numpy(), w.labels)
        np.testing.assert_array_equal(path.cpu().numpy(), rpath)
    # scores only (no path) take the score kernel
    sc2, _, _ = hmm.hmm_viterbi(pi, A, B, seqs, want_path=False)
    np.testing.assert_array_equal(sc2.cpu().numpy(), sc.cpu().numpy())


# every case the FP32 SIMT adjoint accepts (N <= 64)
FB_CASES = [c for c in CASES if c[3].get("N", synth.SPECS[c[0]]["N"]) <= 64]


@pytest.mark.parametrize("case", FB_CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_forward_backward_labelled(case):
    w = _workload(case)
    seqs, pi, A, B = to_gpu(w, labelled=True)
    rng = np.random.default_rng(3)
    wts = rng.uniform(0.5, 2.0, size=w.S).astype(np.float32)
    import torch
    wt = torch.from_numpy(wts).cuda()
    rll, rpi, rA, rB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets, w.lengths,
                                                  w.labels, wts.astype(np.float64), nthreads=8)
    gs = hmm.hmm_tuning_candidates(hmm.HMM_OP_FORWARD_BACKWARD, _npad(w.N))
    rs = hmm.hmm_tuning_candidates(hmm.HMM_TUNE_FB_RANGES, _npad(w.N))
    # every lanes-per-pair choice, and every number of segment ranges per pair
    # (1: the single-kernel adjoint)
    for G, R in [(g, rs[0]) for g in gs] + [(gs[0], r) for r in rs[1:]]:
        hmm.hmm_set_tuning(hmm.HMM_OP_FORWARD_BACKWARD, _npad(w.N), G)
        hmm.hmm_set_tuning(hmm.HMM_TUNE_FB_RANGES, _npad(w.N), R)
        ll, cpi, cA, cB = hmm.hmm_forward_backward(pi, A, B, seqs, weight=wt)
        assert np.all(np.abs(ll.cpu().numpy() - rll) <= ll_tol(w.lengths)), f"G={G} R={R}"
        check_counts((cpi, cA, cB), (rpi, rA, rB), what=f"G={G} R={R}")
        # the logit gradient built from the counts
        g = hmm.hmm_softmax_grad(pi, A, B, cpi, cA, cB)
        rg = oracle.softmax_grad(oparams(w), rpi, rA, rB)
        check_grads(g, rg, (rpi, rA, rB), (w.pi, w.A, w.B), what=f"G={G} R={R}")


@pytest.mark.parametrize("case", FB_CASES[:3], ids=lambda c: f"{c[0]}-{c[1]}-{c[3]}")
def test_forward_backward_all_models_weighted(case):
    import torch
    w = _workload(case)
    seqs, pi, A, B = to_gpu(w)
    wts = np.random.default_rng(4).uniform(-1.0, 1.0, size=(w.S, w.K)).astype(np.float32)
    rll, rpi, rA, rB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets, w.lengths,
                                                  None, wts.astype(np.float64), nthreads=8)
    # signed weights cancel: each entry is held to the scale of its terms,
    # the counts under |weights|
    _, upi, uA, uB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets, w.lengths,
                                                None, np.abs(wts).astype(np.float64), nthreads=8)
    for R in hmm.hmm_tuning_candidates(hmm.HMM_TUNE_FB_RANGES, _npad(w.N)):
        hmm.hmm_set_tuning(hmm.HMM_TUNE_FB_RANGES, _npad(w.N), R)
        ll, cpi, cA, cB = hmm.hmm_forward_backward(pi, A, B, seqs,
                                                   weight=torch.from_numpy(wts).cuda())
        assert np.all(np.abs(ll.cpu().numpy() - rll) <= ll_tol(w.lengths)[:, None])
        check_counts((cpi, cA, cB), (rpi, rA, rB), scale=(upi, uA, uB), what=f"R={R}")


def test_deterministic_repeat():
    w = synth.make_workload("batched", n_seqs=300, lengths=("uniform", 1, 300))
    seqs, pi, A, B = to_gpu(w)
    a = hmm.hmm_forward(pi, A, B, seqs)[0].cpu().numpy()
    b = hmm.hmm_forward(pi, A, B, seqs)[0].cpu().numpy()
    np.testing.assert_array_equal(a, b)
    lab = seqs.labelled(seqs.lengths.new_tensor(w.labels))
    c1 = [t.cpu().numpy() for t in hmm.hmm_forward_backward(pi, A, B, lab)]
    c2 = [t.cpu().numpy() for t in hmm.hmm_forward_backward(pi, A, B, lab)]
    for x, y in zip(c1, c2):
        np.testing.assert_array_equal(x, y)
