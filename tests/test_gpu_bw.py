"""Baum-Welch re-estimation on the GPU (Sec. 2.7 "Baum-Welch"; Rabiner eq. 40)
against the FP64 oracle: the M-step kernel element by element, and the
graph-captured E-step/M-step loop iteration by iteration (parameters and the
total log-likelihood, which never decreases)."""
import dataclasses

import numpy as np
import pytest

import oracle
from helpers import oparams, rel_l2, to_gpu
from paper_1310_3322_gb300 import baum_welch, hmm, synth

pytestmark = pytest.mark.gpu


def test_mstep_matches_oracle_including_empty_rows():
    import torch
    rng = np.random.default_rng(11)
    K, N, M = 3, 9, 13
    pi, A, B = synth.random_model(rng, K, N, M)
    cpi = rng.gamma(0.5, size=(K, N)).astype(np.float32)
    cA = rng.gamma(0.5, size=(K, N, N)).astype(np.float32)
    cB = rng.gamma(0.5, size=(K, N, M)).astype(np.float32)
    cpi[1] = 0.0          # a model that saw no sequence keeps its pi
    cA[2, 4] = 0.0        # a state never left keeps its transition row
    cB[0, 7] = 0.0        # a state never visited keeps its emission row
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B, cpi, cA, cB)]
    out = hmm.hmm_mstep(*t)
    ref = oracle.mstep(oracle.params(pi, A, B), cpi, cA, cB)
    for g, r in zip(out, (ref.pi, ref.A, ref.B)):
        np.testing.assert_allclose(g.cpu().numpy(), r, rtol=2e-6, atol=1e-7)
    # in place
    hmm.hmm_mstep(t[0], t[1], t[2], t[3], t[4], t[5], out=(t[0], t[1], t[2]))
    for g, r in zip(t[:3], (ref.pi, ref.A, ref.B)):
        np.testing.assert_allclose(g.cpu().numpy(), r, rtol=2e-6, atol=1e-7)


def _oracle_bw(w, iters):
    P = oparams(w)
    hist = []
    for _ in range(iters):
        ll, cpi, cA, cB, _ = oracle.forward_backward(P, w.symbols, w.offsets, w.lengths,
                                                     w.labels, nthreads=8)
        hist.append(float(np.sum(ll)))
        P = oracle.mstep(P, cpi, cA, cB)
    return P, hist


# tol: per-observation log-likelihood bound of the path (FP32: 1e-4; BF16: 2u)
@pytest.mark.parametrize("precision,tol", [(hmm.HMM_FP32, 1e-4), (hmm.HMM_BF16_MMA, 2 ** -7)])
def test_baum_welch_loop_matches_oracle(precision, tol):
    name = "gradient" if precision == hmm.HMM_FP32 else "training"
    w = synth.make_workload(name, n_seqs=240, lengths=("uniform", 20, 160), K=3)
    # start from a perturbed model so that re-estimation has work to do
    rng = np.random.default_rng(12)
    start = [x * rng.uniform(0.5, 1.5, size=x.shape).astype(np.float32) for x in (w.pi, w.A, w.B)]
    start = [x / x.sum(axis=-1, keepdims=True) for x in start]
    w0 = dataclasses.replace(w, pi=start[0], A=start[1], B=start[2])
    seqs, pi, A, B = to_gpu(w0, labelled=True)
    iters = 7
    hist = baum_welch.baum_welch(pi, A, B, seqs, max_iters=iters, tol=0.0, chunk=3,
                                 precision=precision)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    assert len(hist) == iters
    P, rhist = _oracle_bw(w0, iters)
    sumT = float(w.lengths.sum())
    # the total log-likelihood rises (up to the path's rounding) ...
    assert all(b >= a - tol * sumT for a, b in zip(hist, hist[1:])), hist
    assert hist[-1] > hist[0]
    # ... and follows the FP64 iteration
    print(f"precision {precision}: max |d total| / sum T "
          f"{np.max(np.abs(np.array(hist) - rhist)) / sumT:.2e}")
    np.testing.assert_allclose(hist, rhist, rtol=0, atol=tol * sumT)
    for g, r in zip((pi, A, B), (P.pi, P.A, P.B)):
        assert rel_l2(g.cpu().numpy(), r) <= 5 * tol, rel_l2(g.cpu().numpy(), r)


def test_baum_welch_graph_replay_matches_eager():
    w = synth.make_workload("gradient", n_seqs=150, lengths=("uniform", 10, 120), K=2)
    results = []
    for graph in (True, False):
        seqs, pi, A, B = to_gpu(w, labelled=True)
        h = baum_welch.baum_welch(pi, A, B, seqs, max_iters=6, tol=0.0, chunk=2, graph=graph)
        results.append((h, [t.cpu().numpy() for t in (pi, A, B)]))
    assert results[0][0] == results[1][0]
    for a, b in zip(results[0][1], results[1][1]):
        np.testing.assert_array_equal(a, b)


def test_baum_welch_above_128_states_follows_the_oracle_and_replays():
    """The re-estimation loop on the 512-state recipe at 300 states (the
    adjoint above 128 states: wide forward and backward passes, the count
    contraction, the M-step), eager and graph-replayed: the total rises and
    follows the FP64 iteration within the BF16 bound, and the replayed loop
    equals the eager one bit for bit."""
    w = synth.make_workload("cuhmm", n_seqs=20, lengths=("uniform", 20, 70), N=300, M=32)
    rng = np.random.default_rng(13)
    start = [x * rng.uniform(0.5, 1.5, size=x.shape).astype(np.float32) for x in (w.pi, w.A, w.B)]
    start = [x / x.sum(axis=-1, keepdims=True) for x in start]
    w0 = dataclasses.replace(w, pi=start[0], A=start[1], B=start[2])
    iters, tol = 4, 2 ** -7
    results = []
    for graph in (True, False):
        seqs, pi, A, B = to_gpu(w0, labelled=True)
        h = baum_welch.baum_welch(pi, A, B, seqs, max_iters=iters, tol=0.0, chunk=2, graph=graph,
                                  precision=hmm.HMM_BF16_MMA)
        assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
        results.append((h, [t.cpu().numpy() for t in (pi, A, B)]))
    assert results[0][0] == results[1][0]
    for a, b in zip(results[0][1], results[1][1]):
        np.testing.assert_array_equal(a, b)
    hist = results[0][0]
    _, rhist = _oracle_bw(w0, iters)
    sumT = float(w.lengths.sum())
    assert hist[-1] > hist[0]
    np.testing.assert_allclose(hist, rhist, rtol=0, atol=tol * sumT)
