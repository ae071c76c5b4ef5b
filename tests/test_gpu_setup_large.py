"""Batches above 4096 sequences take the setup plan over many blocks
(validation and length-bucket counts per block of 4096 sequences, one block
of per-block offsets, then placement and prefix sums per block). Checked
through every output that depends on it: the length-sorted schedule (forward,
Viterbi, adjoint and scan results against the oracle), the backpointer
offsets (Viterbi paths bit-exact), the scan's chunk offsets, the argmax
counters, and the rejection of bad sequences (status bit, NaN, no counts)."""
import numpy as np
import pytest

import oracle
from helpers import ll_tol, margin_filtered, oparams, rel_l2, to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu


def _workload(n=9001, lengths=("uniform", 0, 40)):
    return synth.make_workload("batched", n_seqs=n, lengths=lengths, K=3, N=8, M=16)


def test_many_blocks_forward_viterbi_scan():
    w = margin_filtered(_workload())
    seqs, pi, A, B = to_gpu(w)
    P = oparams(w)
    ll, am = hmm.hmm_forward(pi, A, B, seqs)
    sc, best, path = hmm.hmm_viterbi(pi, A, B, seqs)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    rll, ram, _ = oracle.forward(P, w.symbols, w.offsets, w.lengths, nthreads=16)
    rs, rbest, rpath, _, _ = oracle.viterbi(P, w.symbols, w.offsets, w.lengths, nthreads=16)
    tol = ll_tol(w.lengths)[:, None]
    assert np.all(np.abs(ll.cpu().numpy() - rll) <= tol)
    srt = np.sort(rll, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * tol[:, 0]
    np.testing.assert_array_equal(am.cpu().numpy()[clear], ram[clear])
    assert np.all(np.abs(sc.cpu().numpy() - rs) <= tol)
    np.testing.assert_array_equal(best.cpu().numpy(), rbest)
    np.testing.assert_array_equal(path.cpu().numpy(), rpath)
    # chunk offsets of the parallel-in-time forward (chunks of 8 steps)
    sl, _ = hmm.hmm_forward_scan(pi, A, B, seqs, chunk=8)
    assert np.all(np.abs(sl.cpu().numpy() - rll) <= tol)


def test_many_blocks_adjoint_and_rejections():
    import torch
    w = _workload(n=8300, lengths=("uniform", 1, 40))
    lengths = w.lengths.copy()
    offsets = w.offsets.copy()
    labels = w.labels.copy()
    bad = np.array([5, 4096, 4097, 8299])
    lengths[5] = -3                       # negative length
    offsets[4096] = w.total_obs + 10      # offset past the symbols
    labels[4097] = w.K + 1                # model index out of range
    lengths[8299] = 10_000                # above max_len
    ok = np.setdiff1d(np.arange(w.S), bad)
    seqs = hmm.Sequences.from_numpy(w.symbols, offsets, lengths, model_of_seq=labels,
                                    device="cuda", max_len=int(w.lengths.max()))
    pi, A, B = (torch.from_numpy(x).cuda() for x in (w.pi, w.A, w.B))
    ll, cpi, cA, cB = hmm.hmm_forward_backward(pi, A, B, seqs)
    st = hmm.hmm_get_device_status(hmm.default_workspace())
    assert st & hmm.HMM_STATUS_SEQ
    ll = ll.cpu().numpy()
    assert np.isnan(ll[bad]).all()
    rll, rpi, rA, rB, _ = oracle.forward_backward(oparams(w), w.symbols, w.offsets[ok],
                                                  w.lengths[ok], w.labels[ok], nthreads=16)
    assert np.all(np.abs(ll[ok] - rll) <= ll_tol(w.lengths[ok]))
    for g, r in zip((cpi, cA, cB), (rpi, rA, rB)):
        assert rel_l2(g.cpu().numpy(), r) <= 1e-4
