"""Viterbi above 64 states (64 < N <= 128: one warp per pair, the log
transition matrix in shared memory) against the FP64 oracle (Rabiner eqs.
32-35): scores within the FP32 bound, decoded models and paths bit-exact on
margin-filtered inputs, in all three model modes; the score of the path
kernel equals the score kernel's bit for bit; degenerate inputs."""
import numpy as np
import pytest

import oracle
from helpers import ll_tol, margin_filtered, oparams, to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

CASES = [
    # name, n_seqs, lengths, overrides: 65 (one state past the SIMT limit),
    # 100 (padding inside the last lane group), 128 (full)
    ("large", 70, ("uniform", 1, 160), {"K": 3, "N": 65, "M": 32}),
    ("large", 90, ("uniform", 1, 200), {"K": 2, "N": 100, "M": 50}),
    ("large", 61, ("uniform", 1, 250), {"K": 3, "N": 128, "M": 256}),
]


def _workload(case):
    name, S, lengths, over = case
    return synth.make_workload(name, n_seqs=S, lengths=lengths, **over)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[3]['N']}")
def test_wide_viterbi_all_models(case):
    w = margin_filtered(_workload(case))
    seqs, pi, A, B = to_gpu(w)
    sc, best, path = hmm.hmm_viterbi(pi, A, B, seqs)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    rs, rbest, rpath, _, _ = oracle.viterbi(oparams(w), w.symbols, w.offsets, w.lengths,
                                            nthreads=8)
    sc, best, path = sc.cpu().numpy(), best.cpu().numpy(), path.cpu().numpy()
    assert np.all(np.abs(sc - rs) <= ll_tol(w.lengths)[:, None])
    np.testing.assert_array_equal(best, rbest)
    np.testing.assert_array_equal(path, rpath)
    # the path kernel recomputes the decoded model's scores with the same
    # arithmetic: labelled by the decoded model, its scores are bitwise those
    # of the score kernel
    import torch
    lab = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, model_of_seq=best,
                                   device="cuda")
    lsc, lbest, lpath = hmm.hmm_viterbi(pi, A, B, lab)
    np.testing.assert_array_equal(lsc.cpu().numpy(), sc[np.arange(w.S), best])
    np.testing.assert_array_equal(lpath.cpu().numpy(), path)


def test_wide_viterbi_labelled_and_model_sets():
    import torch
    w = margin_filtered(_workload(CASES[1]), labelled=True)
    seqs, pi, A, B = to_gpu(w, labelled=True)
    rs, _, rpath, _, _ = oracle.viterbi(oparams(w), w.symbols, w.offsets, w.lengths, w.labels)
    sc, best, path = hmm.hmm_viterbi(pi, A, B, seqs)
    assert np.all(np.abs(sc.cpu().numpy() - rs) <= ll_tol(w.lengths))
    np.testing.assert_array_equal(best.cpu().numpy(), w.labels)
    np.testing.assert_array_equal(path.cpu().numpy(), rpath)
    sc2, _, _ = hmm.hmm_viterbi(pi, A, B, seqs, want_path=False)  # the score kernel
    np.testing.assert_array_equal(sc2.cpu().numpy(), sc.cpu().numpy())
    # model sets of one model each: sequence s against its own label
    sets = to_gpu(w)[0].model_sets(torch.from_numpy(w.labels.astype(np.int32)).cuda(), 1)
    ssc, sbest, spath = hmm.hmm_viterbi(pi, A, B, sets)
    np.testing.assert_array_equal(ssc.cpu().numpy()[:, 0], sc.cpu().numpy())
    assert np.all(sbest.cpu().numpy() == 0)
    np.testing.assert_array_equal(spath.cpu().numpy(), rpath)


def test_wide_viterbi_degenerate():
    import torch
    rng = np.random.default_rng(21)
    K, N, M = 2, 90, 12
    pi, A, B = synth.random_model(rng, K, N, M, alpha=0.7)
    B[1, :, 11] = 0.0  # model 1 never emits symbol 11
    B /= B.sum(axis=2, keepdims=True)
    lengths = np.array([0, 1, 2, 40, 33], np.int32)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    sym = rng.integers(0, 11, size=int(lengths.sum())).astype(np.int32)
    sym[offsets[3] + 17] = 11          # impossible under model 1
    bad = sym.copy()
    bad[offsets[4] + 5] = M + 1        # invalid symbol in sequence 4
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    P = oracle.params(pi, A, B)
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths, device="cuda")
    sc, best, path = (x.cpu().numpy() for x in hmm.hmm_viterbi(*t, seqs))
    rs, rbest, rpath, _, _ = oracle.viterbi(P, sym, offsets, lengths)
    assert np.isneginf(sc[3, 1]) and np.isneginf(rs[3, 1])
    assert np.all(sc[0] == 0.0)
    fin = np.isfinite(rs)
    assert np.array_equal(fin, np.isfinite(sc))
    assert np.all(np.abs(sc[fin] - rs[fin]) <= 1e-3)
    # labelled impossible pair: -inf score, path filled with 0
    lab = hmm.Sequences.from_numpy(sym, offsets, lengths, model_of_seq=np.ones(5, np.int32),
                                   device="cuda")
    lsc, _, lpath = (x.cpu().numpy() for x in hmm.hmm_viterbi(*t, lab))
    assert np.isneginf(lsc[3])
    assert np.all(lpath[offsets[3]:offsets[3] + lengths[3]] == 0)
    # invalid symbol: NaN scores, decoded model -1, path -1, status bit
    seqs_b = hmm.Sequences.from_numpy(bad, offsets, lengths, device="cuda")
    bsc, bbest, bpath = (x.cpu().numpy() for x in hmm.hmm_viterbi(*t, seqs_b))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) & hmm.HMM_STATUS_SYMBOL
    assert np.isnan(bsc[4]).all() and bbest[4] == -1
    assert np.all(bpath[offsets[4]:offsets[4] + lengths[4]] == -1)
