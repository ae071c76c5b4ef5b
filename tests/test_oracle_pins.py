"""Pins of the FP64 oracle to things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle -- a dropped
first emission, a transposed A, a wrong log-sum-exp shift, a missing weight,
an off-by-one in the backward variable, the wrong tie-break -- fails at least
one of them:

* exact enumeration over all N^T paths (oracle.bruteforce) for the
  likelihood, the best path and its score, the second-best path and the
  expected counts;
* sum over all M^T symbol strings of P(O) = 1;
* closed forms (N=1, identical emission rows, identity A with one-hot pi,
  uniform model, T=0 and T=1);
* exact rational fixtures (tests/golden/tiny_exact.json);
* count identities and the bound  score <= log P <= score + T log N;
* central finite differences of sum_s w_s log P w.r.t. the softmax logits;
* one Baum-Welch re-estimation never lowers the likelihood.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bruteforce
from paper_1310_3322_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_exact.json")


def _rand_model(seed, K, N, M, alpha=1.0):
    rng = np.random.default_rng(seed)
    pi = rng.dirichlet(np.full(N, alpha), size=K)
    A = rng.dirichlet(np.full(N, alpha), size=(K, N))
    B = rng.dirichlet(np.full(M, alpha), size=(K, N))
    return pi, A, B


def _pack(seqs):
    lengths = np.array([len(s) for s in seqs], np.int32)
    offsets = np.zeros(len(seqs), np.int64)
    if len(seqs):
        offsets[1:] = np.cumsum(lengths.astype(np.int64))[:-1]
    flat = np.array([x for s in seqs for x in s], np.int32)
    return flat, offsets, lengths


# --------------------------------------------------------------------------
# forward
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_forward_matches_enumeration(orc, seed):
    N, M = 3, 4
    pi, A, B = _rand_model(seed, 1, N, M)
    rng = np.random.default_rng(100 + seed)
    seqs = [list(rng.integers(0, M, size=T)) for T in range(0, 8)]
    sym, off, ln = _pack(seqs)
    ll, am, rc = orc.forward(orc.params(pi, A, B), sym, off, ln)
    assert rc == 0
    for s, o in enumerate(seqs):
        ref = bruteforce.likelihood(pi[0], A[0], B[0], o)
        assert ll[s, 0] == pytest.approx(math.log(ref), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("M,T", [(3, 5), (2, 8), (8, 3)])
def test_forward_sums_to_one_over_all_strings(orc, M, T):
    N = 3
    pi, A, B = _rand_model(7 * M + T, 2, N, M, alpha=0.7)
    seqs = [list(o) for o in itertools.product(range(M), repeat=T)]
    sym, off, ln = _pack(seqs)
    ll, _, rc = orc.forward(orc.params(pi, A, B), sym, off, ln)
    assert rc == 0
    tot = np.exp(ll).sum(axis=0)
    np.testing.assert_allclose(tot, 1.0, rtol=1e-12)


def test_forward_closed_forms(orc):
    rng = np.random.default_rng(5)
    M, T = 6, 40
    o = rng.integers(0, M, size=T)
    sym, off, ln = _pack([list(o)])
    # N = 1: log P = sum_t log b(o_t)
    b = rng.dirichlet(np.ones(M))
    ll, _, _ = orc.forward(orc.params([1.0], [[1.0]], [b]), sym, off, ln)
    assert ll[0, 0] == pytest.approx(np.log(b[o]).sum(), rel=1e-13)
    # identical emission rows: the hidden chain is irrelevant
    N = 4
    pi, A, _ = _rand_model(9, 1, N, M)
    Bsame = np.tile(b, (1, N, 1))
    ll, _, _ = orc.forward(orc.params(pi, A, Bsame), sym, off, ln)
    assert ll[0, 0] == pytest.approx(np.log(b[o]).sum(), rel=1e-13)
    # identity A, one-hot pi at state 2: the chain stays in state 2
    Bd = rng.dirichlet(np.ones(M), size=(1, N))
    pi1 = np.zeros((1, N)); pi1[0, 2] = 1.0
    ll, _, _ = orc.forward(orc.params(pi1, np.eye(N)[None], Bd), sym, off, ln)
    assert ll[0, 0] == pytest.approx(np.log(Bd[0, 2, o]).sum(), rel=1e-13)
    # uniform model: log P = -T log M
    ll, _, _ = orc.forward(orc.params(np.full((1, N), 1 / N), np.full((1, N, N), 1 / N),
                                      np.full((1, N, M), 1 / M)), sym, off, ln)
    assert ll[0, 0] == pytest.approx(-T * math.log(M), rel=1e-13)


def test_forward_short_sequences(orc):
    pi, A, B = _rand_model(3, 1, 3, 5)
    sym, off, ln = _pack([[], [4]])
    ll, _, rc = orc.forward(orc.params(pi, A, B), sym, off, ln)
    assert rc == 0
    assert ll[0, 0] == 0.0
    assert ll[1, 0] == pytest.approx(math.log((pi[0] * B[0, :, 4]).sum()), rel=1e-14)


def test_forward_impossible_and_bad_symbol(orc):
    pi = np.array([[1.0, 0.0]])
    A = np.array([[[1.0, 0.0], [0.0, 1.0]]])
    B = np.array([[[1.0, 0.0], [0.0, 1.0]]])
    sym, off, ln = _pack([[0, 0, 1], [0, 0], [0, 2]])
    ll, _, rc = orc.forward(orc.params(pi, A, B), sym, off, ln)
    assert ll[0, 0] == -np.inf and ll[1, 0] == 0.0
    assert np.isnan(ll[2, 0]) and rc == orc.ORC_ERR_SYMBOL


def test_forward_argmax_lowest_index_on_ties(orc):
    pi, A, B = _rand_model(11, 1, 3, 4)
    P = orc.params(np.concatenate([pi, pi]), np.concatenate([A, A]), np.concatenate([B, B]))
    sym, off, ln = _pack([[0, 1, 2, 3]])
    ll, am, _ = orc.forward(P, sym, off, ln)
    assert ll[0, 0] == ll[0, 1] and am[0] == 0


def test_forward_threads_agree(orc):
    w = synth.make_workload("batched", n_seqs=64, lengths=("uniform", 5, 40))
    P = orc.params(w.pi, w.A, w.B)
    a, am1, _ = orc.forward(P, w.symbols, w.offsets, w.lengths, nthreads=1)
    b, am4, _ = orc.forward(P, w.symbols, w.offsets, w.lengths, nthreads=4)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(am1, am4)


# --------------------------------------------------------------------------
# Viterbi
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_viterbi_matches_enumeration(orc, seed):
    N, M = 3, 4
    pi, A, B = _rand_model(50 + seed, 1, N, M)
    rng = np.random.default_rng(200 + seed)
    seqs = [list(rng.integers(0, M, size=T)) for T in range(1, 8)]
    sym, off, ln = _pack(seqs)
    score, best, path, margin, rc = orc.viterbi(orc.params(pi, A, B), sym, off, ln)
    assert rc == 0
    for s, o in enumerate(seqs):
        pb, q, p2 = bruteforce.best_path(pi[0], A[0], B[0], o)
        assert score[s, 0] == pytest.approx(math.log(pb), rel=1e-12)
        assert list(path[off[s]: off[s] + ln[s]]) == list(q)
        if p2 > 0:
            assert margin[s] == pytest.approx(math.log(pb) - math.log(p2), rel=1e-9, abs=1e-12)


def test_viterbi_bounds_and_path_score(orc):
    w = synth.make_workload("batched", n_seqs=48, lengths=("uniform", 1, 60))
    P = orc.params(w.pi, w.A, w.B)
    ll, _, _ = orc.forward(P, w.symbols, w.offsets, w.lengths)
    sc, best, path, _, _ = orc.viterbi(P, w.symbols, w.offsets, w.lengths)
    N = w.N
    T = w.lengths.astype(np.float64)[:, None]
    assert np.all(sc <= ll + 1e-9)
    assert np.all(ll <= sc + T * math.log(N) + 1e-9)
    lpi, lA, lB = np.log(P.pi), np.log(P.A), np.log(P.B)
    for s in range(w.S):
        k, o = best[s], w.symbols[w.offsets[s]: w.offsets[s] + w.lengths[s]]
        q = path[w.offsets[s]: w.offsets[s] + w.lengths[s]]
        j = lpi[k, q[0]] + lB[k, q[0], o[0]]
        for t in range(1, len(o)):
            j += lA[k, q[t - 1], q[t]] + lB[k, q[t], o[t]]
        assert j == pytest.approx(sc[s, k], rel=1e-12)
        assert k == int(np.argmax(sc[s]))


def test_viterbi_exact_ties_take_smallest_index(orc):
    # uniform model: every path ties; the smallest-index backtrack is all zeros
    N, M = 3, 3
    P = orc.params(np.full((1, N), 1 / N), np.full((1, N, N), 1 / N), np.full((1, N, M), 1 / M))
    sym, off, ln = _pack([[0, 1, 2, 1]])
    sc, _, path, margin, _ = orc.viterbi(P, sym, off, ln)
    assert list(path) == [0, 0, 0, 0] and margin[0] == 0.0
    # identity A, equal pi, identical emissions: constant paths tie exactly
    Fr = Fraction
    pi = [Fr(1, 2), Fr(1, 2)]
    A = [[Fr(1), Fr(0)], [Fr(0), Fr(1)]]
    B = [[Fr(1, 4), Fr(3, 4)], [Fr(1, 4), Fr(3, 4)]]
    o = [1, 0, 1]
    pb, q, _ = bruteforce.best_path(pi, A, B, o)
    sym, off, ln = _pack([o])
    sc, _, path, _, _ = orc.viterbi(orc.params([[0.5, 0.5]], [[[1, 0], [0, 1]]],
                                               [[[0.25, 0.75], [0.25, 0.75]]]), sym, off, ln)
    assert list(path) == list(q) == [0, 0, 0]
    assert sc[0, 0] == pytest.approx(math.log(pb), rel=1e-14)


def test_viterbi_empty_sequence(orc):
    pi, A, B = _rand_model(1, 2, 3, 3)
    sym, off, ln = _pack([[], [1, 2]])
    sc, best, path, _, _ = orc.viterbi(orc.params(pi, A, B), sym, off, ln)
    assert sc[0, 0] == 0.0 and sc[0, 1] == 0.0 and best[0] == 0


# --------------------------------------------------------------------------
# exact rational fixtures
# --------------------------------------------------------------------------

def _frac(s):
    n, d = s.split("/")
    return Fraction(int(n), int(d))


def test_golden_exact_fixtures(orc):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        pi = np.array([float(_frac(x)) for x in c["pi"]])
        A = np.array([[float(_frac(x)) for x in r] for r in c["A"]])
        B = np.array([[float(_frac(x)) for x in r] for r in c["B"]])
        sym, off, ln = _pack([c["obs"]])
        P = orc.params(pi, A, B)
        ll, _, _ = orc.forward(P, sym, off, ln)
        assert ll[0, 0] == pytest.approx(math.log(_frac(c["P"])), rel=1e-13)
        sc, _, path, margin, _ = orc.viterbi(P, sym, off, ln)
        assert sc[0, 0] == pytest.approx(math.log(_frac(c["P_best"])), rel=1e-13)
        assert list(path) == c["path"]
        assert margin[0] == pytest.approx(
            math.log(_frac(c["P_best"]) / _frac(c["P_second"])), rel=1e-10)


# --------------------------------------------------------------------------
# expected counts, gradient, re-estimation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_counts_match_enumeration(orc, seed):
    N, M = 3, 3
    pi, A, B = _rand_model(300 + seed, 1, N, M)
    rng = np.random.default_rng(400 + seed)
    seqs = [list(rng.integers(0, M, size=T)) for T in (1, 2, 4, 6)]
    wts = rng.uniform(0.2, 2.0, size=len(seqs))
    sym, off, ln = _pack(seqs)
    mos = np.zeros(len(seqs), np.int32)
    ll, cpi, cA, cB, rc = orc.forward_backward(orc.params(pi, A, B), sym, off, ln, mos, wts)
    assert rc == 0
    epi = np.zeros(N); eA = np.zeros((N, N)); eB = np.zeros((N, M))
    for w, o in zip(wts, seqs):
        a, b, c, lz = bruteforce.expected_counts(pi[0], A[0], B[0], o)
        epi += w * np.array(a); eA += w * np.array(b); eB += w * np.array(c)
    np.testing.assert_allclose(cpi[0], epi, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(cA[0], eA, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(cB[0], eB, rtol=1e-10, atol=1e-13)


def test_count_identities(orc):
    w = synth.make_workload("gradient", n_seqs=40, lengths=("uniform", 1, 50))
    P = orc.params(w.pi, w.A, w.B)
    wts = np.random.default_rng(0).uniform(0.5, 1.5, size=w.S)
    ll, cpi, cA, cB, _ = orc.forward_backward(P, w.symbols, w.offsets, w.lengths, w.labels, wts)
    for k in range(w.K):
        sel = w.labels == k
        assert cpi[k].sum() == pytest.approx(wts[sel].sum(), rel=1e-11)
        assert cA[k].sum() == pytest.approx((wts[sel] * (w.lengths[sel] - 1)).sum(), rel=1e-11)
        assert cB[k].sum() == pytest.approx((wts[sel] * w.lengths[sel]).sum(), rel=1e-11)
        # sum_j xi_t(i,j) = gamma_t(i): row totals of C_A equal the emission
        # totals minus the final-step posteriors, which are non-negative
        assert np.all(cB[k].sum(1) - cA[k].sum(1) >= -1e-9)
    ll2, _, _ = orc.forward(P, w.symbols, w.offsets, w.lengths, w.labels)
    np.testing.assert_allclose(ll, ll2, rtol=1e-13)


def test_softmax_grad_matches_finite_differences(orc):
    """Central differences (h = 1e-6, FP64) of sum_s w_s log P(O_s | softmax(theta))."""
    K, N, M = 2, 3, 4
    rng = np.random.default_rng(21)
    lpi, lA, lB = (rng.standard_normal((K, N)), rng.standard_normal((K, N, N)),
                   rng.standard_normal((K, N, M)))
    seqs = [list(rng.integers(0, M, size=T)) for T in (3, 7, 1, 12, 5, 9)]
    sym, off, ln = _pack(seqs)
    mos = np.array([0, 1, 0, 1, 1, 0], np.int32)
    wts = rng.uniform(0.5, 2.0, size=len(seqs))

    def loss(a, b, c):
        P = orc.params(orc.softmax_rows(a), orc.softmax_rows(b), orc.softmax_rows(c))
        ll, _, _ = orc.forward(P, sym, off, ln, mos)
        return float((wts * ll).sum())

    P = orc.params(orc.softmax_rows(lpi), orc.softmax_rows(lA), orc.softmax_rows(lB))
    _, cpi, cA, cB, _ = orc.forward_backward(P, sym, off, ln, mos, wts)
    gpi, gA, gB = orc.softmax_grad(P, cpi, cA, cB)
    h = 1e-6
    for arr, g in ((lpi, gpi), (lA, gA), (lB, gB)):
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h; fp = loss(lpi, lA, lB)
            arr[idx] = old - h; fm = loss(lpi, lA, lB)
            arr[idx] = old
            fd = (fp - fm) / (2 * h)
            assert g[idx] == pytest.approx(fd, abs=1e-7 * (1 + abs(fd)))
    # softmax invariance: each row's gradient sums to zero
    for g in (gpi, gA, gB):
        np.testing.assert_allclose(g.sum(-1), 0.0, atol=1e-12)


def test_baum_welch_step_never_lowers_likelihood(orc):
    w = synth.make_workload("plain", n_seqs=16, lengths=("uniform", 5, 30))
    P = orc.params(w.pi, w.A, w.B)
    prev = None
    for it in range(5):
        ll, cpi, cA, cB, _ = orc.forward_backward(P, w.symbols, w.offsets, w.lengths, w.labels)
        tot = ll.sum()
        if prev is not None:
            assert tot >= prev - 1e-9
        prev = tot
        P = orc.mstep(P, cpi, cA, cB)
        for arr in (P.pi, P.A, P.B):
            np.testing.assert_allclose(arr.sum(-1), 1.0, rtol=1e-12)


def test_mstep_closed_form_when_the_state_path_is_observable(orc):
    """State i emits only symbols 2i and 2i+1, so each observation fixes its
    state and the posteriors are one-hot: re-estimation (Rabiner eq. 40) is
    then plain frequency counting along the observed state path, and a state
    that is never left (or never entered) keeps its old row."""
    N, M = 4, 8
    pi, A, B = _rand_model(31, 1, N, M)
    B = np.zeros((1, N, M))
    for i in range(N):
        B[0, i, 2 * i], B[0, i, 2 * i + 1] = 0.3, 0.7
    # state 3 is never visited; state 2 only ends sequences
    seqs = [[0, 3, 1, 2, 5], [2, 2, 3, 0, 1], [1, 4], [3, 0, 5]]
    sym, off, ln = _pack(seqs)
    P = orc.params(pi, A, B)
    _, cpi, cA, cB, _ = orc.forward_backward(P, sym, off, ln, np.zeros(len(seqs), np.int32))
    Q = orc.mstep(P, cpi, cA, cB)
    npi = np.zeros(N); nA = np.zeros((N, N)); nB = np.zeros((N, M))
    for o in seqs:
        s = [x // 2 for x in o]
        npi[s[0]] += 1
        for a, b in zip(s, s[1:]):
            nA[a, b] += 1
        for x, st in zip(o, s):
            nB[st, x] += 1
    np.testing.assert_allclose(Q.pi[0], npi / npi.sum(), atol=1e-12)
    for i in range(N):
        ra = nA[i] / nA[i].sum() if nA[i].sum() else A[0, i]
        rb = nB[i] / nB[i].sum() if nB[i].sum() else B[0, i]
        np.testing.assert_allclose(Q.A[0, i], ra, atol=1e-12)
        np.testing.assert_allclose(Q.B[0, i], rb, atol=1e-12)
    assert nA[2].sum() == 0 and nB[3].sum() == 0   # the keep-old-row cases are exercised


def test_mstep_single_state_gives_symbol_frequencies(orc):
    """N = 1: the only free parameter is B, whose maximum-likelihood value is
    the empirical symbol frequency, reached in one step from any start."""
    pi, A, B = _rand_model(32, 1, 1, 5)
    seqs = [[0, 4, 4, 1], [4, 2], [1, 1, 4, 0, 3]]
    sym, off, ln = _pack(seqs)
    P = orc.params(pi, A, B)
    _, cpi, cA, cB, _ = orc.forward_backward(P, sym, off, ln, np.zeros(3, np.int32))
    Q = orc.mstep(P, cpi, cA, cB)
    freq = np.bincount(sym, minlength=5) / sym.size
    np.testing.assert_allclose(Q.B[0, 0], freq, atol=1e-12)
    assert Q.pi[0, 0] == 1.0 and Q.A[0, 0, 0] == 1.0


# --------------------------------------------------------------------------
# sensitivity: the pins catch planted mistakes (made on the oracle's inputs)
# --------------------------------------------------------------------------

def test_pins_detect_transposed_transition_matrix(orc):
    pi, A, B = _rand_model(77, 1, 3, 4)
    o = [0, 3, 1, 2, 2]
    sym, off, ln = _pack([o])
    ll, _, _ = orc.forward(orc.params(pi, A.transpose(0, 2, 1), B), sym, off, ln)
    assert abs(ll[0, 0] - math.log(bruteforce.likelihood(pi[0], A[0], B[0], o))) > 1e-6


def test_pins_detect_dropped_first_emission(orc):
    pi, A, B = _rand_model(78, 1, 3, 4)
    o = [2, 3, 1]
    # dropping b(o_1) equals scoring with a uniform-1 first emission
    ref = math.log(bruteforce.likelihood(pi[0], A[0], B[0], o))
    alt = math.log(sum(pi[0][q0] * A[0][q0][q1] * B[0][q1][o[1]] * A[0][q1][q2] * B[0][q2][o[2]]
                       for q0 in range(3) for q1 in range(3) for q2 in range(3)))
    sym, off, ln = _pack([o])
    ll, _, _ = orc.forward(orc.params(pi, A, B), sym, off, ln)
    assert ll[0, 0] == pytest.approx(ref, rel=1e-12) and abs(ll[0, 0] - alt) > 1e-3
