"""The large-state configuration at full size, in the launch shape the bench
times: K = 4 models, N = 128 states, M = 256 symbols, Dirichlet(0.3) rows,
16384 sequences with T ~ U{100..2000} (sum T = 17.35 M).

* the BF16 and TF32 tensor-core forward of every sequence against every
  model, and the BF16 adjoint of every sequence against its labelled model,
  each on the whole batch; 64 sampled sequences (the 16 longest among them)
  against the FP64 oracle: the hard bound 3 u T (BF16) or 2 u T (TF32), the per-sequence cap
  (u / 4) T + 2 u, and the argmax wherever the top two models are apart by
  more than twice that cap; the adjoint's count identities on every model;
* the BF16 adjoint on a 160-sequence subset that holds the 24 longest
  sequences (tiles of T ~ 2000: 125 checkpoint segments of 16 steps each),
  element by element against the oracle's expected counts on the model the
  kernel holds (A and B rounded to BF16);
* the TF32 adjoint on the whole batch (sampled log-likelihoods, count
  identities, counts against the BF16 adjoint's) and on such a subset,
  element by element against the oracle on A rounded to TF32.
Tolerances and their derivation: tests/test_gpu_mma.py, tests/test_gpu_mma_fb.py.
"""
import os

import numpy as np
import pytest

import oracle
from helpers import check_counts, ll_tol, oparams, to_gpu
from paper_1310_3322_gb300 import hmm, synth
from test_gpu_mma import N_ROUNDED, PRECISIONS, U_BF16, held_model, seq_cap

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def large():
    import torch
    w = synth.make_workload("large")
    seqs, pi, A, B = to_gpu(w)
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    return w, seqs, lab, pi, A, B


def _sample(w, n, longest, seed):
    order = np.argsort(-w.lengths, kind="stable")
    rest = np.random.default_rng(seed).choice(order[longest:], size=n - longest, replace=False)
    return np.sort(np.concatenate([order[:longest], rest]))


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_full_large_forward_all_models_sampled(large, prec):
    w, seqs, _, pi, A, B = large
    precision, u, _ = PRECISIONS[prec]
    ll, am = hmm.hmm_forward(pi, A, B, seqs, precision=precision)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    ll, am = ll.cpu().numpy(), am.cpu().numpy()
    assert np.all(np.isfinite(ll))
    idx = _sample(w, 64, 16, 11)
    assert w.lengths[idx].max() == w.lengths.max()
    ref, ref_am, _ = oracle.forward(oparams(w), w.symbols, w.offsets[idx], w.lengths[idx],
                                    nthreads=NTHREADS)
    T = w.lengths[idx].astype(np.float64)[:, None]
    err = np.abs(ll[idx] - ref)
    assert np.all(err <= N_ROUNDED[prec] * u * T + ll_tol(w.lengths[idx])[:, None])
    cap = seq_cap(u, w.lengths[idx])[:, None]
    print(f"{prec}: max|d|/T {np.max(err / T):.2e} mean {np.mean(err / T):.2e} "
          f"max |d|/cap {np.max(err / cap):.3f}")
    assert np.all(err <= cap)
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * cap[:, 0]
    assert clear.sum() >= len(idx) // 2
    np.testing.assert_array_equal(am[idx][clear], ref_am[clear])


def test_full_large_adjoint_labelled(large):
    w, _, lab, pi, A, B = large
    ll, cpi, cA, cB = (t.cpu().numpy() for t in
                       hmm.hmm_forward_backward(pi, A, B, lab, precision=hmm.HMM_BF16_MMA))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    assert np.all(np.isfinite(ll))
    idx = _sample(w, 64, 16, 12)
    rll, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets[idx], w.lengths[idx],
                               w.labels[idx], nthreads=NTHREADS)
    T = w.lengths[idx].astype(np.float64)
    err = np.abs(ll[idx] - rll)
    assert np.all(err <= 3 * U_BF16 * T + ll_tol(w.lengths[idx]))
    assert np.all(err <= seq_cap(U_BF16, w.lengths[idx])), np.max(err / T)
    # count identities of every model: sum C_pi = #sequences, sum C_A = sum (T - 1),
    # sum C_B = sum T, every count non-negative
    for k in range(w.K):
        Tk = w.lengths[w.labels == k].astype(np.float64)
        assert abs(cpi[k].sum() - Tk.size) <= U_BF16 * Tk.size
        assert abs(cA[k].sum() - (Tk - 1).sum()) <= U_BF16 * Tk.sum()
        assert abs(cB[k].sum() - Tk.sum()) <= U_BF16 * Tk.sum()
        assert np.all(cA[k] >= 0) and np.all(cB[k] >= 0) and np.all(cpi[k] >= 0)
        # and per state: the emission counts of a state add up to its visits,
        # sum_m C_B[j][m] = sum_t gamma_t(j) = sum_i C_A[j][i] + (visits at the last step)
        assert np.all(cB[k].sum(axis=1) + 1e-3 * Tk.sum() / w.N >= cA[k].sum(axis=1))


def test_large_adjoint_longest_subset_elementwise(large):
    import torch
    w = large[0]
    idx = _sample(w, 160, 24, 13)
    assert w.lengths[idx].max() == 2000
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets[idx], w.lengths[idx],
                                    model_of_seq=w.labels[idx])
    pi, A, B = (torch.from_numpy(x).cuda() for x in (w.pi, w.A, w.B))
    wts = np.random.default_rng(14).uniform(0.5, 2.0, size=idx.size).astype(np.float32)
    ll, cpi, cA, cB = (t.cpu().numpy() for t in hmm.hmm_forward_backward(
        pi, A, B, seqs, weight=torch.from_numpy(wts).cuda(), precision=hmm.HMM_BF16_MMA))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    # against the model the kernel holds (A and B rounded to BF16)
    rll, rpi, rA, rB, _ = oracle.forward_backward(held_model(w, "bf16"), w.symbols,
                                                  w.offsets[idx], w.lengths[idx], w.labels[idx],
                                                  wts.astype(np.float64), nthreads=NTHREADS)
    assert np.all(np.abs(ll - rll) <= seq_cap(U_BF16, w.lengths[idx]))
    worst = check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=U_BF16, what="longest subset")
    print(f"longest subset: worst |d|/(1+|ref|) pi {worst[0]:.2e} A {worst[1]:.2e} B {worst[2]:.2e}")


def test_full_large_adjoint_tf32_labelled(large):
    """The TF32 adjoint (every step's rows kept: 4 x 17.35 M rows of 128
    floats) on the whole batch: 64 sampled log-likelihoods against the oracle
    on the model the kernel holds (A rounded to TF32), the count identities of
    every model, and the counts against the BF16 adjoint's (both within their
    bounds of the exact counts: 2^-8 relative L2 apart at most)."""
    from test_gpu_mma import U_TF32
    w, _, lab, pi, A, B = large
    ll, cpi, cA, cB = (t.cpu().numpy() for t in
                       hmm.hmm_forward_backward(pi, A, B, lab, precision=hmm.HMM_TF32_MMA))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    assert np.all(np.isfinite(ll))
    idx = _sample(w, 64, 16, 15)
    rll, _, _ = oracle.forward(held_model(w, "tf32"), w.symbols, w.offsets[idx],
                               w.lengths[idx], w.labels[idx], nthreads=NTHREADS)
    T = w.lengths[idx].astype(np.float64)
    err = np.abs(ll[idx] - rll)
    assert np.all(err <= seq_cap(U_TF32, w.lengths[idx])), np.max(err / T)
    assert np.mean(err / T) <= U_TF32 / 8, np.mean(err / T)
    tol = 2.0 ** -8
    for k in range(w.K):
        Tk = w.lengths[w.labels == k].astype(np.float64)
        assert abs(cpi[k].sum() - Tk.size) <= tol * Tk.size
        assert abs(cA[k].sum() - (Tk - 1).sum()) <= tol * Tk.sum()
        assert abs(cB[k].sum() - Tk.sum()) <= tol * Tk.sum()
        assert np.all(cA[k] >= 0) and np.all(cB[k] >= 0) and np.all(cpi[k] >= 0)
    _, bpi, bA, bB = (t.cpu().numpy() for t in
                      hmm.hmm_forward_backward(pi, A, B, lab, precision=hmm.HMM_BF16_MMA))
    for g, r in zip((cpi, cA, cB), (bpi, bA, bB)):
        assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r)


def test_large_adjoint_tf32_longest_subset_elementwise(large):
    """The TF32 adjoint on a 160-sequence weighted subset that holds the 24
    longest sequences (T ~ 2000), element by element against the oracle's
    expected counts on the model the kernel holds."""
    import torch
    w = large[0]
    idx = _sample(w, 160, 24, 16)
    assert w.lengths[idx].max() == 2000
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets[idx], w.lengths[idx],
                                    model_of_seq=w.labels[idx])
    pi, A, B = (torch.from_numpy(x).cuda() for x in (w.pi, w.A, w.B))
    wts = np.random.default_rng(17).uniform(0.5, 2.0, size=idx.size).astype(np.float32)
    ll, cpi, cA, cB = (t.cpu().numpy() for t in hmm.hmm_forward_backward(
        pi, A, B, seqs, weight=torch.from_numpy(wts).cuda(), precision=hmm.HMM_TF32_MMA))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    rll, rpi, rA, rB, _ = oracle.forward_backward(held_model(w, "tf32"), w.symbols,
                                                  w.offsets[idx], w.lengths[idx], w.labels[idx],
                                                  wts.astype(np.float64), nthreads=NTHREADS)
    from test_gpu_mma import U_TF32
    assert np.all(np.abs(ll - rll) <= seq_cap(U_TF32, w.lengths[idx]))
    worst = check_counts((cpi, cA, cB), (rpi, rA, rB), rtol=2.0 ** -8, what="TF32 longest subset")
    print(f"TF32 longest subset: worst |d|/(1+|ref|) pi {worst[0]:.2e} A {worst[1]:.2e} "
          f"B {worst[2]:.2e}")
