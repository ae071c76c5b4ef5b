"""Edge cases, device status reporting, graph capture and the full-size
configurations (checked on sampled outputs and on size-independent
properties). All through the C-ABI."""
import math

import numpy as np
import pytest

import oracle
from helpers import COUNT_RTOL, ll_tol, oparams, rel_l2, to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu


def _pack(seqs):
    lengths = np.array([len(s) for s in seqs], np.int32)
    offsets = np.zeros(len(seqs), np.int64)
    if len(seqs):
        offsets[1:] = np.cumsum(lengths.astype(np.int64))[:-1]
    flat = np.array([x for s in seqs for x in s], np.int32)
    return flat, offsets, lengths


def _run_all(pi, A, B, sym, off, ln, mos=None, max_len=None):
    import torch
    seqs = hmm.Sequences.from_numpy(sym, off, ln, model_of_seq=mos, max_len=max_len)
    t = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda() for x in (pi, A, B)]
    ll, am = hmm.hmm_forward(*t, seqs)
    st_f = hmm.hmm_get_device_status(hmm.default_workspace())
    sc, best, path = hmm.hmm_viterbi(*t, seqs)
    st_v = hmm.hmm_get_device_status(hmm.default_workspace())
    return ll.cpu().numpy(), sc.cpu().numpy(), path.cpu().numpy(), st_f, st_v, seqs, t


def test_short_and_degenerate_shapes():
    rng = np.random.default_rng(0)
    for (K, N, M) in ((1, 1, 1), (1, 1, 5), (3, 2, 1), (2, 5, 7), (1, 64, 3)):
        pi, A, B = synth.random_model(rng, K, N, M)
        seqs = [list(rng.integers(0, M, size=T)) for T in (0, 1, 2, 3, 0, 1, 40, 5)]
        sym, off, ln = _pack(seqs)
        ll, sc, path, sf, sv, _, _ = _run_all(pi, A, B, sym, off, ln)
        assert sf == 0 and sv == 0
        P = oracle.params(pi, A, B)
        rll, _, _ = oracle.forward(P, sym, off, ln)
        rs, _, _, _, _ = oracle.viterbi(P, sym, off, ln, want_path=False)
        tol = ll_tol(ln)[:, None]
        assert np.all(np.abs(ll - rll) <= tol), (K, N, M)
        assert np.all(np.abs(sc - rs) <= tol), (K, N, M)
        assert np.all(ll[ln == 0] == 0) and np.all(sc[ln == 0] == 0)
        assert path.shape[0] == sym.shape[0]
        assert np.all((path >= 0) & (path < N))


def test_impossible_sequence_gives_minus_inf():
    pi = np.array([[1.0, 0.0]])
    A = np.array([[[1.0, 0.0], [0.0, 1.0]]])
    B = np.array([[[1.0, 0.0], [0.0, 1.0]]])
    sym, off, ln = _pack([[0, 0, 1], [0, 0], [1]])
    ll, sc, path, sf, sv, seqs, t = _run_all(pi, A, B, sym, off, ln)
    assert ll[0, 0] == -np.inf and ll[1, 0] == 0.0 and ll[2, 0] == -np.inf
    assert sc[0, 0] == -np.inf and sc[2, 0] == -np.inf
    np.testing.assert_array_equal(path, [0, 0, 0, 0, 0, 0])
    assert sf == 0 and sv == 0
    import torch
    lab = seqs.labelled(torch.zeros(3, dtype=torch.int32, device="cuda"))
    fll, cpi, cA, cB = hmm.hmm_forward_backward(*t, lab)
    fll = fll.cpu().numpy()
    assert fll[0] == -np.inf and fll[1] == 0.0
    # only the possible sequence contributes: gamma = 1 on state 0
    np.testing.assert_allclose(cpi.cpu().numpy(), [[1.0, 0.0]], atol=1e-6)
    np.testing.assert_allclose(cA.cpu().numpy()[0], [[1.0, 0.0], [0.0, 0.0]], atol=1e-6)


def test_bad_symbol_sets_status_and_nan():
    rng = np.random.default_rng(1)
    pi, A, B = synth.random_model(rng, 2, 4, 6)
    sym, off, ln = _pack([[0, 1, 2], [0, 6, 1], [5, 5], [3, -1]])
    ll, sc, path, sf, sv, seqs, t = _run_all(pi, A, B, sym, off, ln)
    assert sf & hmm.HMM_STATUS_SYMBOL and sv & hmm.HMM_STATUS_SYMBOL
    assert np.all(np.isnan(ll[1])) and np.all(np.isnan(ll[3]))
    assert np.all(np.isfinite(ll[0])) and np.all(np.isfinite(ll[2]))
    assert np.all(np.isnan(sc[1])) and np.all(np.isfinite(sc[0]))
    assert np.all(path[3:6] == -1)
    import torch
    lab = seqs.labelled(torch.tensor([0, 1, 0, 1], dtype=torch.int32, device="cuda"))
    fll, cpi, cA, cB = hmm.hmm_forward_backward(*t, lab)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) & hmm.HMM_STATUS_SYMBOL
    assert np.isnan(fll.cpu().numpy()[1]) and np.isfinite(cA.cpu().numpy()).all()


def test_bad_sequence_layout_sets_status():
    rng = np.random.default_rng(2)
    pi, A, B = synth.random_model(rng, 2, 4, 6)
    sym = rng.integers(0, 6, size=20).astype(np.int32)
    off = np.array([0, 5, 18, -1, 3], np.int64)
    ln = np.array([5, 5, 5, 2, -3], np.int32)       # [2] runs past the end; [3],[4] negative
    ll, sc, _, sf, sv, _, _ = _run_all(pi, A, B, sym, off, ln, max_len=8)
    assert sf & hmm.HMM_STATUS_SEQ and sv & hmm.HMM_STATUS_SEQ
    assert np.all(np.isfinite(ll[:2])) and np.all(np.isnan(ll[2:]))
    # a length above max_len is rejected too
    ll2, _, _, sf2, _, _, _ = _run_all(pi, A, B, sym, off[:2], ln[:2], max_len=4)
    assert sf2 & hmm.HMM_STATUS_SEQ and np.all(np.isnan(ll2))
    # a bad model index in labelled mode
    ll3, _, _, sf3, _, _, _ = _run_all(pi, A, B, sym, off[:2], ln[:2], mos=np.array([0, 2], np.int32))
    assert sf3 & hmm.HMM_STATUS_SEQ and np.isfinite(ll3[0]) and np.isnan(ll3[1])


def test_overlapping_views_exceeding_total_obs():
    rng = np.random.default_rng(5)
    pi, A, B = synth.random_model(rng, 1, 4, 3)
    sym = rng.integers(0, 3, size=10).astype(np.int32)
    off = np.array([0, 0, 0], np.int64)
    ln = np.array([10, 10, 10], np.int32)
    ll, sc, _, sf, sv, _, _ = _run_all(pi, A, B, sym, off, ln)
    assert sf == 0 and np.all(np.isfinite(ll)) and ll[0, 0] == ll[1, 0] == ll[2, 0]
    # backpointers for 30 steps do not fit in total_obs = 10: later ones are rejected
    assert sv & hmm.HMM_STATUS_SEQ and np.isfinite(sc[0, 0]) and np.isnan(sc).sum() >= 1


def test_bad_parameters_set_status_and_nan():
    rng = np.random.default_rng(3)
    pi, A, B = synth.random_model(rng, 2, 4, 6)
    A = A.copy()
    A[1, 2, 3] = np.nan
    sym, off, ln = _pack([[0, 1, 2, 3, 4]])
    ll, sc, path, sf, sv, _, _ = _run_all(pi, A, B, sym, off, ln)
    assert sf & hmm.HMM_STATUS_PARAM and sv & hmm.HMM_STATUS_PARAM
    assert np.isnan(ll[0, 1]) and np.all(np.isnan(sc))
    B2 = B.copy()
    B2[0, 0, 0] = -0.5
    _, _, _, sf, _, _, _ = _run_all(pi, A, B2, sym, off, ln)
    assert sf & hmm.HMM_STATUS_PARAM


def test_one_very_long_sequence_among_short_ones():
    w = synth.make_workload("gradient", n_seqs=40, lengths=("uniform", 1, 30))
    long = synth.make_workload("gradient", n_seqs=1, lengths=("fixed", 6000), seed=7)
    sym = np.concatenate([w.symbols, long.symbols])
    ln = np.concatenate([w.lengths, long.lengths])
    off = np.zeros(ln.size, np.int64)
    off[1:] = np.cumsum(ln.astype(np.int64))[:-1]
    labels = np.concatenate([w.labels, long.labels])
    import torch
    seqs = hmm.Sequences.from_numpy(sym, off, ln, model_of_seq=labels)
    t = [torch.from_numpy(x).cuda() for x in (w.pi, w.A, w.B)]
    P = oparams(w)
    rll, rpi, rA, rB, _ = oracle.forward_backward(P, sym, off, ln, labels, nthreads=8)
    ll, cpi, cA, cB = hmm.hmm_forward_backward(*t, seqs)
    assert np.all(np.abs(ll.cpu().numpy() - rll) <= ll_tol(ln))
    for g, r in zip((cpi, cA, cB), (rpi, rA, rB)):
        assert rel_l2(g.cpu().numpy(), r) <= COUNT_RTOL
    fl, _ = hmm.hmm_forward(*t, seqs)
    assert np.all(np.abs(fl.cpu().numpy() - rll) <= ll_tol(ln))


def test_empty_batch():
    import torch
    rng = np.random.default_rng(6)
    pi, A, B = synth.random_model(rng, 2, 4, 6)
    seqs = hmm.Sequences.from_numpy(np.zeros(0, np.int32), np.zeros(0, np.int64),
                                    np.zeros(0, np.int32), max_len=0)
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    ll, am = hmm.hmm_forward(*t, seqs)
    assert ll.shape == (0, 2)
    _, cpi, cA, cB = hmm.hmm_forward_backward(*t, seqs.labelled(torch.zeros(0, dtype=torch.int32,
                                                                            device="cuda")))
    assert float(cA.abs().sum()) == 0.0


def test_cuda_graph_replay_matches_eager():
    import torch
    w = synth.make_workload("batched", n_seqs=512)
    seqs, pi, A, B = to_gpu(w)
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    ws1, ws2, ws3 = hmm.Workspace(), hmm.Workspace(), hmm.Workspace()
    eager_ll, eager_am = hmm.hmm_forward(pi, A, B, seqs, workspace=ws1)
    eager_sc, eager_best, eager_path = hmm.hmm_viterbi(pi, A, B, seqs, workspace=ws2)
    eager_fb = hmm.hmm_forward_backward(pi, A, B, lab, workspace=ws3)
    outs = [torch.empty_like(eager_ll), torch.empty_like(eager_am), torch.empty_like(eager_sc),
            torch.empty_like(eager_best), torch.empty_like(eager_path)]
    fb_out = [torch.empty_like(x) for x in eager_fb]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            hmm.hmm_forward(pi, A, B, seqs, loglik=outs[0], argmax=outs[1], workspace=ws1)
            hmm.hmm_viterbi(pi, A, B, seqs, score=outs[2], best_model=outs[3], path=outs[4],
                            workspace=ws2)
            hmm.hmm_forward_backward(pi, A, B, lab, loglik=fb_out[0], counts=tuple(fb_out[1:]),
                                     workspace=ws3)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, (eager_ll, eager_am, eager_sc, eager_best, eager_path)):
        assert torch.equal(a, b)
    for a, b in zip(fb_out, eager_fb):
        assert torch.equal(a, b)


@pytest.mark.parametrize("case", [("training", None), ("large", None), ("large", 300)],
                         ids=["bf16-64", "bf16-128", "bf16-512"])
def test_tensor_core_graph_replay_matches_eager(case):
    """The tensor-core forward (N = 64, 128 and the 512-state kernel) and
    adjoint (N = 64, 128) captured in one CUDA graph: replays are bitwise the
    eager results (fixed tile plan, fixed reduction order)."""
    import torch
    name, n_big = case
    over = {"K": 2} if n_big is None else {"K": 2, "N": n_big, "M": 40}
    w = synth.make_workload(name, n_seqs=300, lengths=("uniform", 1, 90), **over)
    seqs, pi, A, B = to_gpu(w)
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    ws1, ws2 = hmm.Workspace(), hmm.Workspace()
    prec = hmm.HMM_BF16_MMA
    with_fb = w.N <= 128
    eager = list(hmm.hmm_forward(pi, A, B, seqs, precision=prec, workspace=ws1))
    if with_fb:
        eager += list(hmm.hmm_forward_backward(pi, A, B, lab, precision=prec, workspace=ws2))
    outs = [torch.empty_like(x) for x in eager]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            hmm.hmm_forward(pi, A, B, seqs, precision=prec, loglik=outs[0], argmax=outs[1],
                            workspace=ws1)
            if with_fb:
                hmm.hmm_forward_backward(pi, A, B, lab, precision=prec, loglik=outs[2],
                                         counts=tuple(outs[3:]), workspace=ws2)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert hmm.hmm_get_device_status(ws1) == 0
    for a, b in zip(outs, eager):
        assert torch.equal(a, b)


def test_concurrent_streams_match_serial():
    """Recognition and the adjoint on three streams with their own workspaces
    (as the batched bench step runs them) give the serial results bitwise."""
    import torch
    w = synth.make_workload("batched", n_seqs=700)
    seqs, pi, A, B = to_gpu(w)
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    ws = [hmm.Workspace() for _ in range(3)]
    ser = [hmm.hmm_forward(pi, A, B, seqs, workspace=ws[0]),
           hmm.hmm_viterbi(pi, A, B, seqs, workspace=ws[1]),
           hmm.hmm_forward_backward(pi, A, B, lab, workspace=ws[2])]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(3)]
    cur = torch.cuda.current_stream()
    for st in streams:
        st.wait_stream(cur)
    with torch.cuda.stream(streams[0]):
        c0 = hmm.hmm_forward_backward(pi, A, B, lab, workspace=ws[2])
    with torch.cuda.stream(streams[1]):
        c1 = hmm.hmm_viterbi(pi, A, B, seqs, workspace=ws[1])
    with torch.cuda.stream(streams[2]):
        c2 = hmm.hmm_forward(pi, A, B, seqs, workspace=ws[0])
    for st in streams:
        cur.wait_stream(st)
    torch.cuda.synchronize()
    for got, ref in ((c2, ser[0]), (c1, ser[1]), (c0, ser[2])):
        for a, b in zip(got, ref):
            if a is not None:
                assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["batched", "gradient"])
def test_full_size_sampled_and_invariants(name):
    """The full configuration in the launch shape the bench uses; the oracle
    checks a sample of sequences, properties check every output."""
    import torch
    w = synth.make_workload(name)
    seqs, pi, A, B = to_gpu(w)
    ll, am = hmm.hmm_forward(pi, A, B, seqs)
    sc, best, path = hmm.hmm_viterbi(pi, A, B, seqs)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    ll, am, sc, best, path = (x.cpu().numpy() for x in (ll, am, sc, best, path))
    T = w.lengths.astype(np.float64)[:, None]
    tol = ll_tol(w.lengths)[:, None]
    assert np.all(sc <= ll + tol)
    assert np.all(ll <= sc + T * math.log(w.N) + tol)
    np.testing.assert_array_equal(best, np.argmax(sc, axis=1))
    assert np.all((path >= 0) & (path < w.N))
    # decoded path's joint log-probability equals its score (float64 recompute)
    lpi, lA, lB = (np.log(x.astype(np.float64)) for x in (w.pi, w.A, w.B))
    for s in range(0, w.S, 97):
        k, o = best[s], w.symbols[w.offsets[s]: w.offsets[s] + w.lengths[s]]
        q = path[w.offsets[s]: w.offsets[s] + w.lengths[s]]
        j = lpi[k, q[0]] + lB[k, q[0], o[0]] + np.sum(lA[k, q[:-1], q[1:]] + lB[k, q[1:], o[1:]])
        assert abs(j - sc[s, k]) <= tol[s, 0]
    # oracle on a sample
    idx = np.random.default_rng(0).choice(w.S, size=48, replace=False)
    P = oparams(w)
    sub = (w.symbols, w.offsets[idx], w.lengths[idx])
    rll, _, _ = oracle.forward(P, *sub, nthreads=8)
    rs, _, _, _, _ = oracle.viterbi(P, *sub, want_path=False, nthreads=8)
    assert np.all(np.abs(ll[idx] - rll) <= tol[idx])
    assert np.all(np.abs(sc[idx] - rs) <= tol[idx])
    # labelled adjoint: count identities at full size
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    fll, cpi, cA, cB = hmm.hmm_forward_backward(pi, A, B, lab)
    cpi, cA, cB = (x.cpu().numpy().astype(np.float64) for x in (cpi, cA, cB))
    for k in range(w.K):
        sel = w.labels == k
        assert cpi[k].sum() == pytest.approx(sel.sum(), rel=1e-4)
        assert cA[k].sum() == pytest.approx((w.lengths[sel] - 1).sum(), rel=1e-4)
        assert cB[k].sum() == pytest.approx(w.lengths[sel].sum(), rel=1e-4)
    np.testing.assert_allclose(fll.cpu().numpy(), ll[np.arange(w.S), w.labels], rtol=1e-6)


def test_autotuner_installs_candidates_and_keeps_results():
    """The autotuner times every candidate (lanes per pair of each kernel and
    the adjoint's segment ranges) on a batch, installs valid choices, and
    the outputs under its choices match those under the defaults."""
    import torch
    from paper_1310_3322_gb300 import tune
    w = synth.make_workload("batched", n_seqs=256, lengths=("uniform", 10, 200))
    seqs, pi, A, B = to_gpu(w)
    lab = seqs.labelled(torch.from_numpy(w.labels).cuda())
    ref_ll = hmm.hmm_forward(pi, A, B, seqs)[0]
    ref_fb = hmm.hmm_forward_backward(pi, A, B, lab)
    try:
        out = tune.autotune(pi, A, B, seqs, lab, repeats=1, cache=None)
        assert set(out) == {"forward", "viterbi_scores", "viterbi_paths", "adjoint",
                            "adjoint_ranges"}
        for op, name in tune.KERNEL_OF.items():
            assert out[name]["lanes"] in hmm.hmm_tuning_candidates(op, 16)
            assert hmm.hmm_get_tuning(op, 16) == out[name]["lanes"]
        torch.testing.assert_close(hmm.hmm_forward(pi, A, B, seqs)[0], ref_ll, rtol=0, atol=1e-4)
        for a, b in zip(hmm.hmm_forward_backward(pi, A, B, lab), ref_fb):
            torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-4)
    finally:
        for op in tune.KERNEL_OF:
            hmm.hmm_set_tuning(op, 16, 0)
