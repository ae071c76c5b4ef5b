"""Parallel-in-time forward (chunk products of A diag(b(o_t)) + ordered
combine) against the FP64 oracle's forward (Rabiner eqs. 19-21) and against
the sequential FP32 forward: every chunk boundary case (T = 0, 1, 2, a
multiple of the chunk plus 0, 1, 2), all three model modes, models with zero
transitions (rows of a chunk product that die), impossible sequences,
invalid symbols inside a chunk, and CUDA-graph replay."""
import numpy as np
import pytest

import oracle
from helpers import ll_tol, oparams
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu


def _gpu(w, labelled=False, device="cuda"):
    return hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths,
                                    model_of_seq=w.labels if labelled else None, device=device)


def _params(w, device="cuda"):
    import torch
    return tuple(torch.from_numpy(np.ascontiguousarray(x)).to(device) for x in (w.pi, w.A, w.B))


def _edge_lengths(L):
    return [0, 1, 2, 3, L - 1, L, L + 1, L + 2, 2 * L + 1, 3 * L + 5, 7 * L + 3]


def _workload(N, L, K=3, M=16, extra=9, seed=11, lo=50, hi=4000):
    rng = np.random.default_rng(seed)
    lengths = np.array(_edge_lengths(L) + list(rng.integers(lo, hi + 1, size=extra)), np.int32)
    w = synth.make_workload("batched", n_seqs=lengths.size, seed=1310100 + N, K=K, N=N, M=M,
                            lengths=("uniform", 1, 1))
    # same parameters, the edge-case lengths (symbols redrawn for them)
    w = synth.replace(w, lengths=lengths, offsets=np.concatenate(
        [[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64),
        symbols=np.zeros(int(lengths.sum()), np.int32))
    return synth.resample(w, np.arange(w.S), 0)


@pytest.mark.parametrize("N", [3, 5, 16, 32])
@pytest.mark.parametrize("chunk", [0, 16, 37])
def test_scan_all_models_matches_oracle(N, chunk):
    w = _workload(N, chunk or 64)
    pi, A, B = _params(w)
    ll, am = hmm.hmm_forward_scan(pi, A, B, _gpu(w), chunk=chunk)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    rll, ram, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths, nthreads=8)
    ll, am = ll.cpu().numpy(), am.cpu().numpy()
    tol = ll_tol(w.lengths)[:, None]
    assert np.all(np.abs(ll - rll) <= tol), np.max(np.abs(ll - rll) / tol)
    assert np.all(ll[w.lengths == 0] == 0.0)
    srt = np.sort(rll, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * tol[:, 0]
    np.testing.assert_array_equal(am[clear], ram[clear])
    # the sequential FP32 forward on the same inputs: same numbers up to rounding order
    sl, _ = hmm.hmm_forward(pi, A, B, _gpu(w))
    assert np.all(np.abs(ll - sl.cpu().numpy()) <= 1e-5 * np.maximum(w.lengths, 1)[:, None])


def test_scan_labelled_and_model_sets():
    import torch
    w = _workload(8, 32, K=6)
    pi, A, B = _params(w)
    P = oparams(w)
    ll, am = hmm.hmm_forward_scan(pi, A, B, _gpu(w, labelled=True), chunk=32)
    assert am is None
    rll, _, _ = oracle.forward(P, w.symbols, w.offsets, w.lengths, w.labels, nthreads=8)
    assert np.all(np.abs(ll.cpu().numpy() - rll) <= ll_tol(w.lengths))
    # model sets: sequence s against models 3 (s % 2) .. 3 (s % 2) + 2
    base = (3 * (np.arange(w.S) % 2)).astype(np.int32)
    seqs = _gpu(w).model_sets(torch.from_numpy(base).cuda(), 3)
    ll, am = hmm.hmm_forward_scan(pi, A, B, seqs, chunk=16)
    full, _, _ = oracle.forward(P, w.symbols, w.offsets, w.lengths, nthreads=8)
    ref = np.stack([full[s, base[s]:base[s] + 3] for s in range(w.S)])
    tol = ll_tol(w.lengths)[:, None]
    assert ll.shape == (w.S, 3)
    assert np.all(np.abs(ll.cpu().numpy() - ref) <= tol)
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * tol[:, 0]
    np.testing.assert_array_equal(am.cpu().numpy()[clear], np.argmax(ref, axis=1)[clear])


def test_scan_long_sequences_match_sequential_and_oracle():
    w = synth.make_workload("longseq", n_seqs=3, lengths=("uniform", 20000, 30000))
    pi, A, B = _params(w)
    ll, am = hmm.hmm_forward_scan(pi, A, B, _gpu(w))
    sl, sam = hmm.hmm_forward(pi, A, B, _gpu(w))
    rll, ram, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths, nthreads=8)
    ll = ll.cpu().numpy()
    tol = ll_tol(w.lengths)[:, None]
    assert np.all(np.abs(ll - rll) <= tol)
    # the measured error stays far inside the 1e-4 T bound
    assert np.all(np.abs(ll - rll) <= 1e-6 * w.lengths[:, None])
    np.testing.assert_array_equal(am.cpu().numpy(), ram)
    np.testing.assert_array_equal(sam.cpu().numpy(), ram)


def test_scan_dead_rows_and_impossible_sequences():
    """Left-to-right models (a_ij = 0 for j < i): the chunk-product rows of
    later start states cannot reach earlier states, and a symbol no state of
    a model emits makes the sequence impossible (-inf)."""
    rng = np.random.default_rng(3)
    K, N, M = 2, 6, 8
    A = np.triu(rng.random((K, N, N)) + 0.05).astype(np.float32)
    A /= A.sum(axis=2, keepdims=True)
    B = rng.dirichlet(np.ones(M), size=(K, N)).astype(np.float32)
    B[1, :, 7] = 0.0  # model 1 never emits symbol 7
    B /= B.sum(axis=2, keepdims=True)
    pi = np.zeros((K, N), np.float32)
    pi[:, 0] = 1.0
    lengths = np.array([0, 1, 5, 33, 64, 65, 300, 1000], np.int32)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    symbols = rng.integers(0, 7, size=int(lengths.sum())).astype(np.int32)
    symbols[offsets[6] + 150] = 7  # impossible under model 1 only
    symbols[offsets[7] + 999] = 7
    import torch
    dev = torch.device("cuda")
    tp = [torch.from_numpy(x).to(dev) for x in (pi, A, B)]
    seqs = hmm.Sequences.from_numpy(symbols, offsets, lengths, device=dev)
    ll, am = hmm.hmm_forward_scan(*tp, seqs, chunk=16)
    rll, ram, _ = oracle.forward(oracle.params(pi, A, B), symbols, offsets, lengths, nthreads=4)
    ll = ll.cpu().numpy()
    assert np.isneginf(ll[6, 1]) and np.isneginf(ll[7, 1]) and np.isneginf(rll[6, 1])
    fin = np.isfinite(rll)
    assert np.array_equal(fin, np.isfinite(ll))
    assert np.all(np.abs(ll[fin] - rll[fin]) <= ll_tol(np.broadcast_to(lengths[:, None], rll.shape)[fin]))
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0


def test_scan_invalid_symbol_inside_a_chunk():
    w = _workload(5, 16, K=2, extra=3)
    sym = w.symbols.copy()
    s_bad = 9  # length 3 L + 5 = 53: symbol 40 lies in the third chunk
    sym[w.offsets[s_bad] + 40] = w.M + 3
    w = synth.replace(w, symbols=sym)
    pi, A, B = _params(w)
    ll, am = hmm.hmm_forward_scan(pi, A, B, _gpu(w), chunk=16)
    st = hmm.hmm_get_device_status(hmm.default_workspace())
    assert st & hmm.HMM_STATUS_SYMBOL
    ll, am = ll.cpu().numpy(), am.cpu().numpy()
    assert np.isnan(ll[s_bad]).all() and am[s_bad] == -1
    ok = np.arange(w.S) != s_bad
    rll, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets, w.lengths)
    assert np.all(np.abs(ll[ok] - rll[ok]) <= ll_tol(w.lengths[ok])[:, None])


def test_scan_graph_replay_is_bitwise_identical():
    import torch
    w = _workload(16, 64, K=2, extra=5)
    pi, A, B = _params(w)
    seqs = _gpu(w)
    ws = hmm.Workspace(torch.device("cuda"))
    ll0, am0 = hmm.hmm_forward_scan(pi, A, B, seqs, chunk=64, workspace=ws)
    ll = torch.empty_like(ll0)
    am = torch.empty_like(am0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        hmm.hmm_forward_scan(pi, A, B, seqs, chunk=64, loglik=ll, argmax=am, workspace=ws)
        with torch.cuda.graph(g, stream=side):
            hmm.hmm_forward_scan(pi, A, B, seqs, chunk=64, loglik=ll, argmax=am, workspace=ws)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(3):
        ll.fill_(7.0)
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ll, ll0) and torch.equal(am, am0)


def _scan_launches(fn):
    hmm.hmm_timing_reset()
    hmm.hmm_timing_enable(True)
    out = fn()
    kt = hmm.hmm_timing_read()
    hmm.hmm_timing_enable(False)
    return out, kt["scan_chunks"][0]


def test_auto_precision_takes_the_scan_for_few_long_sequences():
    """HMM_AUTO picks the parallel-in-time forward for a batch of few long
    sequences (the workspace query leaves room for it; the static-scratch
    entry point too, its chunk products fitting the scratch) and the
    sequential recursion for many short ones."""
    import torch
    w = synth.make_workload("longseq", n_seqs=2, K=2, N=16, lengths=("uniform", 9000, 12000))
    pi, A, B = _params(w)
    seqs = _gpu(w)
    ws = hmm.Workspace(torch.device("cuda"))
    (auto_ll, auto_am), n = _scan_launches(
        lambda: hmm.hmm_forward(pi, A, B, seqs, precision=hmm.HMM_AUTO, workspace=ws))
    assert n == 1
    scan_ll, scan_am = hmm.hmm_forward_scan(pi, A, B, seqs, workspace=ws)
    (seq_ll, seq_am), n = _scan_launches(
        lambda: hmm.hmm_forward(pi, A, B, seqs, precision=hmm.HMM_FP32, workspace=ws))
    assert n == 0
    assert torch.equal(auto_ll, scan_ll) and torch.equal(auto_am, scan_am)
    assert torch.equal(auto_am, seq_am)
    assert np.all(np.abs(auto_ll.cpu().numpy() - seq_ll.cpu().numpy())
                  <= 1e-5 * w.lengths[:, None])
    st_ll, _ = hmm.hmm_forward_static(pi, A, B, seqs, precision=hmm.HMM_AUTO)
    assert torch.equal(st_ll, scan_ll)
    # many short sequences: AUTO is the sequential recursion
    w2 = synth.make_workload("batched", n_seqs=64, lengths=("uniform", 30, 300))
    p2 = _params(w2)
    (a2, _), n = _scan_launches(lambda: hmm.hmm_forward(*p2, _gpu(w2), precision=hmm.HMM_AUTO))
    assert n == 0
    f2, _ = hmm.hmm_forward(*p2, _gpu(w2), precision=hmm.HMM_FP32)
    assert torch.equal(a2, f2)
