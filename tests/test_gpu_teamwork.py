"""Paper-shaped recognition (Sec. 5.7): four roles, one set of six action HMMs
per role (N = 5 hidden states, 64 symbols from six binary features), many
short sequences. Every role's sequences are scored against that role's six
models by one forward call (log-likelihoods + argmax) and one Viterbi call
(scores, decoded action, best path), all reading one shared packed symbol
buffer through per-role offsets and writing one shared path buffer; checked
against the FP64 oracle role by role."""
import numpy as np
import pytest

import oracle
from helpers import ll_tol, margin_filtered
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu


def _packed_roles(n_seqs, lengths):
    w = synth.make_workload("teamwork", n_seqs=n_seqs, lengths=lengths)
    parts = [margin_filtered(p) for p in synth.role_split(w, w.meta["roles"])]
    base = np.cumsum([0] + [p.total_obs for p in parts])
    sym = np.concatenate([p.symbols for p in parts]).astype(np.int32)
    return w, parts, base, sym


@pytest.mark.parametrize("lengths", [("uniform", 1, 120), ("uniform", 20, 120)])
def test_per_role_recognition_matches_oracle(lengths):
    import torch
    w, parts, base, sym = _packed_roles(1600, lengths)
    dev = torch.device("cuda")
    dsym = torch.from_numpy(sym).to(dev)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    path = torch.full((sym.size,), -7, dtype=torch.int32, device=dev)
    Kr = w.K // w.meta["roles"]
    for r, p in enumerate(parts):
        off = p.offsets + base[r]
        seqs = hmm.Sequences(symbols=dsym, offsets=torch.from_numpy(off).to(dev),
                             lengths=torch.from_numpy(p.lengths).to(dev),
                             max_len=int(p.lengths.max()))
        sl = slice(r * Kr, (r + 1) * Kr)
        ll, am = hmm.hmm_forward(pi[sl], A[sl], B[sl], seqs)
        sc, best, _ = hmm.hmm_viterbi(pi[sl], A[sl], B[sl], seqs, path=path)
        assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
        P = oracle.params(p.pi, p.A, p.B)
        rll, ram, _ = oracle.forward(P, sym, off, p.lengths, nthreads=8)
        rs, rbest, rpath, _, _ = oracle.viterbi(P, sym, off, p.lengths, nthreads=8)
        tol = ll_tol(p.lengths)[:, None]
        assert np.all(np.abs(ll.cpu().numpy() - rll) <= tol)
        assert np.all(np.abs(sc.cpu().numpy() - rs) <= tol)
        np.testing.assert_array_equal(best.cpu().numpy(), rbest)
        # the forward's argmax: unique where the two best models are apart
        srt = np.sort(rll, axis=1)
        clear = srt[:, -1] - srt[:, -2] > 2 * tol[:, 0]
        np.testing.assert_array_equal(am.cpu().numpy()[clear], ram[clear])
        seg = slice(base[r], base[r + 1])
        np.testing.assert_array_equal(path.cpu().numpy()[seg], rpath[seg])
    # every position of the shared path buffer was written by exactly its role
    assert np.all(path.cpu().numpy() >= 0)


@pytest.mark.parametrize("lengths", [("uniform", 0, 120), ("uniform", 20, 120)])
def test_model_sets_one_call_matches_per_role_oracle(lengths):
    """All four roles in ONE forward and ONE Viterbi call: sequence s is
    scored against its role's six models only (model_base = 6 * role,
    model_span = 6), outputs [S][6] with role-relative model indices."""
    import torch
    w, parts, base, sym = _packed_roles(1200, lengths)
    Kr = w.K // w.meta["roles"]
    dev = torch.device("cuda")
    off = np.concatenate([p.offsets + base[r] for r, p in enumerate(parts)])
    lens = np.concatenate([p.lengths for p in parts])
    mbase = np.concatenate([np.full(p.S, r * Kr, np.int32) for r, p in enumerate(parts)])
    # interleave the roles so neighbouring sequences use different sets
    perm = np.random.default_rng(5).permutation(off.size)
    seqs = hmm.Sequences(symbols=torch.from_numpy(sym).to(dev),
                         offsets=torch.from_numpy(off[perm]).to(dev),
                         lengths=torch.from_numpy(lens[perm]).to(dev),
                         max_len=int(lens.max()))
    seqs = seqs.model_sets(torch.from_numpy(mbase[perm]).to(dev), Kr)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    path = torch.full((sym.size,), -7, dtype=torch.int32, device=dev)
    ll, am = hmm.hmm_forward(pi, A, B, seqs)
    sc, best, _ = hmm.hmm_viterbi(pi, A, B, seqs, path=path)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    assert ll.shape == (off.size, Kr) and sc.shape == (off.size, Kr)
    ll, am, sc, best = (x.cpu().numpy() for x in (ll, am, sc, best))
    inv = np.argsort(perm)  # row of the call's output for each (role-major) sequence
    row0 = 0
    for r, p in enumerate(parts):
        rows = inv[row0:row0 + p.S]
        row0 += p.S
        P = oracle.params(p.pi, p.A, p.B)
        o = p.offsets + base[r]
        rll, ram, _ = oracle.forward(P, sym, o, p.lengths, nthreads=8)
        rs, rbest, rpath, _, _ = oracle.viterbi(P, sym, o, p.lengths, nthreads=8)
        tol = ll_tol(p.lengths)[:, None]
        assert np.all(np.abs(ll[rows] - rll) <= tol)
        assert np.all(np.abs(sc[rows] - rs) <= tol)
        np.testing.assert_array_equal(best[rows], rbest)
        srt = np.sort(rll, axis=1)
        clear = srt[:, -1] - srt[:, -2] > 2 * tol[:, 0]
        np.testing.assert_array_equal(am[rows][clear], ram[clear])
        seg = slice(base[r], base[r + 1])
        np.testing.assert_array_equal(path.cpu().numpy()[seg], rpath[seg])


def test_model_set_out_of_range_is_flagged():
    """A set that runs past the last model marks its sequence (NaN score,
    best model -1, status bit) and leaves the other sequences intact."""
    import torch
    w = synth.make_workload("teamwork", n_seqs=64, lengths=("uniform", 5, 40))
    dev = torch.device("cuda")
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device=dev)
    mbase = np.zeros(w.S, np.int32)
    mbase[7] = w.K - 2  # span 6 would reach model K + 3
    seqs = seqs.model_sets(torch.from_numpy(mbase).to(dev), 6)
    pi, A, B = (torch.from_numpy(x).to(dev) for x in (w.pi, w.A, w.B))
    ll, am = hmm.hmm_forward(pi, A, B, seqs)
    st = hmm.hmm_get_device_status(hmm.default_workspace())
    assert st & hmm.HMM_STATUS_SEQ
    ll, am = ll.cpu().numpy(), am.cpu().numpy()
    assert np.isnan(ll[7]).all() and am[7] == -1
    ok = np.arange(w.S) != 7
    P = oracle.params(w.pi[:6], w.A[:6], w.B[:6])
    rll, _, _ = oracle.forward(P, w.symbols, w.offsets, w.lengths, nthreads=8)
    assert np.all(np.abs(ll[ok] - rll[ok]) <= ll_tol(w.lengths[ok])[:, None])


def test_padding_is_invisible():
    """An N = 5 model and the same model zero-padded to N = 8 (explicit zero
    rows and columns, which the library's own padding to 8 states also
    produces) give bit-identical forward and Viterbi outputs at one lane per
    pair: padded states contribute exact zeros (forward) and -inf (Viterbi)."""
    import torch
    w = synth.make_workload("teamwork", n_seqs=700, lengths=("uniform", 0, 120))
    pad = lambda x, shape: np.pad(x, [(0, s - d) for s, d in zip(shape, x.shape)])
    K, M = w.K, w.M
    p5 = [torch.from_numpy(x).cuda() for x in (w.pi, w.A, w.B)]
    p8 = [torch.from_numpy(np.ascontiguousarray(pad(x, sh))).cuda()
          for x, sh in ((w.pi, (K, 8)), (w.A, (K, 8, 8)), (w.B, (K, 8, M)))]
    seqs = hmm.Sequences.from_numpy(w.symbols, w.offsets, w.lengths, device="cuda")
    for op in (hmm.HMM_OP_FORWARD, hmm.HMM_OP_VITERBI):
        hmm.hmm_set_tuning(op, 8, 1)
    try:
        l5, a5 = hmm.hmm_forward(*p5, seqs)
        l8, a8 = hmm.hmm_forward(*p8, seqs)
        s5, b5, _ = hmm.hmm_viterbi(*p5, seqs, want_path=False)
        s8, b8, _ = hmm.hmm_viterbi(*p8, seqs, want_path=False)
    finally:
        for op in (hmm.HMM_OP_FORWARD, hmm.HMM_OP_VITERBI):
            hmm.hmm_set_tuning(op, 8, 0)
    assert torch.equal(l5, l8) and torch.equal(a5, a8)
    assert torch.equal(s5, s8) and torch.equal(b5, b8)
    P = oracle.params(w.pi, w.A, w.B)
    rll, _, _ = oracle.forward(P, w.symbols, w.offsets, w.lengths, nthreads=8)
    assert np.all(np.abs(l5.cpu().numpy() - rll) <= ll_tol(w.lengths)[:, None])
