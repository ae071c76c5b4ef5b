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
