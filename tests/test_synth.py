"""Seeded generators: determinism, shapes, the length laws and that symbols
are drawn from the labelled model (CPU only)."""
import numpy as np
import pytest

from paper_1310_3322_gb300 import synth


@pytest.mark.parametrize("name", ["plain", "batched", "gradient", "teamwork"])
def test_workload_shapes_and_determinism(name):
    a = synth.make_workload(name)
    b = synth.make_workload(name)
    spec = synth.SPECS[name]
    assert (a.K, a.N, a.M, a.S) == (spec["K"], spec["N"], spec["M"], spec["S"])
    np.testing.assert_array_equal(a.symbols, b.symbols)
    assert a.symbols.dtype == np.int32 and a.offsets.dtype == np.int64
    assert a.lengths.dtype == np.int32 and a.labels.dtype == np.int32
    assert a.total_obs == int(a.lengths.sum())
    np.testing.assert_array_equal(a.offsets[1:], np.cumsum(a.lengths)[:-1])
    assert a.symbols.min() >= 0 and a.symbols.max() < a.M
    assert a.labels.min() >= 0 and a.labels.max() < a.K
    for arr in (a.pi, a.A, a.B):
        assert arr.dtype == np.float32
        np.testing.assert_allclose(arr.sum(-1), 1.0, rtol=1e-5)


def test_length_laws():
    w = synth.make_workload("batched")
    assert w.lengths.min() >= 30 and w.lengths.max() <= 300
    assert abs(w.lengths.mean() - 165) < 5
    T = synth.draw_lengths(synth.SPECS["training"], 200000, 1310005)
    assert T.min() >= 50 and T.max() <= 1000
    assert abs(T.mean() - 223.6) < 3      # mean of T^-1.5 on [50,1000]


def test_sticky_transitions():
    w = synth.make_workload("batched", n_seqs=4)
    d = np.diagonal(w.A, axis1=1, axis2=2)
    assert d.min() >= 0.6 - 1e-6 and d.max() <= 0.9 + 1e-6


def test_first_symbol_distribution():
    # P(o_1 = m) = sum_i pi_i b_i(m) for the generating model
    w = synth.make_workload("plain", n_seqs=40000, lengths=("fixed", 1))
    expect = (w.pi[0].astype(np.float64)[:, None] * w.B[0]).sum(0)
    freq = np.bincount(w.symbols, minlength=w.M) / w.S
    assert np.abs(freq - expect).max() < 0.01


def test_resample_changes_only_selected():
    w = synth.make_workload("batched", n_seqs=20, lengths=("uniform", 5, 9))
    v = synth.resample(w, [3, 7], 0)
    for s in range(w.S):
        a = w.symbols[w.offsets[s]: w.offsets[s] + w.lengths[s]]
        b = v.symbols[v.offsets[s]: v.offsets[s] + v.lengths[s]]
        if s not in (3, 7):
            np.testing.assert_array_equal(a, b)


def test_role_split_partitions_sequences_and_models():
    w = synth.make_workload("teamwork", n_seqs=300)
    parts = synth.role_split(w, w.meta["roles"])
    assert len(parts) == 4 and sum(p.S for p in parts) == w.S
    seen = np.concatenate([p.meta["index"] for p in parts])
    np.testing.assert_array_equal(np.sort(seen), np.arange(w.S))
    for r, p in enumerate(parts):
        assert p.K == 6 and p.labels.min() >= 0 and p.labels.max() < 6
        np.testing.assert_array_equal(p.A, w.A[6 * r: 6 * r + 6])
        np.testing.assert_array_equal(p.offsets[1:], np.cumsum(p.lengths)[:-1])
        for j, s in enumerate(p.meta["index"]):
            assert w.labels[s] // 6 == r and w.labels[s] % 6 == p.labels[j]
            np.testing.assert_array_equal(
                p.symbols[p.offsets[j]: p.offsets[j] + p.lengths[j]],
                w.symbols[w.offsets[s]: w.offsets[s] + w.lengths[s]])


def test_wide_and_long_sequence_recipes():
    """The 512-state recipe (Dirichlet(0.3) rows, T ~ U{100..500}) and the
    few-long-sequences recipe (T ~ U{2^19..2^20}): shapes, determinism and
    length laws (the long one checked on its length draw alone)."""
    w = synth.make_workload("cuhmm", n_seqs=64)
    assert (w.K, w.N, w.M, w.S) == (1, 512, 64, 64)
    assert w.lengths.min() >= 100 and w.lengths.max() <= 500
    np.testing.assert_array_equal(w.symbols, synth.make_workload("cuhmm", n_seqs=64).symbols)
    np.testing.assert_allclose(w.A.sum(-1), 1.0, rtol=1e-5)
    spec = synth.SPECS["longseq"]
    T = synth.draw_lengths(spec, spec["S"], synth.SEEDS["longseq"])
    assert T.size == 8 and T.min() >= 1 << 19 and T.max() <= 1 << 20
    w = synth.make_workload("longseq", n_seqs=3, lengths=("uniform", 50, 60))
    assert (w.K, w.N, w.M) == (4, 32, 64) and w.symbols.max() < w.M
    # the "batched" parameter recipe: self-transitions in [0.6, 0.9]
    d = np.diagonal(w.A, axis1=1, axis2=2)
    assert d.min() >= 0.6 - 1e-6 and d.max() <= 0.9 + 1e-6
