"""Tensor-core (tcgen05) forward vs the FP64 oracle, BF16 and TF32 operands.

The tensor-core path rounds the transition matrix A and the rescaled forward
variable to BF16 (unit roundoff u = 2^-8) or TF32 (u = 2^-11, round to nearest)
and accumulates in FP32; the BF16 path rounds the emission table B to BF16 as
well (TF32 keeps B in FP32). Two checks:

* against the oracle run on the model as the kernel holds it (A, and on the
  BF16 path B, rounded: the systematic part of the error removed), the
  remaining difference comes from rounding alpha each step and must stay
  within the FP32 bound 1e-4 * max(T, 1) nats plus u T;
* against the oracle on the exact model, every term of every step is a sum of
  non-negative products whose factors carry relative errors <= u (alpha and A,
  and b on the BF16 path), so |delta log P| <= 2 u T (TF32) or 3 u T (BF16)
  is a hard bound; the mean per-step error is reported.
* that hard bound is far above what the kernel does: each step's rounding
  error is a sum of N independently signed terms, so per sequence
  |delta log P| <= (u / 4) T + 2 u is required as well (2 u: one step's worth
  of slack for short sequences); measured values are printed.
* recognition: the argmax over models must agree wherever the top two models
  of the exact model are more than twice that per-sequence cap apart.
"""
import numpy as np
import pytest

import oracle
from helpers import ll_tol, oparams, to_gpu
from paper_1310_3322_gb300 import hmm, synth

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
U_TF32 = 2.0 ** -11


def bf16_round(x):
    """Round-to-nearest-even of float32 values to bfloat16, returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def tf32_round(x):
    """Round to nearest (ties away from zero) of non-negative float32 values to
    a 10-bit mantissa, returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) >> 13) << 13
    return b.astype(np.uint32).view(np.float32)


PRECISIONS = {"bf16": (hmm.HMM_BF16_MMA, U_BF16, bf16_round),
              "tf32": (hmm.HMM_TF32_MMA, U_TF32, tf32_round)}
# rounded factors per product term: alpha, A and (BF16 only) b
N_ROUNDED = {"bf16": 3, "tf32": 2}


def held_model(w, prec):
    """The model as the tensor-core path holds it: A rounded to the operand
    type, and B rounded to BF16 on the BF16 path."""
    _, _, rnd = PRECISIONS[prec]
    return oracle.params(w.pi, rnd(w.A), bf16_round(w.B) if prec == "bf16" else w.B)


def seq_cap(u, lengths):
    """Per-sequence bound |delta log P| <= (u / 4) T + 2 u (see the module text)."""
    return (u / 4) * np.asarray(lengths, np.float64) + 2 * u


CASES = [
    ("large", 48, ("uniform", 20, 400), {"K": 2}),           # N=128, M=256
    ("training", 96, ("uniform", 1, 300), {"K": 3}),         # N=64, M=128
    ("large", 40, ("uniform", 0, 200), {"K": 2, "N": 100}),  # padded to 128
    ("gradient", 60, ("uniform", 1, 150), {"K": 3, "N": 40}),  # padded to 64
    # emission tables too large for shared memory: per-row staging copies
    ("large", 40, ("uniform", 1, 150), {"K": 2, "M": 400}),
    ("training", 60, ("uniform", 1, 150), {"K": 2, "M": 900}),
]


# above 128 states: one tile per CTA with A^T streamed (BF16 only); padded
# and exact N, ragged tiles, an emission table of more than 256 symbols
WIDE_CASES = [
    ("large", 150, ("uniform", 1, 90), {"K": 2, "N": 200, "M": 64}),    # padded to 256
    ("large", 130, ("uniform", 20, 60), {"K": 2, "N": 256, "M": 300}),
    ("large", 140, ("uniform", 1, 40), {"K": 2, "N": 333, "M": 64}),    # padded to 512
    ("large", 129, ("uniform", 10, 40), {"K": 1, "N": 512, "M": 32}),
    # many short sequences: the cluster kernel's 64- and 128-row tiles (few
    # sequences take 32-row tiles)
    ("large", 2000, ("uniform", 1, 12), {"K": 1, "N": 256, "M": 64}),
    ("large", 5000, ("uniform", 1, 8), {"K": 1, "N": 256, "M": 64}),
    # emission slice too large for the cluster kernel: the streamed-A^T kernel
    ("large", 40, ("uniform", 1, 30), {"K": 2, "N": 400, "M": 200}),
]


@pytest.mark.parametrize("case", WIDE_CASES, ids=lambda c: f"{c[0]}-{c[3]}")
def test_wide_tensor_core_forward_matches_oracle(case):
    test_tensor_core_forward_matches_oracle(case, "bf16")


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[3]}")
def test_tensor_core_forward_matches_oracle(case, prec):
    precision, u, rnd = PRECISIONS[prec]
    name, S, lengths, over = case
    w = synth.make_workload(name, n_seqs=S, lengths=lengths, **over)
    seqs, pi, A, B = to_gpu(w)
    ll, am = hmm.hmm_forward(pi, A, B, seqs, precision=precision)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    ll = ll.cpu().numpy()
    T = np.maximum(w.lengths, 1).astype(np.float64)[:, None]
    # systematic rounding of the model removed: only the per-step rounding of
    # alpha (relative <= u per term, all terms non-negative) remains
    ref_r, _, _ = oracle.forward(held_model(w, prec), w.symbols, w.offsets, w.lengths, nthreads=8)
    err_r = np.abs(ll - ref_r)
    assert np.all(err_r <= u * T + ll_tol(w.lengths)[:, None]), (err_r / T).max()
    # ... and it is a random-signed error far below that bound on average
    assert np.mean(err_r / T) <= u / 8 + 1e-5, np.mean(err_r / T)
    # exact model: hard bound 2 u T (TF32) or 3 u T (BF16)
    ref, ref_am, _ = oracle.forward(oracle.params(w.pi, w.A, w.B), w.symbols, w.offsets,
                                    w.lengths, nthreads=8)
    err = np.abs(ll - ref)
    assert np.all(err <= N_ROUNDED[prec] * u * T + ll_tol(w.lengths)[:, None]), (err / T).max()
    print(f"{prec} {name} N={w.N}: max|d|/T vs exact {np.max(err / T):.2e}, "
          f"mean {np.mean(err / T):.2e}; vs held model {np.max(err_r / T):.2e}")
    cap = seq_cap(u, w.lengths)[:, None]
    assert np.all(err <= cap), f"max |d| / cap = {np.max(err / cap):.3f}"
    # recognition: argmax agrees where the top two models are well separated
    if w.K == 1:
        np.testing.assert_array_equal(am.cpu().numpy(), np.where(np.isnan(ll[:, 0]), -1, 0))
        return
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * cap[:, 0]
    np.testing.assert_array_equal(am.cpu().numpy()[clear], ref_am[clear])


def test_bf16_forward_degenerate_and_errors():
    import torch
    rng = np.random.default_rng(4)
    pi, A, B = synth.random_model(rng, 2, 70, 5)
    seqs_l = [rng.integers(0, 5, size=T).tolist() for T in (0, 1, 2, 129, 3)]
    seqs_l[2] = [0, 7]          # bad symbol
    lengths = np.array([len(x) for x in seqs_l], np.int32)
    offsets = np.zeros(len(seqs_l), np.int64)
    offsets[1:] = np.cumsum(lengths)[:-1]
    sym = np.array([x for q in seqs_l for x in q], np.int32)
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths)
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    ll, am = hmm.hmm_forward(*t, seqs, precision=hmm.HMM_BF16_MMA)
    ll = ll.cpu().numpy()
    assert hmm.hmm_get_device_status(hmm.default_workspace()) & hmm.HMM_STATUS_SYMBOL
    assert np.all(ll[0] == 0.0) and np.all(np.isnan(ll[2])) and am.cpu().numpy()[2] == -1
    ref, _, _ = oracle.forward(oracle.params(pi, A, B), sym, offsets, lengths)
    ok = np.array([True, True, False, True, True])
    assert np.all(np.abs(ll[ok] - ref[ok]) <= 3 * U_BF16 * np.maximum(lengths[ok], 1)[:, None])
    # labelled mode and small N are not served by the tensor-core path
    with pytest.raises(hmm.HmmError):
        hmm.hmm_forward(*t, seqs.labelled(torch.zeros(5, dtype=torch.int32, device="cuda")),
                        precision=hmm.HMM_BF16_MMA)
    small = [torch.from_numpy(x).cuda() for x in synth.random_model(rng, 2, 16, 5)]
    with pytest.raises(hmm.HmmError):
        hmm.hmm_forward(*small, seqs, precision=hmm.HMM_BF16_MMA)


def test_wide_forward_full_cuhmm_shape_sampled():
    """The 512-state x 512-sequence workload the bench times: sampled
    sequences against the oracle (exact model, 3uT bound)."""
    w = synth.make_workload("cuhmm")
    seqs, pi, A, B = to_gpu(w)
    ll, am = hmm.hmm_forward(pi, A, B, seqs, precision=hmm.HMM_BF16_MMA)
    assert hmm.hmm_get_device_status(hmm.default_workspace()) == 0
    ll = ll.cpu().numpy()
    assert np.all(np.isfinite(ll))
    idx = np.random.default_rng(10).choice(w.S, size=6, replace=False)
    ref, _, _ = oracle.forward(oparams(w), w.symbols, w.offsets[idx], w.lengths[idx],
                               nthreads=8)
    T = w.lengths[idx].astype(np.float64)[:, None]
    assert np.all(np.abs(ll[idx] - ref) <= 3 * U_BF16 * T + ll_tol(w.lengths[idx])[:, None])


@pytest.mark.parametrize("N", [200, 300])
def test_cluster_forward_degenerate_and_deterministic(N):
    """Above 128 states (a cluster of N_pad / 64 CTAs per tile): empty,
    one- and two-step sequences, an invalid symbol, a sequence impossible
    under one model, rows of different lengths in one tile; two calls agree
    bit for bit."""
    import torch
    rng = np.random.default_rng(12)
    K, M = 2, 16
    pi, A, B = synth.random_model(rng, K, N, M, alpha=0.5)
    B[1, :, 15] = 0.0  # model 1 never emits symbol 15
    B /= B.sum(axis=2, keepdims=True)
    lengths = np.array([0, 1, 2, 150, 3, 70, 31], np.int32)
    offsets = np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
    sym = rng.integers(0, 15, size=int(lengths.sum())).astype(np.int32)
    sym[offsets[5] + 33] = 15          # impossible under model 1 only
    sym[offsets[6] + 7] = M + 3        # invalid symbol in sequence 6
    t = [torch.from_numpy(x).cuda() for x in (pi, A, B)]
    seqs = hmm.Sequences.from_numpy(sym, offsets, lengths, device="cuda")

    def run():
        ll, am = hmm.hmm_forward(*t, seqs, precision=hmm.HMM_BF16_MMA)
        return ll.cpu().numpy(), am.cpu().numpy(), hmm.hmm_get_device_status(hmm.default_workspace())

    (ll, am, status), (ll2, am2, _) = run(), run()
    assert np.array_equal(ll, ll2, equal_nan=True) and np.array_equal(am, am2)
    assert status & hmm.HMM_STATUS_SYMBOL
    assert np.all(ll[0] == 0.0)
    assert np.all(np.isnan(ll[6])) and am[6] == -1
    assert np.isneginf(ll[5, 1]) and np.isfinite(ll[5, 0])
    ref, ref_am, _ = oracle.forward(oracle.params(pi, A, B), sym, offsets, lengths)
    ok = np.array([True, True, True, True, True, False, False])
    T = np.maximum(lengths[ok], 1)[:, None]
    assert np.all(np.abs(ll[ok] - ref[ok]) <= 3 * U_BF16 * T + ll_tol(lengths[ok])[:, None])
    assert np.abs(ll[5, 0] - ref[5, 0]) <= 3 * U_BF16 * lengths[5] + ll_tol(lengths[5:6])[0]
