"""Seeded synthetic workloads for the HMM recognition hot path.

This module only draws random numbers: model parameters, activity labels,
sequence lengths and symbol sequences sampled from the models. It holds none
of the scoring, decoding or counting arithmetic, and it is the one module that
both the CUDA path's callers and the FP64 oracle's callers import, so the two
always see the same inputs.

The paper's own workload (the UCF teamwork recordings, Sec. 5.7) is not
available; these draws stand in for it with the shapes of its HMM stage
(Sec. 4.1: number of hidden states, symbols, actions) scaled to five
configurations:

  plain      K=1,  N=4,   M=8    Dirichlet(1) rows; 64 sequences of T=50
  batched    K=10, N=16,  M=32   Dirichlet(0.5) pi/B, self-transition U(0.6,0.9),
                                 off-diagonal (1-a_ii)*Dirichlet(0.5); 4096
                                 sequences, T ~ U{30..300}, label ~ U{0..9}
  gradient   K=10, N=32,  M=64   logits ~ N(0,1); 2048 sequences, T ~ U{50..500}
  large      K=4,  N=128, M=256  Dirichlet(0.3) rows; 16384 sequences,
                                 T ~ U{100..2000}
  training   K=20, N=64,  M=128  logits ~ N(0,0.5^2); 65536 sequences,
                                 P(T) ~ T^-1.5 on [50,1000] (inverse CDF, floor)
  cuhmm      K=1,  N=512, M=64   Dirichlet(0.3) rows; 512 sequences,
                                 T ~ U{100..500} (the 512-state x 512-sequence
                                 shape Sec. 5.6 quotes; M and T not stated)
  teamwork   4 roles x 6 actions = 24 models, N=5, M=64 (six binary features
                                 as one mixed-radix symbol); parameters as
                                 "batched"; 16384 sequences, T ~ U{20..120};
                                 label = role * 6 + action, role and action
                                 uniform (the application shape of Sec. 5.7)
  longseq    K=4,  N=32,  M=64   parameters as "batched"; 8 sequences,
                                 T ~ U{2^19..2^20} (few very long recordings)

Every sequence is sampled from the model of its label. Parameters are stored
as float32 (what the GPU computes with); the oracle reads the same float32
values widened to float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

SEEDS = {"plain": 1310001, "batched": 1310002, "gradient": 1310003, "large": 1310004,
         "training": 1310005, "teamwork": 1310006, "cuhmm": 1310007, "longseq": 1310008}

SPECS = {
    "plain": dict(K=1, N=4, M=8, S=64, lengths=("fixed", 50), params=("dirichlet", 1.0)),
    "batched": dict(K=10, N=16, M=32, S=4096, lengths=("uniform", 30, 300),
                    params=("sticky", 0.5, 0.6, 0.9)),
    "gradient": dict(K=10, N=32, M=64, S=2048, lengths=("uniform", 50, 500),
                     params=("logits", 1.0)),
    "large": dict(K=4, N=128, M=256, S=16384, lengths=("uniform", 100, 2000),
                  params=("dirichlet", 0.3)),
    "training": dict(K=20, N=64, M=128, S=65536, lengths=("powerlaw", 1.5, 50, 1000),
                     params=("logits", 0.5)),
    "cuhmm": dict(K=1, N=512, M=64, S=512, lengths=("uniform", 100, 500),
                  params=("dirichlet", 0.3)),
    "teamwork": dict(K=24, N=5, M=64, S=16384, lengths=("uniform", 20, 120),
                     params=("sticky", 0.5, 0.6, 0.9), roles=4),
    # few very long recordings: too few (sequence, model) pairs to fill the
    # GPU, the regime of the parallel-in-time forward
    "longseq": dict(K=4, N=32, M=64, S=8, lengths=("uniform", 1 << 19, 1 << 20),
                    params=("sticky", 0.5, 0.6, 0.9)),
}


@dataclass
class Workload:
    name: str
    K: int
    N: int
    M: int
    pi: np.ndarray          # [K,N] float32
    A: np.ndarray           # [K,N,N] float32, row = from-state
    B: np.ndarray           # [K,N,M] float32
    symbols: np.ndarray     # [total] int32
    offsets: np.ndarray     # [S] int64
    lengths: np.ndarray     # [S] int32
    labels: np.ndarray      # [S] int32, generating model
    seed: int
    logits: Optional[tuple] = None   # (pi, A, B) float32 logits for gradient configs
    meta: dict = field(default_factory=dict)

    @property
    def S(self) -> int:
        return int(self.lengths.shape[0])

    @property
    def total_obs(self) -> int:
        return int(self.symbols.shape[0])

    @property
    def max_len(self) -> int:
        return int(self.lengths.max()) if self.S else 0


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def _softmax64(x):
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(x - x.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def draw_params(spec: dict, seed: int):
    """Returns (pi, A, B float32 probabilities, logits or None)."""
    K, N, M = spec["K"], spec["N"], spec["M"]
    rng = _rng(seed, 0)
    kind = spec["params"][0]
    logits = None
    if kind == "dirichlet":
        a = spec["params"][1]
        pi = rng.dirichlet(np.full(N, a), size=K)
        A = rng.dirichlet(np.full(N, a), size=(K, N))
        B = rng.dirichlet(np.full(M, a), size=(K, N))
    elif kind == "sticky":
        a, lo, hi = spec["params"][1:]
        pi = rng.dirichlet(np.full(N, a), size=K)
        B = rng.dirichlet(np.full(M, a), size=(K, N))
        A = np.zeros((K, N, N))
        diag = rng.uniform(lo, hi, size=(K, N))
        off = rng.dirichlet(np.full(N - 1, a), size=(K, N)) if N > 1 else None
        for k in range(K):
            for i in range(N):
                A[k, i, i] = diag[k, i] if N > 1 else 1.0
                if N > 1:
                    others = [j for j in range(N) if j != i]
                    A[k, i, others] = (1.0 - diag[k, i]) * off[k, i]
    elif kind == "logits":
        sd = spec["params"][1]
        lpi = (rng.standard_normal((K, N)) * sd).astype(np.float32)
        lA = (rng.standard_normal((K, N, N)) * sd).astype(np.float32)
        lB = (rng.standard_normal((K, N, M)) * sd).astype(np.float32)
        logits = (lpi, lA, lB)
        pi, A, B = _softmax64(lpi), _softmax64(lA), _softmax64(lB)
    else:
        raise ValueError(kind)
    return (pi.astype(np.float32), A.astype(np.float32), B.astype(np.float32), logits)


def draw_lengths(spec: dict, S: int, seed: int, override=None) -> np.ndarray:
    rng = _rng(seed, 1)
    law = override if override is not None else spec["lengths"]
    if law[0] == "fixed":
        T = np.full(S, law[1], dtype=np.int64)
    elif law[0] == "uniform":
        T = rng.integers(law[1], law[2] + 1, size=S)
    elif law[0] == "powerlaw":
        alpha, lo, hi = law[1:]
        u = rng.random(S)
        e = 1.0 - alpha
        T = np.floor((lo ** e + u * (hi ** e - lo ** e)) ** (1.0 / e))
        T = np.clip(T, lo, hi)
    else:
        raise ValueError(law)
    return T.astype(np.int32)


class _RowSampler:
    """Inverse-CDF sampling of one column per row of a row-stochastic table."""

    def __init__(self, P: np.ndarray):
        P = np.asarray(P, dtype=np.float64)
        self.W = P.shape[-1]
        P = P.reshape(-1, self.W)
        cum = np.cumsum(P, axis=1)
        cum = cum / cum[:, -1:]
        cum[:, -1] = 1.0
        self.key = (cum + np.arange(P.shape[0])[:, None]).ravel()

    def __call__(self, rows: np.ndarray, u: np.ndarray) -> np.ndarray:
        pos = np.searchsorted(self.key, rows + u, side="right")
        col = pos - rows * self.W
        return np.minimum(col, self.W - 1)


def sample_sequences(pi, A, B, labels, lengths, rng) -> np.ndarray:
    """Draws O_s ~ lambda_{labels[s]} of length lengths[s], packed."""
    K, N = pi.shape
    S = labels.shape[0]
    offsets = np.zeros(S, np.int64)
    if S:
        offsets[1:] = np.cumsum(lengths.astype(np.int64))[:-1]
    total = int(lengths.astype(np.int64).sum())
    symbols = np.zeros(total, np.int32)
    if S == 0 or total == 0:
        return symbols
    s_pi, s_A, s_B = _RowSampler(pi), _RowSampler(A), _RowSampler(B)
    lab = labels.astype(np.int64)
    state = s_pi(lab, rng.random(S))
    Tmax = int(lengths.max())
    for t in range(Tmax):
        act = np.nonzero(lengths > t)[0]
        if act.size == 0:
            break
        st = state[act]
        symbols[offsets[act] + t] = s_B(lab[act] * N + st, rng.random(act.size))
        state[act] = s_A(lab[act] * N + st, rng.random(act.size))
    return symbols


def make_workload(name: str, n_seqs: Optional[int] = None, seed: Optional[int] = None,
                  lengths=None, K: Optional[int] = None, N: Optional[int] = None,
                  M: Optional[int] = None) -> Workload:
    """The named configuration, optionally with fewer sequences, another
    length law (e.g. ("uniform", 1, 40)) or other K/N/M for small parity
    cases; the parameter recipe stays that of the configuration."""
    spec = dict(SPECS[name])
    for key, v in (("K", K), ("N", N), ("M", M)):
        if v is not None:
            spec[key] = v
    seed = SEEDS[name] if seed is None else seed
    S = spec["S"] if n_seqs is None else n_seqs
    pi, A, B, logits = draw_params(spec, seed)
    Kk = spec["K"]
    T = draw_lengths(spec, S, seed, lengths)
    labels = _rng(seed, 1, 1).integers(0, Kk, size=S).astype(np.int32)
    symbols = sample_sequences(pi.astype(np.float64), A.astype(np.float64),
                               B.astype(np.float64), labels, T, _rng(seed, 2))
    offsets = np.zeros(S, np.int64)
    if S:
        offsets[1:] = np.cumsum(T.astype(np.int64))[:-1]
    return Workload(name=name, K=Kk, N=spec["N"], M=spec["M"], pi=pi, A=A, B=B,
                    symbols=symbols, offsets=offsets, lengths=T, labels=labels, seed=seed,
                    logits=logits, meta={"S": S, "lengths": lengths or spec["lengths"],
                                         "roles": spec.get("roles", 1)})


def resample(w: Workload, idx, round_: int) -> Workload:
    """Redraws the symbols of sequences ``idx`` (same lengths and labels) from
    the sub-stream (seed, 3, round_); used to regenerate sequences that fail a
    test's input filter."""
    idx = np.asarray(idx, dtype=np.int64)
    if idx.size == 0:
        return w
    sub = sample_sequences(w.pi.astype(np.float64), w.A.astype(np.float64),
                           w.B.astype(np.float64), w.labels[idx], w.lengths[idx],
                           _rng(w.seed, 3, round_))
    symbols = w.symbols.copy()
    pos = 0
    for s in idx:
        T = int(w.lengths[s])
        symbols[w.offsets[s]: w.offsets[s] + T] = sub[pos: pos + T]
        pos += T
    return replace(w, symbols=symbols)


def random_model(rng: np.random.Generator, K: int, N: int, M: int, alpha: float = 1.0):
    """K random models with Dirichlet(alpha) rows, float32 (small test cases)."""
    pi = rng.dirichlet(np.full(N, alpha), size=K).astype(np.float32)
    A = rng.dirichlet(np.full(N, alpha), size=(K, N)).astype(np.float32)
    B = rng.dirichlet(np.full(M, alpha), size=(K, N)).astype(np.float32)
    return pi, A, B


def random_sequences(rng: np.random.Generator, S: int, M: int, lo: int, hi: int):
    """Uniform random symbols with lengths U{lo..hi}, packed."""
    T = rng.integers(lo, hi + 1, size=S).astype(np.int32)
    offsets = np.zeros(S, np.int64)
    if S:
        offsets[1:] = np.cumsum(T.astype(np.int64))[:-1]
    symbols = rng.integers(0, M, size=int(T.astype(np.int64).sum())).astype(np.int32)
    return symbols, offsets, T


def role_split(w: Workload, roles: int):
    """Splits a workload whose K models are ``roles`` consecutive sets (one HMM
    set per role, Sec. 5.7) into one workload per role: that role's models,
    its sequences (own packed buffer) and labels relative to the set."""
    if w.K % roles:
        raise ValueError("K is not a multiple of the number of roles")
    Kr = w.K // roles
    out = []
    for r in range(roles):
        idx = np.nonzero(w.labels // Kr == r)[0]
        T = w.lengths[idx]
        off = np.zeros(idx.size, np.int64)
        if idx.size:
            off[1:] = np.cumsum(T.astype(np.int64))[:-1]
        sym = (np.concatenate([w.symbols[w.offsets[i]:w.offsets[i] + w.lengths[i]] for i in idx])
               if idx.size else np.zeros(0, np.int32)).astype(np.int32)
        sl = slice(r * Kr, (r + 1) * Kr)
        out.append(replace(w, name=f"{w.name}/role{r}", K=Kr, pi=w.pi[sl].copy(),
                           A=w.A[sl].copy(), B=w.B[sl].copy(), symbols=sym, offsets=off,
                           lengths=T.copy(), labels=(w.labels[idx] % Kr).astype(np.int32),
                           logits=None, meta={**w.meta, "role": r, "index": idx}))
    return out
