"""The algebra two GPU designs rest on, checked in FP64 numpy against the
oracle on small random models (CPU only; nothing here touches the library):

* parallel-in-time forward: the steps 1 .. T-1 cut into chunks of L steps,
  each chunk's product of step matrices A diag(b(o_t)) formed row by row
  from unit vectors with one power-of-two exponent per row, then combined in
  order against the largest term, give log P(O) (Rabiner eqs. 19-21);
* tensor-core adjoint in segment ranges: the forward rows kept with the
  one-step-late power-of-two exponents, the backward recursion
  Y_t = b(o_t) o (A Y_{t+1}) 2^-f_t c_t with c_{T-1} = w / sigma_{T-1},
  c_t = w / (c_{t+1} rho_{t+1}), run range by range, each range that ends
  before the sequence restarting from an arbitrarily scaled checkpoint of
  Y at its end rescaled by w / rho (rho = X_{t1-1} . A Y_{t1}) with c = 1,
  reproduces the expected counts (Rabiner eqs. 24-25, 37-38);
* adjoint above 128 states: Y_t = b(o_t) o beta_t obeys the forward
  recursion with A^T run backwards from Y_{T-1} = b(o_{T-1}), and with rows
  of arbitrary power-of-two scale, gamma_t = X_t o Bh_t / z_t and
  xi_t = (X_t / z_t) a_ij (b(o_{t+1}) o Bh_{t+1}) 2^-f_t with z_t = X_t . Bh_t
  reproduce the expected counts (Rabiner eqs. 24-25, 37-38).
"""
import numpy as np
import pytest

import oracle
from paper_1310_3322_gb300 import synth


def _case(seed, N, M, T):
    rng = np.random.default_rng(seed)
    pi, A, B = synth.random_model(rng, 1, N, M, alpha=0.6)
    obs = rng.integers(0, M, size=T).astype(np.int32)
    return pi[0].astype(np.float64), A[0].astype(np.float64), B[0].astype(np.float64), obs


def _oracle_loglik(pi, A, B, obs):
    P = oracle.params(pi[None], A[None], B[None])
    ll, _, _ = oracle.forward(P, obs, np.array([0], np.int64), np.array([obs.size], np.int32))
    return float(ll[0, 0])


def _split(v):
    """v = m 2^e with max |m| in [1, 2) (e for the whole vector)."""
    mx = np.max(np.abs(v))
    if mx == 0:
        return v, None
    e = int(np.floor(np.log2(mx)))
    return v * 2.0 ** -e, e


def _scan_loglik(pi, A, B, obs, L):
    T = obs.size
    v, Ev = _split(pi * B[:, obs[0]])
    chunks = [range(t0, min(T, t0 + L)) for t0 in range(1, T, L)]
    for ch in chunks:
        # chunk product, row i = the recursion started from e_i, own exponent
        rows, exps = [], []
        for i in range(pi.size):
            x, E = np.eye(pi.size)[i], 0
            for t in ch:
                x = (x @ A) * B[:, obs[t]]
                x, e = _split(x)
                if e is None:
                    break
                E += e
            rows.append(x)
            exps.append(None if e is None else E)
        # combine: weights against the largest term
        keys = [exps[i] + np.floor(np.log2(v[i])) if (v[i] > 0 and exps[i] is not None) else None
                for i in range(pi.size)]
        kmax = max(k for k in keys if k is not None)
        w = np.array([0.0 if keys[i] is None else v[i] * 2.0 ** (exps[i] - kmax)
                      for i in range(pi.size)])
        y = w @ np.array(rows)
        v, e = _split(y)
        Ev += kmax + e
    return float(np.log(v.sum()) + Ev * np.log(2.0))


@pytest.mark.parametrize("L", [1, 3, 7, 16, 100])
def test_chunked_step_products_give_the_forward(L):
    for seed in range(4):
        pi, A, B, obs = _case(seed, N=5, M=6, T=53)
        ref = _oracle_loglik(pi, A, B, obs)
        assert abs(_scan_loglik(pi, A, B, obs, L) - ref) <= 1e-9 * abs(ref)


def _backward_rows(A, B, obs):
    """Y_t by the forward recursion with A^T in reversed time, each row scaled
    by 2^-f_t (f_t from the previous row's sum, as the kernel does one step
    late); returns Bh_t = D_t 2^-f_t (before the emission) and f_t."""
    T, N = obs.size, A.shape[0]
    Bh = np.zeros((T, N))
    f = np.zeros(T, int)
    Bh[T - 1] = 1.0
    y = B[:, obs[T - 1]] * Bh[T - 1]
    for t in range(T - 2, -1, -1):
        D = y @ A.T                      # (A Y_{t+1})_i = sum_j a_ij Y_{t+1}(j)
        f[t] = int(np.floor(np.log2(y.sum())))
        Bh[t] = D * 2.0 ** -f[t]
        y = Bh[t] * B[:, obs[t]]
    return Bh, f


def test_backward_as_reversed_forward_with_transposed_matrix():
    pi, A, B, obs = _case(7, N=6, M=5, T=30)
    Bh, f = _backward_rows(A, B, obs)
    # the textbook beta, unscaled: beta_{T-1} = 1, beta_t = A (b(o_{t+1}) beta_{t+1})
    beta = np.ones((obs.size, pi.size))
    for t in range(obs.size - 2, -1, -1):
        beta[t] = A @ (B[:, obs[t + 1]] * beta[t + 1])
    # same direction at every t (scales differ only by the stored powers of two)
    for t in range(obs.size):
        r = Bh[t] / beta[t]
        assert np.allclose(r, r[0], rtol=1e-12)
    # the scale of Bh_t is 2^-(f_t + f_{t+1} + ... + f_{T-2})
    for t in range(obs.size - 1):
        assert np.isclose(Bh[t][0] / beta[t][0], 2.0 ** -f[t:obs.size - 1].sum(), rtol=1e-12)


def test_counts_from_arbitrarily_scaled_rows():
    pi, A, B, obs = _case(11, N=4, M=5, T=25)
    T, N, M = obs.size, pi.size, B.shape[1]
    # forward rows with arbitrary power-of-two scales
    rng = np.random.default_rng(3)
    X = np.zeros((T, N))
    x = pi * B[:, obs[0]]
    for t in range(T):
        if t > 0:
            x = (x @ A) * B[:, obs[t]]
        X[t] = x * 2.0 ** int(rng.integers(-20, 20))
    Bh, f = _backward_rows(A, B, obs)
    cpi = np.zeros(N)
    cA = np.zeros((N, N))
    cB = np.zeros((N, M))
    for t in range(T):
        z = X[t] @ Bh[t]
        g = X[t] * Bh[t] / z
        cB[:, obs[t]] += g
        if t == 0:
            cpi += g
        if t + 1 < T:
            V = B[:, obs[t + 1]] * Bh[t + 1] * 2.0 ** -f[t]
            cA += A * np.outer(X[t] / z, V)
    P = oracle.params(pi[None], A[None], B[None])
    _, rpi, rA, rB, _ = oracle.forward_backward(P, obs, np.array([0], np.int64),
                                                np.array([T], np.int32), None, None)
    np.testing.assert_allclose(cpi, rpi[0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(cA, rA[0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(cB, rB[0], rtol=1e-9, atol=1e-12)
    # the exponent must be the one removed when Bh_t was formed (f_t), not
    # Bh_{t+1}'s (f_{t+1}): the wrong index changes the transition counts
    assert np.any(f[:-2] != f[1:-1])
    wrong = np.zeros((N, N))
    for t in range(T - 1):
        z = X[t] @ Bh[t]
        wrong += A * np.outer(X[t] / z, B[:, obs[t + 1]] * Bh[t + 1] * 2.0 ** -f[t + 1])
    assert not np.allclose(wrong, rA[0], rtol=1e-3)


def _range_counts(pi, A, B, obs, w, cuts, restart=True, seed=0):
    """Counts by the segment-range recursion (ranges [cuts[r], cuts[r+1]) of
    the steps, processed independently, each from checkpoints only)."""
    T, N, M = obs.size, pi.size, B.shape[1]
    rng = np.random.default_rng(seed)
    # forward rows as the pass keeps them: X_t = (X_{t-1} A) o b(o_t) 2^-f_t,
    # f_t the exponent of the previous row sum (one step late)
    X = np.zeros((T, N))
    f = np.zeros(T, int)
    X[0] = pi * B[:, obs[0]]
    for t in range(1, T):
        f[t] = int(np.floor(np.log2(X[t - 1].sum())))
        X[t] = (X[t - 1] @ A) * B[:, obs[t]] * 2.0 ** -f[t]
    sigma = X[T - 1].sum()
    # backward operand checkpoints: Y_t = b(o_t) o beta_t at an arbitrary scale
    beta = np.ones((T, N))
    for t in range(T - 2, -1, -1):
        beta[t] = A @ (B[:, obs[t + 1]] * beta[t + 1])
    Yck = {t: B[:, obs[t]] * beta[t] * 2.0 ** int(rng.integers(-30, 30)) for t in cuts[1:-1]}
    cpi, cA, cB = np.zeros(N), np.zeros((N, N)), np.zeros((N, M))
    for lo, t1 in zip(cuts[:-1], cuts[1:]):
        c, rho_prev, Ynext = 0.0, 0.0, None
        if t1 < T:
            Ynext = Yck[t1]
            rho = X[t1 - 1] @ (A @ Ynext)
            if restart:
                Ynext = Ynext * (w / rho)
            c, rho_prev = 1.0, w
        for t in range(t1 - 1, lo - 1, -1):
            if t == T - 1:
                c, Bt = w / sigma, np.ones(N)
            else:
                c, Bt = w / (c * rho_prev), A @ Ynext
            G = X[t] * Bt * c
            rho_prev = X[t] @ Bt
            cB[:, obs[t]] += G
            if t == 0:
                cpi += G
            if t < T - 1:
                cA += A * np.outer(X[t], Ynext)
            Ynext = B[:, obs[t]] * Bt * 2.0 ** -f[t] * c
    return cpi, cA, cB


@pytest.mark.parametrize("ranges", [1, 2, 3, 5, 11])
def test_segment_ranges_restarted_from_scaled_checkpoints(ranges):
    pi, A, B, obs = _case(13 + ranges, N=5, M=6, T=44)
    T = obs.size
    cuts = [int(round(r * T / ranges)) for r in range(ranges + 1)]
    w = 1.7
    cpi, cA, cB = _range_counts(pi, A, B, obs, w, cuts)
    P = oracle.params(pi[None], A[None], B[None])
    _, rpi, rA, rB, _ = oracle.forward_backward(P, obs, np.array([0], np.int64),
                                                np.array([T], np.int32), None,
                                                np.array([w], np.float64))
    np.testing.assert_allclose(cpi, rpi[0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(cA, rA[0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(cB, rB[0], rtol=1e-9, atol=1e-12)
    if ranges > 1:
        # without the renormalisation the arbitrary checkpoint scale leaks
        # into the counts of every range but the last
        wpi, wA, wB = _range_counts(pi, A, B, obs, w, cuts, restart=False)
        assert not np.allclose(wB, rB[0], rtol=1e-3)
