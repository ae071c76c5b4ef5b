"""Exhaustive enumeration over all N^T hidden-state paths (pure Python).

TEST INFRASTRUCTURE ONLY (pins the FP64 oracle on tiny inputs; never used by
the product path).

For a discrete HMM lambda = (pi, A, B) the joint probability of a state path
Q = q_1..q_T and symbols O = o_1..o_T is
    P(O, Q) = pi_{q_1} b_{q_1}(o_1) prod_{t>1} a_{q_{t-1} q_t} b_{q_t}(o_t)
(Rabiner 1989, eqs. 13-15). Everything here is that product summed, maximised
or weighted over every path -- no recursion -- so it checks the forward,
Viterbi and expected-count recursions by a route that shares nothing with
them. Probabilities may be floats or ``fractions.Fraction`` (exact ties).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction


def joint(pi, A, B, obs, path):
    """P(O, Q) as a product, in the number type of the parameters."""
    if len(obs) == 0:
        return 1
    p = pi[path[0]] * B[path[0]][obs[0]]
    for t in range(1, len(obs)):
        p = p * A[path[t - 1]][path[t]] * B[path[t]][obs[t]]
    return p


def all_paths(N, T):
    return itertools.product(range(N), repeat=T)


def likelihood(pi, A, B, obs):
    """P(O) = sum over all N^T paths of P(O, Q)."""
    N = len(pi)
    return sum(joint(pi, A, B, obs, q) for q in all_paths(N, len(obs)))


def best_path(pi, A, B, obs):
    """(max_Q P(O,Q), Q*, second-largest P(O,Q) over the other paths).

    Among equal maxima the path chosen is the one a smallest-index Viterbi
    backtrack returns: the smallest q_T, then the smallest q_{T-1}, ..., i.e.
    the minimum under lexicographic order of the reversed path.
    """
    N, T = len(pi), len(obs)
    if T == 0:
        return 1, (), 0
    scored = [(joint(pi, A, B, obs, q), q) for q in all_paths(N, T)]
    best = max(v for v, _ in scored)
    winners = [q for v, q in scored if v == best]
    q_star = min(winners, key=lambda q: tuple(reversed(q)))
    vals = sorted((v for v, _ in scored), reverse=True)
    second = vals[1] if len(vals) > 1 else 0
    return best, q_star, second


def expected_counts(pi, A, B, obs):
    """E[n_pi(i)], E[n_ij], E[n_j(k)] under P(Q | O), by enumeration.

    n_pi(i) = [q_1 = i]; n_ij = #{t : q_t = i, q_{t+1} = j};
    n_j(k) = #{t : q_t = j, o_t = k}.
    """
    N, M, T = len(pi), len(B[0]), len(obs)
    cpi = [0.0] * N
    cA = [[0.0] * N for _ in range(N)]
    cB = [[0.0] * M for _ in range(N)]
    Z = 0.0
    for q in all_paths(N, T):
        w = float(joint(pi, A, B, obs, q))
        if w == 0.0:
            continue
        Z += w
        cpi[q[0]] += w
        for t in range(T - 1):
            cA[q[t]][q[t + 1]] += w
        for t in range(T):
            cB[q[t]][obs[t]] += w
    if Z == 0.0:
        return cpi, cA, cB, -math.inf
    cpi = [x / Z for x in cpi]
    cA = [[x / Z for x in row] for row in cA]
    cB = [[x / Z for x in row] for row in cB]
    return cpi, cA, cB, math.log(Z)


def to_fraction_rows(rows, denom):
    """Helper for exact fixtures: integer numerators over a common denominator."""
    return [[Fraction(x, denom) for x in r] for r in rows]
