"""Writes tests/golden/tiny_exact.json: exact rational values of P(O),
max_Q P(O,Q), the maximising path and the second-best path probability for
two small discrete HMMs with rational parameters.

Every value is the plain definition P(O,Q) = pi_{q1} b_{q1}(o1) prod a b
(Rabiner 1989, eqs. 13-15) summed or maximised over all N^T paths in exact
``fractions.Fraction`` arithmetic by ``oracle.bruteforce``; nothing else is
called. Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
from fractions import Fraction as F

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import bruteforce  # noqa: E402

CASES = [
    dict(name="two_state_three_symbol",
         pi=[F(3, 5), F(2, 5)],
         A=[[F(7, 10), F(3, 10)], [F(2, 5), F(3, 5)]],
         B=[[F(1, 2), F(2, 5), F(1, 10)], [F(1, 10), F(3, 10), F(3, 5)]],
         obs=[0, 1, 2, 2, 1, 0]),
    dict(name="three_state_left_right",
         pi=[F(1), F(0), F(0)],
         A=[[F(1, 2), F(1, 2), F(0)], [F(0), F(2, 3), F(1, 3)], [F(0), F(0), F(1)]],
         B=[[F(3, 4), F(1, 4)], [F(1, 3), F(2, 3)], [F(1, 5), F(4, 5)]],
         obs=[0, 0, 1, 1, 0, 1, 1]),
]


def fr(x):
    x = F(x)
    return f"{x.numerator}/{x.denominator}"


def main():
    out = {"source": "exact enumeration of P(O,Q) over all paths (Rabiner 1989 eqs. 13-15)",
           "cases": []}
    for c in CASES:
        p = bruteforce.likelihood(c["pi"], c["A"], c["B"], c["obs"])
        best, path, second = bruteforce.best_path(c["pi"], c["A"], c["B"], c["obs"])
        out["cases"].append(dict(
            name=c["name"],
            pi=[fr(x) for x in c["pi"]],
            A=[[fr(x) for x in r] for r in c["A"]],
            B=[[fr(x) for x in r] for r in c["B"]],
            obs=c["obs"], P=fr(p), P_best=fr(best), path=list(path), P_second=fr(second)))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_exact.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=None, separators=(",", ": "))
        f.write("\n")


if __name__ == "__main__":
    main()
