"""Writes tests/golden/loglik_golden.json (run from the repository root:
``python tests/golden/make_golden.py``).

Two kinds of fixtures, both for the likelihood of Eq. "likelihood func"
(Section 2) with the emissions of Eq. "emission-matrix":

* "exact": inputs whose numbers are dyadic rationals and whose observations
  are all "no tremor", so every emission is the constant 1 - p_k and the
  likelihood is a finite sum of products of dyadic rationals. L is evaluated
  here in exact rational arithmetic (fractions.Fraction), straight from the
  matrix-product definition, for both places the initial vector can enter
  (pi^T D_1 P D_2 ... and the printed pi^T P D_1 P D_2 ...); the file stores
  L as a fraction and log L as a float.
* "bruteforce": small seeded inputs with tremors (K = 3, T <= 7), with the
  stored value from the oracle's sum over all K^T hidden paths.

Only the seeded input generator and oracle/ are used; nothing here touches
the CUDA library.
"""
from __future__ import annotations

import json
import math
import sys
from fractions import Fraction
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2003_03508_gb300 import synth  # noqa: E402


def exact_L(pi, P, q, T, transition_first):
    """pi^T [P] D P D ... P D 1 with D = diag(q) (all steps "no tremor"), exactly."""
    K = len(pi)
    v = [Fraction(x) for x in pi]
    if transition_first:
        v = [sum(v[i] * Fraction(P[i][j]) for i in range(K)) for j in range(K)]
    for t in range(T):
        if t > 0:
            v = [sum(v[i] * Fraction(P[i][j]) for i in range(K)) for j in range(K)]
        v = [v[k] * Fraction(q[k]) for k in range(K)]
    return sum(v)


EXACT_CASES = [
    # K = 2, hand-checkable: P rows (7/8, 1/8), (1/4, 3/4); p = (1/4, 1/2)
    dict(pi=[0.5, 0.5], P=[[0.875, 0.125], [0.25, 0.75]], p=[0.25, 0.5], T=3),
    dict(pi=[0.5, 0.5], P=[[0.875, 0.125], [0.25, 0.75]], p=[0.25, 0.5], T=1),
    # K = 3, a reducible-looking but connected chain
    dict(pi=[0.25, 0.5, 0.25], P=[[0.5, 0.25, 0.25], [0.125, 0.75, 0.125], [0.0, 0.0625, 0.9375]],
         p=[0.125, 0.375, 0.0625], T=6),
    # K = 1: L = (1 - p)^T
    dict(pi=[1.0], P=[[1.0]], p=[0.5], T=5),
]


def main():
    out = {"citation": "Eq. \"likelihood func\" and Eq. \"emission-matrix\" (Section 2); "
                       "exact cases: rational evaluation of the matrix product; brute-force cases: "
                       "the oracle's sum over all K^T hidden paths",
           "exact": [], "bruteforce": []}
    for c in EXACT_CASES:
        K = len(c["pi"])
        q = [1.0 - x for x in c["p"]]
        rec = dict(c)
        for mode, name in ((0, "emit_first"), (1, "transition_first")):
            L = exact_L(c["pi"], c["P"], q, c["T"], mode == 1)
            rec[name] = {"L": f"{L.numerator}/{L.denominator}", "log_L": math.log(L.numerator) - math.log(L.denominator)}
        # dummy locations: ignored where no tremor is flagged
        rec["mu"] = [[100.0 + 10 * k, 50.0] for k in range(K)]
        rec["cov"] = [[100.0, 0.0, 100.0] for _ in range(K)]
        out["exact"].append(rec)
    for seed, T in ((11, 1), (12, 4), (13, 7)):
        rng = np.random.default_rng(seed)
        prm = synth.random_params(3, rng, diag=(0.3, 0.8))
        obs = synth.sample_observations(prm, T, rng)
        rec = {"seed": seed, "K": 3, "T": T,
               "pi": prm.pi.astype(float).tolist(), "P": prm.P.astype(float).tolist(),
               "p": prm.p_tremor.astype(float).tolist(), "mu": prm.mu.astype(float).tolist(),
               "cov": prm.cov.astype(float).tolist(), "xy": obs.xy.astype(float).tolist(),
               "tremor": obs.tremor.astype(int).tolist()}
        for mode, name in ((0, "emit_first"), (1, "transition_first")):
            rec[name] = {"log_L": oracle.loglik_bruteforce(prm, obs.xy, obs.tremor, mode)}
        out["bruteforce"].append(rec)
    path = Path(__file__).with_name("loglik_golden.json")
    path.write_text(json.dumps(out, indent=1) + "\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
