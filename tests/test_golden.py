"""Stored fixtures for the likelihood (tests/golden/loglik_golden.json,
written by tests/golden/make_golden.py from the definition and the oracle).

* "exact": every observation is "no tremor", every number a dyadic rational,
  so L of Eq. "likelihood func" is a rational number, evaluated exactly when
  the file was written; the oracle's scaled forward recursion, backward
  recursion and brute force must reproduce log L to rounding, for both
  places the initial vector can enter. (The first case, K = 2 and T = 3, is
  small enough to check by hand: L = 2265/8192 emit-first and 18969/65536
  with the printed transition-first form.)
* "bruteforce": tiny seeded inputs with tremors; the stored value is the
  oracle's sum over all K^T paths, which the forward recursion must match
  and the brute force must still reproduce.
"""
import json
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle

GOLDEN = json.loads((Path(__file__).parent / "golden" / "loglik_golden.json").read_text())
MODES = (("emit_first", 0), ("transition_first", 1))


def _params(rec):
    f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return (f(rec["pi"]), f(rec["P"]), f(rec["p"]), f(rec["mu"]), f(rec["cov"]))


@pytest.mark.parametrize("i", range(len(GOLDEN["exact"])))
def test_exact_rational_cases(i):
    rec = GOLDEN["exact"][i]
    prm = _params(rec)
    T = rec["T"]
    xy = np.zeros((T, 2), np.float32)
    fl = np.zeros(T, np.uint8)
    for name, mode in MODES:
        L = Fraction(rec[name]["L"])
        want = math.log(L.numerator) - math.log(L.denominator)
        assert want == rec[name]["log_L"]
        for fn in (oracle.loglik, oracle.loglik_backward, oracle.loglik_longdouble, oracle.loglik_bruteforce):
            got = fn(prm, xy, fl, mode)
            assert abs(got - want) <= 1e-14 * abs(want) + 1e-15, (fn.__name__, name, got, want)


def test_hand_checked_case():
    rec = GOLDEN["exact"][0]
    assert rec["T"] == 3 and rec["emit_first"]["L"] == "2265/8192"
    assert rec["transition_first"]["L"] == "18969/65536"


@pytest.mark.parametrize("i", range(len(GOLDEN["bruteforce"])))
def test_bruteforce_cases(i):
    rec = GOLDEN["bruteforce"][i]
    prm = _params(rec)
    xy = np.ascontiguousarray(np.asarray(rec["xy"], np.float32).reshape(-1, 2))
    fl = np.ascontiguousarray(np.asarray(rec["tremor"], np.uint8))
    for name, mode in MODES:
        want = rec[name]["log_L"]
        assert abs(oracle.loglik_bruteforce(prm, xy, fl, mode) - want) <= 1e-15 * abs(want)
        for fn in (oracle.loglik, oracle.loglik_backward, oracle.loglik_longdouble):
            got = fn(prm, xy, fl, mode)
            assert abs(got - want) <= 1e-13 * abs(want), (fn.__name__, name, got, want)
