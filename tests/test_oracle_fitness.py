"""Pins for the oracle's Eq. (1) and crowding penalty.

Values are checked against exact high-precision evaluation (mpmath, 60
digits) of the formula's hand-derived closed forms, not against a retyped
double-precision formula.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 60


def _ulps(a: float, exact) -> float:
    if exact == 0:
        return 0.0 if a == 0 else math.inf
    return abs(mpmath.mpf(a) - exact) / mpmath.mpf(math.ulp(float(exact)))


def _eval_hand(expr: str):
    env = {"ln": mpmath.log}
    return mpmath.mpf(eval(expr.replace("^", "**"), {"__builtins__": {}}, env)) \
        if expr != "0" else mpmath.mpf(0)


def test_hand_values(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fitness_eq1_hand.json")))
    for c in g["cases"]:
        f = oracle.fitness(c["n"], c["J"], c["sigma"])
        exact = _eval_hand(c["f"])
        if exact == 0:
            assert f == 0.0, c
        else:
            assert _ulps(f, exact) <= 2.0, (c, f, exact)  # log (<=1 ulp) then one rounded product


def test_power_of_two_factor_is_exact():
    # 2^min(n - sigma, 0) is a power of two, so for n < sigma the value is the
    # n >= sigma value scaled exactly.
    for n in range(2, 60):
        for sigma in range(n, n + 40):
            for J in (1, 3, 17):
                full = oracle.fitness(n, J, n)
                assert oracle.fitness(n, J, sigma) == math.ldexp(full, n - sigma)


def test_random_values_within_two_ulp():
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = int(rng.integers(2, 60000))
        J = int(rng.integers(1, 65))
        sigma = int(rng.integers(1, 2000))
        exact = mpmath.ldexp(mpmath.log(n - 1), min(n - sigma, 0)) * J
        assert _ulps(oracle.fitness(n, J, sigma), exact) <= 2.0


def test_underflow_goes_to_zero_monotonically():
    vals = [oracle.fitness(10, 5, 10 + d) for d in range(1000, 1200)]
    assert vals[-1] == 0.0
    assert all(a >= b for a, b in zip(vals, vals[1:]))


def test_more_columns_more_fitness_when_rows_kept():
    # The design of Eq. (1) rewards longer series at equal support.
    for n in (30, 100, 1000):
        assert oracle.fitness(n, 6, 25) > oracle.fitness(n, 5, 25)


def test_penalty_division_reading():
    for f, S, L in [(5.0, 0, 3), (5.0, 3, 3), (7.25, 17, 4), (1.0, 1000, 7)]:
        exact = mpmath.mpf(f) / mpmath.power(mpmath.mpf(1.2), mpmath.mpf(S) / L)
        # pow and the quotient theta = S/L each round once: a few ulps at most.
        assert _ulps(oracle.penalized(f, S, L, 1.2), exact) <= 4.0 + 0.2 * S / L


def test_tournament_hand_cases():
    seqs = [[0, 1], [2, 3], [0, 2], [4, 5]]
    C = 6
    pen = np.zeros(C, np.int64)
    # No penalty: the fittest entrant wins.
    assert oracle.tournament([0, 1], seqs, [1.0, 2.0, 0, 0], pen, 1.2) == 1
    # Equal fitness: the lower population index wins, whatever the draw order.
    assert oracle.tournament([3, 1], seqs, [0, 2.0, 0, 2.0], pen, 1.2) == 1
    # 2.4 / 1.2^1 == 2.0 exactly (2.4 is exactly twice 1.2 in binary64):
    # a tie with an unpenalised 2.0, so the lower index wins.
    pen[2] = pen[3] = 1            # series 1 = (2, 3): theta = (1 + 1) / 2 = 1
    assert oracle.tournament([1, 0], seqs, [2.0, 2.4, 0, 0], pen, 1.2) == 0
    # A heavier penalty makes the fitter series lose.
    pen[2] = pen[3] = 3            # theta = 3: 2.4 / 1.728 < 2.0
    assert oracle.tournament([1, 0], seqs, [2.0, 2.4, 0, 0], pen, 1.2) == 0
    assert oracle.tournament([1, 3], seqs, [0, 2.4, 0, 1.3], pen, 1.2) == 1
    pen[2] = pen[3] = 4            # 2.4 / 1.2^4 = 1.157 < 1.3
    assert oracle.tournament([1, 3], seqs, [0, 2.4, 0, 1.3], pen, 1.2) == 3
