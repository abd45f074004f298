"""Pins for the oracle's support count (section "Motivation") and CBF (Fig. 3).

Each test checks the oracle against something other than itself: hand-worked
values, an independent sort-based characterisation, a closed form over all
L-tuples, invariants of strict order, planted rows, and the R/L! expectation.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1801_03039_gb300 import synth


def _support_of(A, seqs):
    off, cols = oracle.to_cbf(seqs)
    return oracle.support(A, off, cols)


def test_hand_worked_5x4(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "support_hand_5x4.json")))
    A = np.array([[float(v) for v in row] for row in g["matrix"]], dtype=np.float32)
    assert np.signbit(A[4, 0]) and not np.signbit(A[4, 1])
    inc, dec = _support_of(A, [c["series"] for c in g["cases"]])
    for i, c in enumerate(g["cases"]):
        assert (inc[i], dec[i]) == (c["inc"], c["dec"]), c


def test_cbf_fig3_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "cbf_fig3.json")))
    offsets = np.array(g["starts"] + [len(g["cols"])], np.int32)
    cols = np.array(g["cols"], np.int32)
    series = [cols[offsets[i]:offsets[i + 1]].tolist() for i in range(len(g["starts"]))]
    assert series == g["series"]
    A = np.random.default_rng(3).standard_normal((64, 6)).astype(np.float32)
    inc, dec = oracle.support(A, offsets, cols)
    for i, s in enumerate(g["series"]):
        one_inc, one_dec = _support_of(A, [s])
        assert (inc[i], dec[i]) == (one_inc[0], one_dec[0])


def _sort_based(row, s):
    """Independent definition: the values along s, once sorted, keep their order
    and are pairwise distinct (no NaN)."""
    v = row[list(s)]
    if len(s) == 1:
        return True
    if np.isnan(v).any():
        return False
    if len(set(v.tolist())) != len(v):
        return False
    return bool(np.array_equal(np.argsort(v, kind="stable"), np.arange(len(v))))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    R, C = 8, 5
    A = rng.integers(-2, 3, (R, C)).astype(np.float32)   # many ties
    A[rng.random((R, C)) < 0.08] = np.nan
    A[rng.random((R, C)) < 0.1] = -0.0
    seqs = [s for L in range(1, 5) for s in itertools.product(range(C), repeat=L)]
    inc, dec = _support_of(A, seqs)
    for i, s in enumerate(seqs):
        e_inc = sum(_sort_based(A[k], s) for k in range(R))
        e_dec = sum(_sort_based(-A[k], s) for k in range(R))
        assert inc[i] == e_inc and dec[i] == e_dec, (s, inc[i], e_inc, dec[i], e_dec)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_closed_form_sum_over_tuples(L):
    # Rows of distinct values: each L-subset of columns has exactly one rising
    # order, so summing inc over all ordered L-tuples gives R * C(C, L).
    rng = np.random.default_rng(L)
    R, C = 7, 6
    A = np.stack([rng.permutation(C) for _ in range(R)]).astype(np.float32) * 0.5 - 1.0
    seqs = list(itertools.permutations(range(C), L))
    inc, dec = _support_of(A, seqs)
    assert int(inc.sum()) == R * math.comb(C, L)
    assert int(dec.sum()) == R * math.comb(C, L)


def test_reversal_swaps_inc_and_dec():
    rng = np.random.default_rng(5)
    A = rng.integers(-3, 4, (300, 12)).astype(np.float32)
    A[rng.random(A.shape) < 0.02] = np.nan
    seqs = [rng.choice(12, int(rng.integers(1, 7)), replace=False).tolist() for _ in range(200)]
    inc, dec = _support_of(A, seqs)
    rinc, rdec = _support_of(A, [s[::-1] for s in seqs])
    assert np.array_equal(inc, rdec) and np.array_equal(dec, rinc)


def test_pair_complement_without_ties():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((500, 10)).astype(np.float32)
    pairs = [(p, q) for p in range(10) for q in range(10) if p != q]
    inc, _ = _support_of(A, pairs)
    d = {pq: int(v) for pq, v in zip(pairs, inc)}
    for p, q in pairs:
        assert d[(p, q)] + d[(q, p)] == 500


def test_planted_rows_always_count():
    prob = synth.matrix_tiny(seed=7, noise=0.0)
    rng = np.random.default_rng(8)
    for pl in prob.plants:
        for _ in range(30):
            L = int(rng.integers(2, len(pl.order) + 1))
            s = pl.order[np.sort(rng.choice(len(pl.order), L, replace=False))].tolist()
            inc, dec = _support_of(prob.A, [s, s[::-1]])
            rows_ok = [k for k in pl.rows if _sort_based(prob.A[k], s)]
            assert len(rows_ok) == len(pl.rows)
            assert inc[0] >= len(pl.rows) and dec[1] >= len(pl.rows)


def test_monotone_in_subsequences():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((400, 15)).astype(np.float32)
    for _ in range(50):
        s = rng.choice(15, int(rng.integers(2, 8)), replace=False).tolist()
        subs = [s[:-1], s[1:], [c for i, c in enumerate(s) if i != len(s) // 2]]
        inc, _ = _support_of(A, [s] + subs)
        assert all(inc[i] >= inc[0] for i in range(1, 4))


@pytest.mark.parametrize("L", [2, 3, 4])
def test_iid_expectation_R_over_L_factorial(L):
    # For iid continuous rows a fixed series is rising with probability 1/L!.
    rng = np.random.default_rng(10 + L)
    R, C, n = 2000, 30, 400
    A = rng.standard_normal((R, C)).astype(np.float32)
    seqs = [rng.choice(C, L, replace=False).tolist() for _ in range(n)]
    inc, _ = _support_of(A, seqs)
    p = 1.0 / math.factorial(L)
    mean, sd = R * p, math.sqrt(R * p * (1 - p) / n)
    assert abs(inc.mean() - mean) < 5 * sd


def test_threads_give_identical_counts():
    prob = synth.matrix_paper(seed=1)
    off, cols = synth.population(2, 300, 100, 3, 20, plants=prob.plants)
    a = oracle.support(prob.A, off, cols, nthreads=1)
    b = oracle.support(prob.A, off, cols, nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
