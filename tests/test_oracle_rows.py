"""Pins for the oracle's Step 6 rows, Step 7 negative-trend expansion and the
recovery / relevance scores of Eq. (2)-(3)."""
import json
import os

import numpy as np
import pytest

import oracle


def _hand_matrix(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "support_hand_5x4.json")))
    return np.array([[float(v) for v in row] for row in d["matrix"]], np.float32)


def test_rows_hand(golden_dir):
    A = _hand_matrix(golden_dir)
    cases = json.load(open(os.path.join(golden_dir, "rows_hand_5x4.json")))["cases"]
    for c in cases:
        assert oracle.rows(A, c["series"], 0).tolist() == c["rows"], c
        assert oracle.rows(A, c["series"], 1).tolist() == c["rows_neg"], c


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rows_count_is_support_and_rows_are_the_definition(seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-3, 4, (60, 7)).astype(np.float32)
    A[rng.random(A.shape) < 0.05] = np.nan
    for _ in range(40):
        L = int(rng.integers(1, 6))
        s = rng.choice(7, L, replace=False)
        off = np.array([0, L], np.int32)
        inc, dec = oracle.support(A, off, s.astype(np.int32))
        r0, r1 = oracle.rows(A, s, 0), oracle.rows(A, s, 1)
        assert len(r0) == inc[0]
        assert len(r1) == (inc[0] if L == 1 else inc[0] + dec[0])
        # brute force on the definition, row by row (numpy comparisons)
        sub = A[:, s]
        rising = np.all(sub[:, :-1] < sub[:, 1:], axis=1)
        falling = np.all(sub[:, :-1] > sub[:, 1:], axis=1)
        assert r0.tolist() == np.flatnonzero(rising).tolist()
        assert r1.tolist() == np.flatnonzero(rising | falling).tolist()


def test_reversal_swaps_rising_and_falling_rows():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 9)).astype(np.float32)
    s = [3, 1, 7, 0]
    fall = np.setdiff1d(oracle.rows(A, s, 1), oracle.rows(A, s, 0))
    assert oracle.rows(A, s[::-1], 0).tolist() == fall.tolist()


def test_recovery_relevance_hand():
    e1 = (range(0, 10), range(0, 4))           # 40 cells
    e2 = (range(20, 30), range(5, 9))          # 40 cells
    # identical sets
    assert oracle.recovery_relevance([e1], [e1]) == (1.0, 1.0)
    # disjoint
    assert oracle.recovery_relevance([e1], [e2]) == (0.0, 0.0)
    # half the rows: |e & f| = 5 x 4 = 20, |e | f| = 40 + 20 - 20 = 40 -> 0.5
    f = (range(0, 5), range(0, 4))
    assert oracle.recovery_relevance([e1], [f]) == (0.5, 0.5)
    # one found bicluster matching e1 exactly, one expected missing:
    # recovery = (1 + 0) / 2, relevance = 1 / 1
    assert oracle.recovery_relevance([e1, e2], [e1]) == (0.5, 1.0)
    # a spurious extra found: relevance = (1 + 0) / 2
    assert oracle.recovery_relevance([e1], [e1, e2]) == (1.0, 0.5)
    # rows and columns both partial: |e & f| = 5 x 2 = 10, |e | f| = 40 + 30 - 10 = 60
    g = (range(5, 15), range(2, 5))
    rec, rel = oracle.recovery_relevance([e1], [g])
    assert rec == pytest.approx(10 / 60) and rel == pytest.approx(10 / 60)
    assert oracle.recovery_relevance([], [e1]) == (0.0, 0.0)


# ---------------------------------------------------------------------------
# Step 7 by approximate trends (reading: at most e adjacent pairs of a row may
# break the order).  Over the L! orderings of L columns, the rows with exactly
# v pairs out of order (descents) number the Eulerian number A(L, v).
def _eulerian(n):
    a = [1]                                   # A(1, 0) = 1
    for m in range(2, n + 1):                 # A(m, k) = (k+1) A(m-1, k) + (m-k) A(m-1, k-1)
        a = [(k + 1) * (a[k] if k < len(a) else 0) + (m - k) * (a[k - 1] if k >= 1 else 0)
             for k in range(m)]
    return a


def _all_orderings(L):
    import itertools
    return np.array(list(itertools.permutations(range(L))), np.float32)


def test_eulerian_numbers_are_the_textbook_ones():
    assert _eulerian(4) == [1, 11, 11, 1]
    assert _eulerian(5) == [1, 26, 66, 26, 1]
    assert sum(_eulerian(6)) == 720


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6])
def test_approximate_rows_count_by_descents(L):
    A = _all_orderings(L)
    seq = list(range(L))
    eul = _eulerian(L)
    for e in range(L):
        rising = oracle.rows_approx(A, seq, e, 0)
        assert len(rising) == sum(eul[:e + 1])
        # rising or falling: at most e descents or at most e ascents
        want = sum(eul[v] for v in range(L) if v <= e or (L - 1 - v) <= e)
        assert len(oracle.rows_approx(A, seq, e, 1)) == want


def test_approximate_rows_reduce_to_step6_and_nest():
    rng = np.random.default_rng(3)
    A = rng.integers(-2, 3, (300, 9)).astype(np.float32)     # many ties
    A[rng.random(A.shape) < 0.03] = np.nan
    for _ in range(40):
        seq = rng.choice(9, int(rng.integers(1, 7)), replace=False).tolist()
        for mode in (0, 1):
            prev = oracle.rows_approx(A, seq, 0, mode)
            assert prev.tolist() == oracle.rows(A, seq, mode).tolist()
            for e in range(1, len(seq)):
                cur = oracle.rows_approx(A, seq, e, mode)
                assert set(prev.tolist()) <= set(cur.tolist())
                assert np.all(np.diff(cur) > 0)
                prev = cur
            # every pair may break: every row
            assert len(oracle.rows_approx(A, seq, max(len(seq) - 1, 0), mode)) == 300


def test_approximate_rows_ties_and_nan_break_both_directions():
    A = np.array([[1.0, 1.0, 1.0],          # ties: no pair rises or falls
                  [1.0, np.nan, 3.0],       # NaN: no pair compares
                  [1.0, 2.0, 3.0],          # rising
                  [3.0, 2.0, 1.0],          # falling
                  [1.0, 3.0, 2.0]], np.float32)
    seq = [0, 1, 2]
    assert oracle.rows_approx(A, seq, 0, 1).tolist() == [2, 3]
    assert oracle.rows_approx(A, seq, 1, 0).tolist() == [2, 4]
    assert oracle.rows_approx(A, seq, 1, 1).tolist() == [2, 3, 4]
    assert oracle.rows_approx(A, seq, 2, 0).tolist() == [0, 1, 2, 3, 4]
