"""The synthetic generators plant what they state (CPU, through the oracle's
Step 6 rows): every planted row rises strictly along the plant's recorded
column order, the shapes are the paper's benchmark shapes, and seeds differ."""
import numpy as np
import pytest

import oracle
from paper_1801_03039_gb300 import synth


@pytest.mark.parametrize("size", sorted(synth.PATTERN_SIZES))
@pytest.mark.parametrize("pattern", synth.PATTERNS)
def test_pattern_plants_follow_their_order(pattern, size):
    prob = synth.matrix_pattern(3, pattern, size)
    R, C, n, w = synth.PATTERN_SIZES[size]
    assert prob.A.shape == (R, C) and len(prob.plants) == n
    seen_rows, seen_cols = set(), set()
    for pl in prob.plants:
        assert len(pl.rows) == w and pl.kind == pattern
        assert not (seen_rows & set(pl.rows.tolist()))             # disjoint plants
        seen_rows |= set(pl.rows.tolist())
        if pattern == "row-constant":
            assert len(pl.order) == 0
            continue
        assert len(pl.order) == w and not (seen_cols & set(pl.order.tolist()))
        seen_cols |= set(pl.order.tolist())
        rising = set(oracle.rows(prob.A, pl.order.tolist(), 0).tolist())
        assert set(pl.rows.tolist()) <= rising


def test_row_constant_rows_have_no_column_order():
    prob = synth.matrix_pattern(1, "row-constant", "150x100")
    for pl in prob.plants:
        block = prob.A[np.ix_(pl.rows, pl.cols)]
        assert len(pl.cols) == 15 and np.all(block == block[:, :1])   # flat rows
        # ties: no planted row rises or falls along any of its columns
        got = set(oracle.rows(prob.A, pl.cols[:3].tolist(), 1).tolist())
        assert not (got & set(pl.rows.tolist()))


@pytest.mark.parametrize("width", [10, 20, 30])
def test_narrow_plants(width):
    prob = synth.matrix_narrow(2, width)
    assert prob.A.shape == (1000, 100) and len(prob.plants) == 3
    for pl in prob.plants:
        assert len(pl.rows) == 100 and len(pl.order) == width
        assert set(pl.rows.tolist()) <= set(oracle.rows(prob.A, pl.order.tolist(), 0).tolist())


def test_noise_is_added_and_seeds_differ():
    a = synth.matrix_pattern(0, "shift", "200x150")
    b = synth.matrix_pattern(0, "shift", "200x150", noise=0.25)
    c = synth.matrix_pattern(1, "shift", "200x150")
    d = b.A - a.A
    assert 0.2 < float(np.std(d)) < 0.3 and abs(float(np.mean(d))) < 0.01
    assert not np.array_equal(a.A, c.A)
    # with noise the plants are only approximately ordered
    pl = b.plants[0]
    assert len(oracle.rows(b.A, pl.order.tolist(), 0)) < len(pl.rows)


@pytest.mark.parametrize("overlap", [0, 3, 6, 9])
def test_overlap_plants(overlap):
    """Three 20 x 20 plants in 200 x 150, each sharing exactly `overlap` rows
    and columns with the next and none with the one after; the last plant is
    not overwritten, so all its rows rise along its order, and an earlier
    plant keeps its order on the columns no later plant touches."""
    prob = synth.matrix_overlap(4, overlap, noise=0.0)
    assert prob.A.shape == (200, 150) and len(prob.plants) == 3
    rs = [set(pl.rows.tolist()) for pl in prob.plants]
    cs = [set(pl.order.tolist()) for pl in prob.plants]
    assert all(len(r) == 20 for r in rs) and all(len(c) == 20 for c in cs)
    for a, b in ((0, 1), (1, 2)):
        assert len(rs[a] & rs[b]) == overlap and len(cs[a] & cs[b]) == overlap
    assert not (rs[0] & rs[2]) and not (cs[0] & cs[2])
    last = prob.plants[2]
    assert rs[2] <= set(oracle.rows(prob.A, last.order.tolist(), 0).tolist())
    first = prob.plants[0]
    free = [c for c in first.order.tolist() if c not in cs[1]]
    assert rs[0] <= set(oracle.rows(prob.A, free, 0).tolist())
