"""Step 6 rows, Step 7's expansions by negative and by approximate trends and
Eq. (2)-(3) on the GPU against the oracle (exact), and a recovery /
relevance check of whole EBIC runs on planted biclusters."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    eb.build()
    yield


def _cbf(seqs):
    return oracle.to_cbf(seqs)


def test_rows_hand(golden_dir):
    d = json.load(open(os.path.join(golden_dir, "support_hand_5x4.json")))
    A = np.array([[float(v) for v in row] for row in d["matrix"]], np.float32)
    cases = json.load(open(os.path.join(golden_dir, "rows_hand_5x4.json")))["cases"]
    h = eb.ebic_load_matrix(A)
    try:
        off, cols = _cbf([c["series"] for c in cases])
        for mode, key in ((eb.ROWS_RISING, "rows"), (eb.ROWS_RISING_OR_FALLING, "rows_neg")):
            got = eb.ebic_extract_rows(h, off, cols, mode)
            assert [g.tolist() for g in got] == [c[key] for c in cases]
    finally:
        eb.ebic_free(h)


@pytest.mark.parametrize("shape", [(37, 6), (1000, 30), (4099, 64), (20000, 200)])
def test_rows_match_oracle(shape):
    R, C = shape
    rng = np.random.default_rng(R)
    if R < 100:
        A = rng.integers(-2, 3, (R, C)).astype(np.float32)
        A[rng.random(A.shape) < 0.05] = np.nan
        seqs = [rng.choice(C, int(rng.integers(1, 5)), replace=False).tolist() for _ in range(60)]
        seqs.append([1, 1])
    else:
        prob = synth.matrix_random(R, R, C, n_plants=3, plant_rows=(R // 20, R // 8),
                                   plant_cols=(3, 10))
        A = prob.A
        off, cols = synth.population(R, 120, C, 1, 12, plants=prob.plants)
        seqs = [cols[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    off, cols = _cbf(seqs)
    h = eb.ebic_load_matrix(A)
    try:
        for mode in (eb.ROWS_RISING, eb.ROWS_RISING_OR_FALLING):
            got = eb.ebic_extract_rows(h, off, cols, mode)
            for s, g in zip(seqs, got):
                want = oracle.rows(A, s, mode)
                assert g.tolist() == want.tolist(), (s, mode)
        # the counts agree with Step 4's support
        inc, dec, _ = eb.ebic_eval_population(h, off, cols, 10, 1, want_dec=True)
        got = eb.ebic_extract_rows(h, off, cols, eb.ROWS_RISING)
        assert [len(g) for g in got] == inc.tolist()
    finally:
        eb.ebic_free(h)


@pytest.mark.parametrize("shape", [(37, 6), (1000, 30), (4099, 64)])
def test_approximate_rows_match_oracle(shape):
    """Step 7 by approximate trends (at most e broken adjacent pairs per row)
    against the oracle, both modes, e = 0 included (the rows of Step 6)."""
    R, C = shape
    rng = np.random.default_rng(R + 1)
    if R < 100:
        A = rng.integers(-2, 3, (R, C)).astype(np.float32)
        A[rng.random(A.shape) < 0.05] = np.nan
        seqs = [rng.choice(C, int(rng.integers(1, 6)), replace=False).tolist() for _ in range(60)]
    else:
        prob = synth.matrix_random(R, R, C, n_plants=3, plant_rows=(R // 20, R // 8),
                                   plant_cols=(3, 10))
        A = prob.A
        off, cols = synth.population(R, 80, C, 1, 12, plants=prob.plants)
        seqs = [cols[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    off, cols = _cbf(seqs)
    h = eb.ebic_load_matrix(A)
    try:
        for mode in (eb.ROWS_RISING, eb.ROWS_RISING_OR_FALLING):
            exact = eb.ebic_extract_rows(h, off, cols, mode)
            for e in (0, 1, 2, 5):
                got = eb.ebic_extract_rows_approx(h, off, cols, e, mode)
                for s, g in zip(seqs, got):
                    assert g.tolist() == oracle.rows_approx(A, s, e, mode).tolist(), (s, e, mode)
                if e == 0:
                    assert [g.tolist() for g in got] == [x.tolist() for x in exact]
        for bad in (-1, 1025):
            with pytest.raises(eb.EbicError):
                eb.ebic_extract_rows_approx(h, off, cols, bad)
    finally:
        eb.ebic_free(h)


def test_rows_capacity_and_arguments():
    A = np.random.default_rng(0).standard_normal((300, 8)).astype(np.float32)
    h = eb.ebic_load_matrix(A)
    try:
        import ctypes
        off, cols = _cbf([[0], [1, 2]])
        roff = np.zeros(3, np.int64)
        cap = ctypes.c_int64(10)
        rows = np.zeros(10, np.int32)
        st = eb.lib().ebic_extract_rows(h, off.ctypes.data_as(ctypes.c_void_p),
                                        cols.ctypes.data_as(ctypes.c_void_p), 2, 0,
                                        roff.ctypes.data_as(ctypes.c_void_p),
                                        rows.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cap))
        assert st == 1 and cap.value == 300 + len(oracle.rows(A, [1, 2], 0))
        assert not roff.any() and not rows.any()          # nothing written
        with pytest.raises(eb.EbicError):
            eb.ebic_extract_rows(h, *_cbf([[0, 8]]))       # column out of range
        with pytest.raises(eb.EbicError):
            eb.ebic_extract_rows(h, *_cbf([[0, 1]]), mode=3)
    finally:
        eb.ebic_free(h)


def _random_biclusters(rng, n, R, C):
    out = []
    for _ in range(n):
        r = np.sort(rng.choice(R, int(rng.integers(1, 40)), replace=False))
        c = np.sort(rng.choice(C, int(rng.integers(1, 8)), replace=False))
        out.append((r, c))
    return out


def test_recovery_relevance_matches_oracle():
    rng = np.random.default_rng(1)
    for E, F in [(1, 1), (3, 7), (10, 100), (5, 2)]:
        ex = _random_biclusters(rng, E, 60, 12)
        fo = _random_biclusters(rng, F, 60, 12) + [ex[0]]
        rec, rel, J = eb.ebic_recovery_relevance(ex, fo, want_jaccard=True)
        orec, orel = oracle.recovery_relevance(ex, fo)
        assert rec == pytest.approx(orec, rel=1e-12, abs=1e-15)
        assert rel == pytest.approx(orel, rel=1e-12, abs=1e-15)
        assert J[0, -1] == 1.0
    assert eb.ebic_recovery_relevance([], [(np.arange(3), np.arange(2))]) == (0.0, 0.0)
    with pytest.raises(eb.EbicError):
        eb.ebic_recovery_relevance([(np.array([2, 1]), np.array([0]))],
                                   [(np.array([1]), np.array([0]))])


def _ebic_biclusters(h, prob, gens, P, Lmax, sigma, seed, k_out, mode):
    p = eb.ebic_default_params(pop_size=P, len_min=3, len_max=Lmax, iterations=gens, sigma=sigma,
                               toprank_size=100, tournament_k=2, seed=seed)
    top, fit, st = eb.ebic_run_generations(h, p)
    top = top[:k_out]
    rows = eb.ebic_extract_rows(h, *_cbf(top), mode)
    return [(r, np.sort(np.asarray(t))) for r, t in zip(rows, top)], top


@pytest.mark.parametrize("case", [
    dict(name="narrow 1000x100, 3 x (50 x 10)", make=lambda: synth.matrix_paper(seed=0),
         gens=10000, P=600, Lmax=20, sigma=25, floor=0.8),
    dict(name="overlap 200x150, 3 x (20 x 20), 0x0", make=lambda: synth.matrix_overlap(0, 0),
         gens=10000, P=600, Lmax=24, sigma=10, floor=0.6),
    dict(name="overlap 200x150, 3 x (20 x 20), 6x6", make=lambda: synth.matrix_overlap(0, 6),
         gens=10000, P=600, Lmax=24, sigma=10, floor=0.45),
])
def test_whole_runs_recover_planted_biclusters(case):
    """Quality of the whole method, scored as in the paper (Eq. (2)-(3)): EBIC
    on seeded matrices with planted order-preserving biclusters, then Step 6
    and Step 7's negative-trend expansion on as many best top-rank series as
    there are plants."""
    prob = case["make"]()
    expected = [(np.sort(pl.rows), np.sort(pl.order)) for pl in prob.plants]
    h = eb.ebic_load_matrix(prob.A)
    try:
        found, top = _ebic_biclusters(h, prob, case["gens"], case["P"], case["Lmax"],
                                      case["sigma"], 0, len(expected), eb.ROWS_RISING_OR_FALLING)
        rec, rel = eb.ebic_recovery_relevance(expected, found)
        orec, orel = oracle.recovery_relevance(
            expected, [(oracle.rows(prob.A, t, 1), np.sort(t)) for t in top])
        assert rec == pytest.approx(orec, rel=1e-12) and rel == pytest.approx(orel, rel=1e-12)
        print(f"{case['name']}: recovery {rec:.3f} relevance {rel:.3f}")
        assert rec > case["floor"] and rel > case["floor"]
    finally:
        eb.ebic_free(h)
