"""Whole EBIC searches on the seeded benchmark shapes (the paper's pattern
suite, narrow and overlapping biclusters, a noise sweep) on the GPU: the search, the rows of
the found biclusters with the negative-trend expansion (and with the
approximate-trend expansion) and Eq. (2)-(3) give the recovery and relevance
the oracle gives (tests/golden/quality_suite.json, written by
make_quality_suite.py from the oracle only)."""
import json
import os

import numpy as np
import pytest

import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "quality_suite.json")))


@pytest.fixture(scope="module", autouse=True)
def built():
    eb.build()
    yield


def _problem(case):
    seed = case.get("dataset", 0)
    if case["suite"] == "narrow":
        return synth.matrix_narrow(seed, case["width"], case["noise"])
    if case["suite"] == "overlap":
        return synth.matrix_overlap(seed, case["overlap"], case["noise"])
    return synth.matrix_pattern(seed, case["pattern"], case["size"], case["noise"])


def _name(case):
    return case["problem"] + (f"-noise{case['noise']}" if case["noise"] else "")


@pytest.mark.parametrize("case", GOLD["cases"], ids=_name)
def test_search_quality_matches_the_oracle(case):
    prob = _problem(case)
    assert prob.name == case["problem"]
    expected = [(np.sort(pl.rows), np.sort(pl.cols if pl.cols is not None else pl.order))
                for pl in prob.plants]
    h = eb.ebic_load_matrix(prob.A)
    try:
        top, fit, st = eb.ebic_run_generations(h, eb.ebic_default_params(**case["params"]))
        top = top[:len(expected)]
        off = np.cumsum([0] + [len(t) for t in top]).astype(np.int32)
        flat = np.concatenate([np.asarray(t, np.int32) for t in top])
        rows = eb.ebic_extract_rows(h, off, flat, eb.ROWS_RISING_OR_FALLING)
        found = [(r, np.sort(np.asarray(t))) for r, t in zip(rows, top)]
        rec, rel = eb.ebic_recovery_relevance(expected, found)
        approx = {}
        for e in case["approximate_trends"]:
            rows_e = eb.ebic_extract_rows_approx(h, off, flat, int(e), eb.ROWS_RISING_OR_FALLING)
            approx[e] = eb.ebic_recovery_relevance(
                expected, [(r, np.sort(np.asarray(t))) for r, t in zip(rows_e, top)])
    finally:
        eb.ebic_free(h)
    assert st["generations_done"] == case["generations_done"]
    assert st["stop_reason"] == case["stop_reason"]
    assert rec == pytest.approx(case["recovery"], rel=1e-12, abs=1e-15)
    assert rel == pytest.approx(case["relevance"], rel=1e-12, abs=1e-15)
    for e, (arec, arel) in case["approximate_trends"].items():
        assert approx[e][0] == pytest.approx(arec, rel=1e-12, abs=1e-15), e
        assert approx[e][1] == pytest.approx(arel, rel=1e-12, abs=1e-15), e
