"""The stored quality-suite figures on the CPU: the five-dataset file agrees
with the single-dataset file on dataset 0, its means are the means of its
cases, and every stored case names the seeded problem and the search
parameters that make_quality_suite.py derives for it today."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(__file__)
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_quality_suite as mqs  # noqa: E402


def _load(name):
    return json.load(open(os.path.join(HERE, "golden", name)))


ONE = _load("quality_suite.json")
FIVE = _load("quality_suite_5datasets.json")


def _key(c):
    return c["problem"] + (f" noise {c['noise']}" if c["noise"] else "")


def test_the_files_cover_every_case_and_dataset():
    assert ONE.get("datasets", 1) == 1 and FIVE["datasets"] == 5
    assert ONE["generations"] == FIVE["generations"] == 10000
    assert len(ONE["cases"]) == len(mqs.cases(1))
    assert len(FIVE["cases"]) == len(mqs.cases(5))
    assert sorted(c["dataset"] for c in FIVE["cases"]) == sorted(
        d for d in range(5) for _ in mqs._cases())


def test_dataset_zero_is_the_single_dataset_file():
    zero = [c for c in FIVE["cases"] if c["dataset"] == 0]
    assert len(zero) == len(ONE["cases"])
    for a, b in zip(ONE["cases"], zero):
        for k in ("problem", "noise", "params", "generations_done", "stop_reason", "recovery",
                  "relevance", "approximate_trends"):
            assert a[k] == b[k], (a["problem"], k)


def test_means_are_the_means_of_the_cases():
    groups = {}
    for c in FIVE["cases"]:
        groups.setdefault(_key(c), []).append(c)
    assert set(groups) == set(FIVE["means"])
    for k, cs in groups.items():
        assert len(cs) == 5 and sorted(c["dataset"] for c in cs) == list(range(5))
        for q in ("recovery", "relevance"):
            assert FIVE["means"][k][q] == pytest.approx(sum(c[q] for c in cs) / 5, rel=1e-12)


def test_scores_are_fractions_and_relevance_bounds_recovery_on_clean_data():
    for c in FIVE["cases"]:
        for rec, rel in [(c["recovery"], c["relevance"]), *c["approximate_trends"].values()]:
            assert 0.0 <= rec <= 1.0 and 0.0 <= rel <= 1.0


@pytest.mark.parametrize("dataset", [0, 3])
def test_cases_name_today_s_problems_and_parameters(dataset):
    """The stored problem names and parameters are what the generator and the
    script produce now, so a change to either shows up here first."""
    stored = [c for c in FIVE["cases"] if c["dataset"] == dataset]
    for case in stored:
        prob = mqs.problem(case)
        assert prob.name == case["problem"]
        assert mqs.params(case, prob, FIVE["generations"]) == case["params"]
