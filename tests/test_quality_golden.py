"""The stored quality-suite figures on the CPU: each five-dataset file agrees
with its single-dataset file on dataset 0, the means are the means of the
cases, the 20,000-generation files (the paper's run length) cover the same
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
ONE_20K = _load("quality_suite_20000gens.json")
FIVE_20K = _load("quality_suite_5datasets_20000gens.json")


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


def test_the_longer_runs_cover_the_same_cases():
    assert ONE_20K["generations"] == 20000 and ONE_20K.get("datasets", 1) == 1
    assert FIVE_20K["generations"] == 20000 and FIVE_20K["datasets"] == 5
    assert [c["problem"] for c in ONE_20K["cases"]] == [c["problem"] for c in ONE["cases"]]
    for c in ONE_20K["cases"] + FIVE_20K["cases"]:
        assert c["params"]["iterations"] == 20000
        assert c["generations_done"] == 20000 or c["stop_reason"] != 0
    zero = [c for c in FIVE_20K["cases"] if c["dataset"] == 0]
    for a, b in zip(ONE_20K["cases"], zero):
        for k in ("problem", "noise", "params", "recovery", "relevance", "approximate_trends"):
            assert a[k] == b[k], (a["problem"], k)


@pytest.mark.parametrize("gold", [FIVE, FIVE_20K], ids=["10000", "20000"])
def test_means_are_the_means_of_the_cases(gold):
    assert len(gold["cases"]) == len(mqs.cases(5))
    groups = {}
    for c in gold["cases"]:
        groups.setdefault(_key(c), []).append(c)
    assert set(groups) == set(gold["means"])
    for k, cs in groups.items():
        assert len(cs) == 5 and sorted(c["dataset"] for c in cs) == list(range(5))
        for q in ("recovery", "relevance"):
            assert gold["means"][k][q] == pytest.approx(sum(c[q] for c in cs) / 5, rel=1e-12)
        for e, pair in gold["means"][k]["approximate_trends"].items():
            for j in (0, 1):
                want = sum(c["approximate_trends"][e][j] for c in cs) / 5
                assert pair[j] == pytest.approx(want, rel=1e-12), (k, e)


def test_scores_are_fractions():
    for c in FIVE["cases"] + FIVE_20K["cases"]:
        for rec, rel in [(c["recovery"], c["relevance"]), *c["approximate_trends"].values()]:
            assert 0.0 <= rec <= 1.0 and 0.0 <= rel <= 1.0


@pytest.mark.parametrize("gold,dataset", [(FIVE, 0), (FIVE, 3), (FIVE_20K, 4)])
def test_cases_name_today_s_problems_and_parameters(gold, dataset):
    """The stored problem names and parameters are what the generator and the
    script produce now, so a change to either shows up here first."""
    stored = [c for c in gold["cases"] if c["dataset"] == dataset]
    for case in stored:
        prob = mqs.problem(case)
        assert prob.name == case["problem"]
        assert mqs.params(case, prob, gold["generations"]) == case["params"]
