"""Pin of the oracle's crowding bookkeeping in Steps 2-3 ("EBIC Algorithm",
Steps 2-3, and the crowding paragraph of arXiv 1801.03039).

The stored case (tests/golden/crowding_steps23.json) lists one generation
attempt by attempt: the use counts pen[c] after the elites and before every
attempt, the tournament outcome and child of every attempt, and whether the
child was a tabu hit.  The counts follow the paper's rule, restated on its own
in the script that wrote the file: elites count, every accepted child counts
before the next attempt, hits do not count, counts restart each generation.
The file also holds, for three plausible mistakes in that rule, the first
attempt whose outcome they change."""
import json
import os

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def case(golden_dir):
    return json.load(open(os.path.join(golden_dir, "crowding_steps23.json")))


def _kw(case):
    kw = dict(case["params"])
    kw["seed"] = case["seed"]
    return kw


def test_counts_follow_the_rule(case):
    """The stored counts obey the paper's rule on their own: after the elites
    they are the elites' column uses, and each attempt adds its child's columns
    exactly when the child was accepted."""
    C = case["cols"]
    pen = [0] * C
    for e in case["elites"]:
        for c in e:
            pen[c] += 1
    assert pen == case["pen_after_elites"]
    added = []
    for a in case["attempts"]:
        assert a["pen_before"] == pen, a["attempt"]
        if not a["hit"]:
            for c in a["child"]:
                pen[c] += 1
            added.append(a["child"])
    assert case["elites"] + added == case["generation1"]
    # the case exercises what the rule is about
    assert any(a["hit"] for a in case["attempts"])
    assert any(x > 0 for x in case["pen_after_elites"])


def test_each_attempt_sees_the_stored_counts(case):
    """The oracle's single attempt, given the stored counts, gives the stored
    outcome and child (the tournament applies f / 1.2^(S/L) with these S)."""
    g0 = case["generation0"]
    for a in case["attempts"]:
        r = oracle.screen_attempt(case["cols"], 1, a["attempt"], g0["seqs"], g0["f"],
                                  np.array(a["pen_before"], np.int64), **_kw(case))
        assert r["outcome"] == a["outcome"], a["attempt"]
        assert r["child"] == a["child"], a["attempt"]


def test_whole_generation_matches(case):
    """oracle.run's own bookkeeping gives generation 0 and, after Steps 2-3,
    exactly the stored generation 1."""
    A = np.array(case["A"], np.float32)
    out = oracle.run(A, trace=True, **_kw(case))
    assert out["stats"]["generations_done"] == 1
    assert out["trace_pop"][0]["seqs"] == case["generation0"]["seqs"]
    np.testing.assert_array_equal(out["trace_pop"][0]["f"], case["generation0"]["f"])
    assert out["trace_top"][0]["seqs"] == case["generation0"]["toprank"]
    assert out["trace_pop"][1]["seqs"] == case["generation1"]
    assert out["stats"]["last_gen_hits"] == sum(a["hit"] for a in case["attempts"])


@pytest.mark.parametrize("mistake", ["count_hits", "skip_elites", "once_per_generation"])
def test_mistakes_would_be_caught(case, mistake):
    """Each plausible mistake changes an attempt's outcome, so an oracle that
    made it would fail test_whole_generation_matches: its counts at the stored
    witness attempt, rebuilt here from the stored log, give a different child."""
    C = case["cols"]
    w = case["mistakes"][mistake]
    pen = [0] * C
    if mistake != "skip_elites":
        for e in case["elites"]:
            for c in e:
                pen[c] += 1
    for a in case["attempts"]:
        if a["attempt"] == w["attempt"]:
            break
        if a["hit"] and mistake == "count_hits":
            for c in a["child"]:
                pen[c] += 1
        if not a["hit"] and mistake != "once_per_generation":
            for c in a["child"]:
                pen[c] += 1
    assert pen == w["pen_before"]
    g0 = case["generation0"]
    r = oracle.screen_attempt(C, 1, w["attempt"], g0["seqs"], g0["f"],
                              np.array(pen, np.int64), **_kw(case))
    right = case["attempts"][w["attempt"]]
    assert (r["outcome"], r["child"]) == (w["outcome"], w["child"])
    assert (r["outcome"], r["child"]) != (right["outcome"], right["child"])
