"""Pins of the oracle's offspring screening (make_child with oversample V > 1;
not in the paper): properties fixed by its stated definition, checked on
single attempts through or_screen_attempt --

* candidate 0 is the plain child (the V = 1 draws), and candidate v does not
  depend on V (each candidate has its own draws 2k+1+5v .. 2k+5+5v);
* the pseudo score of candidate v is word 0 of Philox-4x32-10 at counter
  (j, g, 65536 + c V + v, 0), key = seed, shifted right by 8, computed here
  from the known-answer-pinned Philox binding and the traced outcome c;
* the pick: candidates by decreasing score (ties: lower v), the first one
  not in the tabu list as it stood at the generation's start, else the best;
* every candidate is a valid series (distinct columns below C, length in
  [Lmin, Lmax]) and the outcome c lies in [0, k^2), with tb = 0 without
  crossover."""
import numpy as np
import pytest

import oracle


def _population(seed, P=40, C=24, Lmin=2, Lmax=7):
    rng = np.random.default_rng(seed)
    seqs = [rng.choice(C, int(rng.integers(Lmin, Lmax + 1)), replace=False).tolist()
            for _ in range(P)]
    f = rng.random(P) * 3.0
    pen = rng.integers(0, 6, C).astype(np.int64)
    return seqs, f, pen


KW = dict(pop_size=40, len_min=2, len_max=7, tournament_k=2, p_crossover=0.5,
          penalty_base=1.2, seed=11)


def _order(scores):
    return sorted(range(len(scores)), key=lambda v: (-scores[v], v))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_candidate_zero_is_the_plain_child_and_candidates_do_not_depend_on_v(k):
    seqs, f, pen = _population(k)
    kw = dict(KW, tournament_k=k)
    for g, j in [(1, 0), (2, 7), (5, 123), (9, 1000)]:
        plain = oracle.screen_attempt(24, g, j, seqs, f, pen, **kw, oversample=1)
        r4 = oracle.screen_attempt(24, g, j, seqs, f, pen, **kw, oversample=4)
        r8 = oracle.screen_attempt(24, g, j, seqs, f, pen, **kw, oversample=8)
        assert plain["child"] == plain["cands"][0] == r4["cands"][0] == r8["cands"][0]
        assert r8["cands"][:4] == r4["cands"]
        assert plain["outcome"] == r4["outcome"] == r8["outcome"]


@pytest.mark.parametrize("V", [2, 5, 8])
def test_scores_follow_the_philox_counter_layout(V):
    seqs, f, pen = _population(V)
    seed = KW["seed"]
    for g, j in [(1, 3), (4, 77), (12, 601)]:
        r = oracle.screen_attempt(24, g, j, seqs, f, pen, **KW, oversample=V)
        c = r["outcome"]
        for v in range(V):
            w = oracle.philox4x32_10([j, g, 65536 + c * V + v, 0], [seed & 0xffffffff, seed >> 32])
            assert r["scores"][v] == int(w[0]) >> 8
            assert r["scores"][v] < 1 << 24


def test_pick_rule_against_the_tabu_list_at_generation_start():
    seqs, f, pen = _population(5)
    V = 6
    checked = 0
    for j in range(60):
        r = oracle.screen_attempt(24, 3, j, seqs, f, pen, **KW, oversample=V)
        cands, order = r["cands"], _order(r["scores"])
        distinct = {tuple(x) for x in cands}
        # empty list: the best-scoring candidate
        assert r["child"] == cands[order[0]]
        if len(distinct) < 3:
            continue
        # the best one listed: the best of the others that is not listed
        top = cands[order[0]]
        r2 = oracle.screen_attempt(24, 3, j, seqs, f, pen, [top], **KW, oversample=V)
        want = next(cands[v] for v in order if cands[v] != top)
        assert r2["child"] == want
        # every candidate listed: the best-scoring one (a hit)
        r3 = oracle.screen_attempt(24, 3, j, seqs, f, pen, [list(x) for x in distinct], **KW,
                                   oversample=V)
        assert r3["child"] == top
        checked += 1
    assert checked > 30


@pytest.mark.parametrize("pc", [0.0, 1.0])
def test_candidates_are_valid_series_and_outcomes_in_range(pc):
    seqs, f, pen = _population(9)
    k = 3
    kw = dict(KW, tournament_k=k, p_crossover=pc)
    for j in range(40):
        r = oracle.screen_attempt(24, 2, j, seqs, f, pen, **kw, oversample=5)
        assert 0 <= r["outcome"] < k * k
        if pc == 0.0:
            assert r["outcome"] % k == 0          # no second tournament: tb = 0
        for x in r["cands"]:
            assert 2 <= len(x) <= 7 and len(set(x)) == len(x) and all(0 <= c < 24 for c in x)
