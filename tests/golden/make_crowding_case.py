"""Writes tests/golden/crowding_steps23.json: one generation of Steps 2-3 on a
small matrix, attempt by attempt, with the crowding penalty counts that each
tournament sees.

Paper: "EBIC Algorithm", Step 2 (the best quarter of the top-rank list is
copied into the new population), Step 3 (tournaments on the previous
population, crossover and mutation, tabu check, until the population is full;
sequential) and the crowding paragraph (a column's use by an individual added
to the new population, elites included, raises the penalty that later
tournaments of the same generation apply: f' = f / 1.2^theta, theta = the mean
use count over the series' columns).

The bookkeeping is restated here on its own, from that text:
  * pen[c] starts at 0 for the generation;
  * every elite adds 1 to each of its columns;
  * every accepted child adds 1 to each of its columns, before the next
    attempt;
  * an attempt whose child is already in the tabu list (a hit) adds nothing.
Each attempt's child comes from the oracle's single-attempt entry point
(``oracle.screen_attempt``, one candidate), given the penalty counts of the
restatement; the whole generation from ``oracle.run``.  The script keeps the
first seed for which the three plausible mistakes -- counting hits, leaving
the elites out, adding the children's uses only once the generation is full --
each change the generation's population, and records for each the first
attempt where its penalty counts change the outcome.

Run from the repository root:  python tests/golden/make_crowding_case.py
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "crowding_steps23.json")
R, C = 12, 4
PARAMS = dict(pop_size=6, len_min=2, len_max=3, iterations=1, sigma=2, toprank_size=6,
              tournament_k=2, overlap_tau=0.5, elite_frac=0.25, penalty_base=1.2,
              p_crossover=0.5, fitness_support=0, oversample=1)
VARIANTS = ("paper", "count_hits", "skip_elites", "once_per_generation")


def matrix(seed: int) -> np.ndarray:
    """Values on a coarse grid (multiples of 1/8 in [-2, 2)), exact in fp32 and
    with ties, so that series differ in support by small amounts."""
    rng = np.random.default_rng(seed)
    return (rng.integers(-16, 16, (R, C)) / 8.0).astype(np.float32)


def steps23(variant, seqs0, f0, elites, seed):
    """Steps 2-3 of generation 1 under one bookkeeping rule.  Returns the new
    population and the attempt log."""
    P = PARAMS["pop_size"]
    pen = [0] * C                 # counts the tournaments see
    deferred = [0] * C            # once_per_generation: uses held back
    nxt = [list(e) for e in elites]
    if variant != "skip_elites":
        for e in elites:
            for c in e:
                pen[c] += 1
    tabu = {tuple(s) for s in seqs0}
    log = []
    j = 0
    while len(nxt) < P:
        r = oracle.screen_attempt(C, 1, j, seqs0, f0, np.array(pen, np.int64), **PARAMS,
                                  seed=seed)
        child = r["child"]
        hit = tuple(child) in tabu
        log.append({"attempt": j, "pen_before": list(pen), "outcome": r["outcome"],
                    "child": child, "hit": hit})
        if hit:
            if variant == "count_hits":
                for c in child:
                    pen[c] += 1
        else:
            tabu.add(tuple(child))
            nxt.append(child)
            for c in child:
                if variant == "once_per_generation":
                    deferred[c] += 1
                else:
                    pen[c] += 1
        j += 1
        if j > 4 * P:
            return None, log
    return nxt, log


def first_difference(log_ok, log_bad):
    for a, b in zip(log_ok, log_bad):
        if a["outcome"] != b["outcome"] or a["child"] != b["child"]:
            return {"attempt": a["attempt"], "pen_before": b["pen_before"],
                    "outcome": b["outcome"], "child": b["child"]}
    return None


def find_case():
    for seed in range(1, 20000):
        A = matrix(seed)
        run = oracle.run(A, trace=True, **PARAMS, seed=seed)
        if run["stats"]["generations_done"] != 1:
            continue
        pop0, top0 = run["trace_pop"][0], run["trace_top"][0]
        seqs0, f0 = pop0["seqs"], pop0["f"]
        if len(set(np.round(f0, 12))) < len(f0) - 1:
            continue                                   # want distinct fitness values
        n_elite = math.ceil(PARAMS["elite_frac"] * len(top0["seqs"]))
        elites = top0["seqs"][:n_elite]
        res = {v: steps23(v, seqs0, f0, elites, seed) for v in VARIANTS}
        ok, log = res["paper"]
        if ok is None or ok != run["trace_pop"][1]["seqs"]:
            continue
        hits_before_accept = any(e["hit"] for e in log[:-1])
        if not hits_before_accept:
            continue
        wit = {}
        for v in VARIANTS[1:]:
            bad, blog = res[v]
            if bad is None or bad == ok:
                break
            d = first_difference(log, blog)
            if d is None:
                break
            wit[v] = d
        else:
            return seed, A, run, elites, log, ok, wit
    raise SystemExit("no case found")


def main():
    seed, A, run, elites, log, ok, wit = find_case()
    pop0 = run["trace_pop"][0]
    doc = {
        "citation": "arXiv 1801.03039, 'EBIC Algorithm' Steps 2-3 and the crowding paragraph: "
                    "elites (best quarter of the top-rank list) and every child added to the "
                    "new population raise the use counts of their columns; a tabu hit adds "
                    "nothing; every tournament sees the counts left by all earlier additions "
                    "of the same generation; f' = f / 1.2^(sum of counts / L).",
        "written_by": "tests/golden/make_crowding_case.py (calls only oracle/)",
        "seed": seed, "params": PARAMS, "rows": R, "cols": C,
        "A": [[float(x) for x in row] for row in A],
        "generation0": {"seqs": pop0["seqs"], "f": [float(x) for x in pop0["f"]],
                        "toprank": run["trace_top"][0]["seqs"]},
        "elites": elites,
        "pen_after_elites": log[0]["pen_before"],
        "attempts": log,
        "generation1": ok,
        "mistakes": wit,
    }
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=1)
        fh.write("\n")
    print(f"seed {seed}: {len(log)} attempts, {sum(e['hit'] for e in log)} hits; "
          f"witnesses {{{', '.join(f'{k}: attempt {v['attempt']}' for k, v in wit.items())}}}")


if __name__ == "__main__":
    main()
