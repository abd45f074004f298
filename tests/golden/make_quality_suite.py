"""Writes quality_suite.json: recovery and relevance (Eq. (2)-(3)) of whole
EBIC searches on the seeded synthetic benchmark shapes (the pattern suite,
the narrow biclusters, the overlapping biclusters and a noise sweep),
computed with the CPU oracle only -- the search (Steps 1-5), the rows of the found biclusters with the
negative-trend expansion (Steps 6-7) and the scores; also the scores with
the expansion by approximate trends (at most 1 or 2 broken adjacent pairs per
row) of the same found series.  The device path is
bit-identical to the oracle on these searches, so the stored figures are also
the device's.  Found biclusters: the best top-rank series, as many as there
are planted biclusters.

    python tests/golden/make_quality_suite.py [--generations 10000] [--jobs 16]
        [--datasets 1]

With --datasets n > 1 every case is run on datasets (generator seeds)
0 .. n-1 and quality_suite_<n>datasets.json gets the per-dataset figures
and their means (the paper averages five datasets per case).  Another
generation count than 10,000 adds _<g>gens to the file name (the paper's
synthetic runs stop after 20,000 generations or at the tabu-hit rule).
--resume keeps the cases already computed for the same generation count --
in the output file, in its checkpoint (<output>.partial, rewritten as cases
finish and removed at the end) or, for dataset 0, in the single-dataset
file; this script wrote them all and the oracle is deterministic -- and runs
only the missing ones.
"""
import argparse
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor, as_completed

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def cases(datasets=1):
    return [dict(c, dataset=d) for c in _cases() for d in range(datasets)]


def _cases():
    out = []
    for size in ("150x100", "200x150", "300x200"):
        for pattern in ("trend-preserving", "column-constant", "row-constant", "shift", "scale",
                        "shift-scale"):
            out.append({"suite": "pattern", "pattern": pattern, "size": size, "noise": 0.0})
    for width in (10, 20, 30):
        out.append({"suite": "narrow", "width": width, "noise": 0.0})
    for noise in (0.05, 0.1, 0.25):
        out.append({"suite": "pattern", "pattern": "trend-preserving", "size": "200x150",
                    "noise": noise})
    for overlap in (0, 3, 6, 9):
        out.append({"suite": "overlap", "overlap": overlap, "noise": 0.0})
    return out


def problem(case):
    from paper_1801_03039_gb300 import synth
    seed = case.get("dataset", 0)
    if case["suite"] == "narrow":
        return synth.matrix_narrow(seed, case["width"], case["noise"])
    if case["suite"] == "overlap":
        return synth.matrix_overlap(seed, case["overlap"], case["noise"])
    return synth.matrix_pattern(seed, case["pattern"], case["size"], case["noise"])


def params(case, prob, generations):
    width = max(len(pl.cols if pl.cols is not None else pl.order) for pl in prob.plants)
    return dict(pop_size=600, len_min=3, len_max=min(prob.A.shape[1], width + 5),
                iterations=generations, sigma=prob.sigma, toprank_size=100, tournament_k=2,
                overlap_tau=0.5, elite_frac=0.25, penalty_base=1.2, p_crossover=0.5, seed=0)


def run_case(args):
    case, generations = args
    import numpy as np
    import oracle
    prob = problem(case)
    kw = params(case, prob, generations)
    res = oracle.run(prob.A, **kw)
    expected = [(np.sort(pl.rows), np.sort(pl.cols if pl.cols is not None else pl.order))
                for pl in prob.plants]
    top = res["toprank"][:len(expected)]
    found = [(oracle.rows(prob.A, t, 1), np.sort(np.asarray(t, np.int64))) for t in top]
    rec, rel = oracle.recovery_relevance(expected, found)
    # the same found series expanded by approximate trends (at most e broken
    # adjacent pairs per row)
    approx = {}
    for e in (1, 2):
        fe = [(oracle.rows_approx(prob.A, t, e, 1), np.sort(np.asarray(t, np.int64))) for t in top]
        approx[str(e)] = oracle.recovery_relevance(expected, fe)
    return {**case, "problem": prob.name, "params": kw,
            "generations_done": res["stats"]["generations_done"],
            "stop_reason": res["stats"]["stop_reason"], "recovery": rec, "relevance": rel,
            "approximate_trends": approx}


def means(rows):
    """Per case (problem and noise), the means over its datasets of recovery,
    relevance and the approximate-trend scores."""
    groups = {}
    for r in rows:
        groups.setdefault(r["problem"] + (f" noise {r['noise']}" if r["noise"] else ""),
                          []).append(r)
    out = {}
    for key, rs in groups.items():
        n = len(rs)
        out[key] = {"recovery": sum(r["recovery"] for r in rs) / n,
                    "relevance": sum(r["relevance"] for r in rs) / n,
                    "approximate_trends": {
                        e: [sum(r["approximate_trends"][e][q] for r in rs) / n for q in (0, 1)]
                        for e in rs[0]["approximate_trends"]}}
    return out


def _case_key(c):
    return tuple(sorted((k, c[k]) for k in ("suite", "pattern", "size", "width", "overlap",
                                              "noise") if k in c)) + (c.get("dataset", 0),)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--generations", type=int, default=10000)
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--datasets", type=int, default=1)
    ap.add_argument("--resume", action="store_true")
    a = ap.parse_args()
    name = "quality_suite" + ("" if a.datasets == 1 else f"_{a.datasets}datasets") + \
        ("" if a.generations == 10000 else f"_{a.generations}gens") + ".json"
    path = os.path.join(HERE, name)
    partial = path + ".partial"
    kept = {}
    if a.resume:
        single = os.path.join(HERE, "quality_suite" + (
            "" if a.generations == 10000 else f"_{a.generations}gens") + ".json")
        for src in (single, path, partial):
            if os.path.exists(src):
                old = json.load(open(src))
                if old["generations"] == a.generations:
                    kept.update({_case_key(c): c for c in old["cases"]})
    wanted = {_case_key(c) for c in cases(a.datasets)}
    kept = {k: c for k, c in kept.items() if k in wanted}
    import oracle
    oracle.build()
    todo = [(c, a.generations) for c in cases(a.datasets) if _case_key(c) not in kept]
    import multiprocessing as mp
    done = dict(kept)
    with ProcessPoolExecutor(a.jobs, mp_context=mp.get_context("spawn")) as ex:
        futs = {ex.submit(run_case, t): _case_key(t[0]) for t in todo}
        for fut in as_completed(futs):
            done[futs[fut]] = fut.result()
            with open(partial, "w") as f:
                json.dump({"generations": a.generations, "cases": list(done.values())}, f)
    rows = [done[_case_key(c)] for c in cases(a.datasets)]
    out = {"generator": "tests/golden/make_quality_suite.py", "generations": a.generations,
           "datasets": a.datasets, "cases": rows}
    if a.datasets > 1:
        out["means"] = means(rows)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    if os.path.exists(partial):
        os.remove(partial)
    for r in rows:
        name = r["problem"] + (f" noise {r['noise']}" if r["noise"] else "")
        print(f"{name:40s} recovery {r['recovery']:.3f} relevance {r['relevance']:.3f} "
              f"({r['generations_done']} generations, stop {r['stop_reason']})")


if __name__ == "__main__":
    main()
