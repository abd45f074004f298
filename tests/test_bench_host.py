"""Host-side logic of bench.py on the CPU: the multi-rank helpers over a
two-process gloo group, the reference arm's rank handling and JSON line, the
clock-sample summary, the per-rank seeding of the weak-scaling workloads,
and the surrogate comparison's time-to-quality bookkeeping."""
import argparse
import json
import os
import socket

import numpy as np
import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        bench.barrier(ws)
        # per-rank step times: the job's time is the slowest rank's
        slowest = bench.aggregate_max(1.5 + 2.25 * rank, ws, device="cpu")
        bench.barrier(ws)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"slowest": slowest}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks(tmp_path):
    """bench.py's barrier and max-over-ranks timing on a world of two."""
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert json.load(open(tmp_path / f"rank{r}.json")) == {"slowest": 3.75}


def test_single_rank_helpers_need_no_group():
    assert bench.aggregate_max(3.25, 1) == 3.25
    bench.barrier(1)


def test_reference_arm_runs_on_rank_zero_only():
    args = argparse.Namespace(workload="eval-expression", steps=1, warmup=3, impl="reference")
    assert bench.run_reference(args, 2, 1) is None
    out = bench.run_reference(args, 2, 0)
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["metric"] == bench.METRIC and out["unit"] == "tests/s"
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": "tests/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["config"]["workload"] == "eval-expression-20000x200-P4096-L3-30"
    json.dumps(out)


def _row(bus, sm, mx, stamp, reasons=("Not Active",) * 4):
    return ", ".join([bus, str(sm), str(mx), "900.0", "0x0", *reasons, stamp])


def test_clock_summary_keeps_this_gpu_inside_the_timed_region():
    t0 = bench.ClockSampler._when("2026/12/03 10:00:00.000")
    t1 = bench.ClockSampler._when("2026/12/03 10:00:02.000")
    lines = [
        _row("00000000:0A:00.0", 1000, 2070, "2026/12/03 09:59:58.000"),      # before
        _row("00000000:0A:00.0", 2070, 2070, "2026/12/03 10:00:00.500"),
        _row("00000000:0A:00.0", 2060, 2070, "2026/12/03 10:00:01.000",
             ("Not Active", "Not Active", "Not Active", "Active")),
        _row("00000000:0A:00.0", 2070, 2070, "2026/12/03 10:00:01.500"),
        _row("00000000:1B:00.0", 500, 2070, "2026/12/03 10:00:01.000",         # other GPU
             ("Active", "Not Active", "Not Active", "Not Active")),
        _row("00000000:0A:00.0", 300, 2070, "2026/12/03 10:00:09.000"),       # after
        "malformed line",
    ]
    got = bench.ClockSampler.summarize(lines, "00000000:0a:00.0", t0, t1)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    # without usable stamps every sample of the GPU counts
    bare = [",".join(line.split(",")[:9]) for line in lines[:4]]
    got = bench.ClockSampler.summarize(bare, "", t0, t1)
    assert got["samples"] == 4 and got["sm_mhz"] == 2065.0


def test_weak_scaling_workloads_are_seeded_by_rank():
    """Each rank times its own problem (no data-path collective)."""
    a, b = bench.GenerationsPaper(0), bench.GenerationsPaper(1)
    assert a.prob.A.shape == b.prob.A.shape == (1000, 100)
    assert not np.array_equal(a.prob.A, b.prob.A)
    assert a.params_kw(10)["seed"] == 0 and b.params_kw(10)["seed"] == 1
    e0, e1 = bench.EvalExpression(0), bench.EvalExpression(1)
    assert not np.array_equal(e0.prob.A, e1.prob.A)
    assert e0.units_per_step() == e1.units_per_step() == 4096 * 20000


def test_screened_comparison_scores_time_to_quality():
    """The surrogate comparison's bookkeeping: generations and seconds (at the
    arm's rate) to 99% of the plain run's final best, and the summary."""
    def arm(gps, best, curve):
        return {"generations_per_s": gps, "generations": len(curve), "final_best_fitness": best,
                "tabu_hits": 0, "curve": curve}
    arms = ["plain", "screened", "random_scores"]
    rows = []
    for seed, scale in ((0, 1.0), (1, 2.0)):
        row = {"seed": seed,
               "plain": arm(1000.0, 10.0 * scale, [scale * x for x in (5.0, 9.0, 9.95, 10.0)]),
               "screened": arm(500.0, 12.0 * scale, [scale * x for x in (9.9, 11.0, 12.0, 12.0)]),
               "random_scores": arm(1100.0, 9.0 * scale, [scale * x for x in (5.0, 6.0, 8.0, 9.0)])}
        rows.append(bench.GenerationsScreened.score_seed(row, arms))
    for r in rows:
        assert r["plain"]["generations_to_99pct_of_plain_best"] == 3
        assert r["plain"]["seconds_to_99pct_of_plain_best"] == pytest.approx(3 / 1000.0)
        assert r["screened"]["generations_to_99pct_of_plain_best"] == 1
        assert r["screened"]["seconds_to_99pct_of_plain_best"] == pytest.approx(1 / 500.0)
        assert r["random_scores"]["generations_to_99pct_of_plain_best"] is None
        assert r["random_scores"]["seconds_to_99pct_of_plain_best"] is None
        assert r["screened_best_over_plain_best"] == pytest.approx(1.2)
        assert "curve" not in r["plain"]
    out = bench.GenerationsScreened.summarize(rows, arms)
    assert out["within_1pct_every_seed"] and out["screened_best_over_plain_best_min"] == pytest.approx(1.2)
    s = out["summary"]
    assert s["screened"]["mean_seconds_to_99pct_of_plain_best"] == pytest.approx(0.002)
    assert s["random_scores"]["seeds_reaching_99pct_of_plain_best"] == 0
    assert s["random_scores"]["mean_seconds_to_99pct_of_plain_best"] is None
    assert s["plain"]["mean_final_best_fitness"] == pytest.approx(15.0)


def test_byte_counts_of_the_fitness_pass():
    """The roofline's byte counts on a hand-sized population: without the
    early exit every AND step reads a whole table row; with it, only the
    128-row blocks still alive, so never more."""
    wl = bench.EvalExpression(0)
    R = wl.prob.A.shape[0]
    row = (R + 127) // 128 * 16                        # 157 blocks x 16 B at R = 20,000
    assert row == 157 * 16
    wl.off = np.array([0, 3, 4, 9], np.int32)          # lengths 3, 1, 5 -> 2 + 0 + 4 steps
    wl.cols = np.array([0, 1, 2, 7, 3, 4, 5, 6, 8], np.int32)
    wl.P = 3
    io = wl.off.nbytes + wl.cols.nbytes + 3 * 12
    assert wl.full_table_bytes() == 6 * row + io
    alg, _ = wl.algorithmic_bytes()
    assert io + 157 * 16 <= alg <= wl.full_table_bytes()   # the first step reads every block


def _brute_bytes(A, off, cols, unit, first_column):
    R = A.shape[0]
    Rp = (R + 127) // 128 * 128
    total = 0
    for i in range(len(off) - 1):
        s = cols[off[i]:off[i + 1]]
        if len(s) < 2:
            continue
        alive = np.zeros(Rp, bool)
        alive[:] = True                                   # the running AND starts all ones
        if first_column:
            total += Rp // unit
        for t in range(len(s) - 1):
            total += int(alive.reshape(-1, unit).any(axis=1).sum())
            rises = np.zeros(Rp, bool)
            rises[:R] = A[:, s[t]] < A[:, s[t + 1]]
            alive &= rises
    return 16 * total


@pytest.mark.parametrize("path,unit,first", [("bitmask", 128, False), ("gather", 4, True)])
def test_support_bytes_matches_a_direct_count(path, unit, first):
    """The roofline's algorithmic-byte model against a direct count of the
    alive 128-row blocks (bitmask) or 4-row groups (gather) before every AND
    step, on ragged shapes with ties, NaN and repeated columns."""
    rng = np.random.default_rng(3)
    for R, C in ((1, 3), (130, 5), (700, 9), (2000, 12)):
        A = rng.integers(-3, 4, (R, C)).astype(np.float32)
        A[rng.random(A.shape) < 0.02] = np.nan
        seqs = [rng.integers(0, C, int(rng.integers(1, 7))).tolist() for _ in range(40)]
        seqs += [list(range(C)), [0]]
        off = np.zeros(len(seqs) + 1, np.int32)
        off[1:] = np.cumsum([len(x) for x in seqs])
        cols = np.array([c for x in seqs for c in x], np.int32)
        assert bench.support_bytes(A, off, cols, path) == _brute_bytes(A, off, cols, unit, first)


def test_traffic_lookup_per_kernel_and_staged_steps(tmp_path, monkeypatch):
    """The DRAM traffic of the timed kernel comes from the committed ncu
    summary of that kernel and number of staged steps, else null."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_w.json").write_text(json.dumps({"kernels": [
        {"kernel": "k_support_staged<checked, CbfPop, NVT>",
         "dram_bytes_per_launch_by_dense_steps": {"4": 11, "6": 12}},
        {"kernel": "k_support_phased<checked, CbfPop>",
         "dram_bytes_per_launch_by_dense_steps": {"5": 21}}]}))
    (prof / "traffic_one.json").write_text(json.dumps({"kernel": "k_support_bitmask_warp<x>",
                                                       "dram_bytes_per_launch": 7}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic("w", "k_support_staged", {"dense_steps": 6}) == 12
    assert bench.read_traffic("w", "k_support_staged", {"dense_steps": 0}) == 11
    assert bench.read_traffic("w", "k_support_phased", {"dense_steps": 0}) == 21
    assert bench.read_traffic("w", "k_support_phased", {"dense_steps": 6}) is None
    assert bench.read_traffic("w", "k_support_bitmask_warp", {}) is None
    assert bench.read_traffic("one", "k_support_bitmask_warp", {}) == 7
    assert bench.read_traffic("missing", "k_support_staged", {}) is None
    assert bench.kernel_name({"kernel": 4}) == "k_support_phased"
