#!/usr/bin/env python
"""Measurement of the EBIC hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Prints ONE JSON line (rank 0).  Workloads (seeded synthetic inputs, see
paper_1801_03039_gb300/synth.py):

  eval-expression  (default) 20,000 x 200 log-normal matrix with 10 planted
                   overlapping order-preserving biclusters; a population of
                   4,096 series of length 3-30.  A step is one fitness pass
                   (support + Eq. (1)) of the whole population through the C ABI
                   on device buffers.  The line also carries, as sub-objects,
                   the generation workload below (rank 0) and an L2 probe.
  generations-paper 1,000 x 100 N(0,1) matrix with shift, scale and
                   order-preserving 50 x 10 plants; population 600 of length
                   3-20.  A step is one generation of Steps 2-5, run on the
                   device as a replayed CUDA graph.
  generations-screened  the generations-paper run with offspring screening
                   (8 candidate children per attempt, best surrogate score
                   goes on); the surrogate is trained first on pairs logged
                   from plain runs of other seeds.  Reports the plain-vs-
                   screened comparison and the held-out ranking quality.
  eval-batch       64 independent problems of uneven size in one persistent
                   launch (graph replay).

Timing: W untimed warm-up steps, then K steps, each timed with CUDA events on
the launching stream.  Before every timed step the L2 is flushed outside the
timed interval: a 512 MiB buffer is overwritten and then a second 512 MiB
buffer is read, so that the L2 holds no line of the workload and no dirty line
whose write-back would land in the timed step.  SM clocks and throttle reasons
are sampled with nvidia-smi during the timed steps.  With torchrun (N > 1)
every rank runs its own independent problem (seeded by its rank; no
collective on the data path) and rank 0 reports the whole-job aggregate over
the slowest rank's time (weak scaling).

``--impl reference`` times the CPU oracle (the plain restatement of the
method used by the tests) on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidate×row support tests/sec and generations/sec at 1 GB300; % of roofline"
L2_FLUSH_BYTES = 512 << 20


# ---------------------------------------------------------------------------
# distributed plumbing (rank-local problems, max-over-ranks timing)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_max(value: float, ws: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "timestamp")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-f", self.path], stdout=subprocess.DEVNULL,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        self.t0 = time.time()

    @staticmethod
    def _when(stamp: str):
        """nvidia-smi's local timestamp ("YYYY/MM/DD HH:MM:SS.mmm") as epoch seconds."""
        try:
            import datetime
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t1 = time.time()
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        return self.summarize(lines, self.bus_id, self.t0, t1)

    @classmethod
    def summarize(cls, lines, bus_id: str, t0: float, t1: float) -> dict:
        """Median SM clock, max clock and active throttle reasons of the
        nvidia-smi samples (CSV lines in FIELDS order) of this GPU taken
        between t0 and t1 (all samples if none carries a usable stamp)."""
        rows = []
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        buses = {r[0].lower()[-7:] for r in rows}
        if len(buses) > 1 and bus_id:
            rows = [r for r in rows if r[0].lower()[-7:] == bus_id.lower()[-7:]]
        # keep the samples taken inside the timed region when the stamps allow
        inside = [r for r in rows if len(r) >= 10 and (cls._when(r[9]) or 0) >= t0 - 0.05
                  and (cls._when(r[9]) or 0) <= t1 + 0.05]
        if inside:
            rows = inside
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def load_peaks() -> dict:
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        d["source"] = "measured"
        return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


class L2Flush:
    """Leaves the L2 without any line of the workload and without dirty lines:
    a 512 MiB buffer is overwritten, then a second 512 MiB buffer is read."""

    def __init__(self, torch):
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        self.r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        self.desc = ("flushed before every timed step: a 512 MiB buffer overwritten, then a "
                     "second 512 MiB buffer read (no workload line and no dirty line left in L2)")

    def __call__(self, i: int):
        self.w.fill_(i)
        self.r.max()


def support_bytes(A, offsets, cols, path: str) -> int:
    """Algorithmic bytes of one support pass over a CBF population, with the
    early exit of the kernels (the rows of a series that stop rising are not
    read again):
      bitmask  16 B per (series, 128-row block, AND step) taken while the block
               still holds a rising row (every block at step 0);
      gather   16 B per (series, 4-row group, column read) while the group
               still holds a rising row: the first column and every step.
    Rows are padded to a multiple of 128, as on the device."""
    A = np.asarray(A, np.float32)
    R = A.shape[0]
    Rp = (R + 127) // 128 * 128
    At = np.ascontiguousarray(A.T)
    unit = 128 if path == "bitmask" else 4
    total = 0
    for i in range(len(offsets) - 1):
        s = cols[offsets[i]:offsets[i + 1]]
        L = len(s)
        if L < 2:
            continue
        groups = Rp // unit
        total += groups * (0 if path == "bitmask" else 1)          # the gather's first column
        rows = np.arange(R)
        for t in range(L - 1):
            total += groups
            a, b = At[s[t]], At[s[t + 1]]
            rows = rows[a[rows] < b[rows]]
            if rows.size == 0:
                break
            g = rows // unit
            groups = int(np.count_nonzero(np.diff(g))) + 1
    return 16 * total


# ---------------------------------------------------------------------------
# workload: one fitness pass over an expression-shaped matrix
# ---------------------------------------------------------------------------
class EvalExpression:
    name = "eval-expression"
    DEFAULT_STEPS = 5000           # 0.1 s of timed passes (plus the flushes)
    R, C, P, LMIN, LMAX, SIGMA = 20000, 200, 4096, 3, 30, 50

    def __init__(self, rank: int):
        from paper_1801_03039_gb300 import synth
        self.prob = synth.matrix_expression(seed=rank)
        self.off, self.cols = synth.population(2 + rank, self.P, self.C, self.LMIN, self.LMAX,
                                               plants=self.prob.plants)

    def config(self):
        return {"workload": "eval-expression-20000x200-P4096-L3-30",
                "rows": self.R, "cols": self.C, "population": self.P,
                "series_len": [self.LMIN, self.LMAX], "sigma": self.SIGMA,
                "support_path": "bitmask", "support_mode": "inc",
                "launch_shape": getattr(self, "tuning", None),
                "launch_shape_source": getattr(self, "tuning_source", None),
                "l2": getattr(self, "l2_desc", None)}

    def units_per_step(self) -> int:          # candidate x row tests per step
        return self.P * self.R

    # -- GPU ---------------------------------------------------------------
    def setup_gpu(self, torch, eb):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.h = eb.ebic_load_matrix(self.prob.A)
        eb.ebic_set_path(self.h, eb.PATH_BITMASK)
        self.d_off = torch.from_numpy(self.off).to(dev)
        self.d_cols = torch.from_numpy(self.cols).to(dev)
        self.d_inc = torch.zeros(self.P, dtype=torch.int32, device=dev)
        self.d_fit = torch.zeros(self.P, dtype=torch.float64, device=dev)
        if getattr(self, "forced_tuning", None):
            eb.ebic_set_eval_tuning(self.h, **self.forced_tuning)
            self.tuning = eb.ebic_get_eval_tuning(self.h)
            self.tuning_source = "set by --tuning"
        else:
            # one-time autotuning of the launch shape on this population
            # (untimed), each candidate timed with the L2 emptied first, as the
            # timed steps are
            self.tuning, self.tuned_us = eb.ebic_autotune_eval(
                self.h, self.d_off, self.d_cols, self.P, len(self.cols), self.SIGMA,
                eb.SUPPORT_INC, self.d_inc, None, self.d_fit, flags=eb.TUNE_COLD_L2)
            self.tuning_source = "ebic_autotune_eval with EBIC_TUNE_COLD_L2"
        torch.cuda.synchronize()

    def step_gpu(self, torch, eb, stream):
        eb.ebic_eval_population_dev(self.h, self.d_off, self.d_cols, self.P, len(self.cols),
                                    self.SIGMA, eb.SUPPORT_INC, self.d_inc, None, self.d_fit,
                                    stream=stream)

    def e2e_gpu(self, torch, eb, steps: int) -> dict:
        """Same metric through the host-buffer C-ABI call (copies inside)."""
        off = torch.from_numpy(self.off).pin_memory().numpy()
        cols = torch.from_numpy(self.cols).pin_memory().numpy()
        eb.ebic_eval_population(self.h, off, cols, self.SIGMA, eb.SUPPORT_INC, want_dec=False)
        t0 = time.perf_counter()
        for _ in range(steps):
            inc, _, fit = eb.ebic_eval_population(self.h, off, cols, self.SIGMA, eb.SUPPORT_INC,
                                                  want_dec=False)
        dt = time.perf_counter() - t0
        return {"value": self.units_per_step() * steps / dt, "unit": "tests/s",
                "h2d_bytes_per_step": int(off.nbytes + cols.nbytes),
                "d2h_bytes_per_step": int(inc.nbytes + fit.nbytes)}

    def algorithmic_bytes(self) -> tuple[int, str]:
        """Bytes the early-exit bitmask algorithm reads per pass (support_bytes)
        plus the CBF in and the rising counts and fitness out."""
        io = self.off.nbytes + self.cols.nbytes + self.P * (4 + 8)
        return (support_bytes(self.prob.A, self.off, self.cols, "bitmask") + io,
                "16 B per (series, 128-row block, AND step) while the block holds a rising "
                "row + CBF in + inc/fitness out")

    def full_table_bytes(self) -> int:
        """The same count without the early exit: every series reads the whole
        table row (R padded to 128 rows, one bit per row) of each of its L - 1
        pairs; plus the CBF and the outputs."""
        R = self.prob.A.shape[0]
        row_bytes = (R + 127) // 128 * 16
        steps = int(np.maximum(np.diff(self.off.astype(np.int64)) - 1, 0).sum())
        return steps * row_bytes + self.off.nbytes + self.cols.nbytes + self.P * (4 + 8)

    # -- CPU oracle ----------------------------------------------------------
    def oracle_sample(self, oracle, budget_s: float, nthreads: int):
        """Times the oracle on the first n series (all rows), n sized to about a
        quarter of budget_s; once n is the whole population, whole passes are
        repeated until budget_s is spent.  Returns (series evaluated, seconds)."""
        n = 64
        while True:
            off = self.off[:n + 1]
            cols = self.cols[:off[-1]]
            t0 = time.perf_counter()
            oracle.support(self.prob.A, off, cols, nthreads=nthreads)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or n >= self.P:
                break
            n = min(self.P, n * 4)
        done = n
        while dt < budget_s and n >= self.P:
            t0 = time.perf_counter()
            oracle.support(self.prob.A, self.off, self.cols, nthreads=nthreads)
            dt += time.perf_counter() - t0
            done += n
        return done, dt


class GenerationsPaper:
    """1000 x 100 N(0,1) matrix with shift, scale and order-preserving 50 x 10
    plants; population 600, lengths 3-20, sigma 25.  A step is one generation
    (Steps 2-5: elitism, tournaments, operators, tabu, evaluation, top-rank)."""
    name = "generations-paper"
    R, C, P, LMIN, LMAX, SIGMA, T, GENS = 1000, 100, 600, 3, 20, 25, 100, 1000
    DEFAULT_STEPS = 1000           # the configuration's 1,000 generations

    def __init__(self, rank: int):
        from paper_1801_03039_gb300 import synth
        self.rank = rank
        self.prob = synth.matrix_paper(seed=rank)

    def params_kw(self, iterations: int):
        return dict(pop_size=self.P, len_min=self.LMIN, len_max=self.LMAX, iterations=iterations,
                    sigma=self.SIGMA, toprank_size=self.T, tournament_k=2, overlap_tau=0.5,
                    elite_frac=0.25, penalty_base=1.2, p_crossover=0.5, seed=self.rank)

    def config(self):
        return {"workload": "generations-paper-1000x100-P600-L3-20",
                "rows": self.R, "cols": self.C, "population": self.P,
                "series_len": [self.LMIN, self.LMAX], "sigma": self.SIGMA, "toprank": self.T,
                "tournament_k": 2, "overlap_tau": 0.5, "elite_frac": 0.25, "penalty_base": 1.2,
                "p_crossover": 0.5, "step": "one generation (Steps 2-5) as a replayed CUDA graph",
                "launch_shape": getattr(self, "tuning", None),
                "l2": getattr(self, "l2_desc", None)}

    def units_per_step(self) -> int:
        return self.P * self.R

    def setup_gpu(self, torch, eb, capacity: int):
        self.h = eb.ebic_load_matrix(self.prob.A)
        self.eb = eb
        eb.ebic_set_kernel_timing(self.h, capacity)    # event nodes around k_build
        eb.ebic_run_init(self.h, eb.ebic_default_params(**self.params_kw(capacity)))
        eb.ebic_set_kernel_timing(self.h, 0)           # later runs of the handle: off
        self.tuning = eb.ebic_get_eval_tuning(self.h)
        self.capacity = capacity

    def step_gpu(self, torch, eb, stream):
        eb.ebic_run_step_async(self.h, 1, stream)

    def check_gpu(self, torch, eb, expect_done: int):
        st = eb.ebic_run_step(self.h, 0)
        if st["stop_reason"] != 0 or st["generations_done"] != expect_done:
            raise RuntimeError(f"run stopped early: {st}")
        return st

    def profile_gpu(self, eb, n: int = 5) -> dict:
        acc = {}
        for _ in range(n):
            for k, v in eb.ebic_run_step_profiled(self.h).items():
                acc.setdefault(k, []).append(v)
        return {k: statistics.mean(v) for k, v in acc.items()}

    def e2e_gpu(self, torch, eb, steps: int) -> dict:
        """A whole user run through the host API: load the matrix, run the
        configuration's 1,000 generations, read the top-rank list, free."""
        t0 = time.perf_counter()
        h = eb.ebic_load_matrix(self.prob.A)
        top, fit, st = eb.ebic_run_generations(h, eb.ebic_default_params(
            **self.params_kw(self.GENS)))
        eb.ebic_free(h)
        dt = time.perf_counter() - t0
        gens = st["generations_done"]
        return {"value": self.units_per_step() * gens / dt, "unit": "tests/s",
                "generations_per_s": gens / dt, "generations": gens,
                "h2d_bytes_per_step": int(self.prob.A.nbytes / max(gens, 1)),
                "d2h_bytes_per_step": int(sum(len(t) for t in top) * 4 + len(fit) * 12),
                "scope": "ebic_load_matrix + ebic_run_generations (Step 1 + 1,000 generations, "
                         "top-rank read back) + ebic_free, wall clock"}

    def oracle_generations(self, oracle, budget_s: float):
        g = 2
        while True:
            t0 = time.perf_counter()
            oracle.run(self.prob.A, **self.params_kw(g))
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or g >= 256:
                return g, dt
            g *= 4


class GenerationsScreened(GenerationsPaper):
    """The generations-paper run with offspring screening by the learned
    surrogate: the surrogate is trained on (series, exact fitness) pairs logged
    from plain runs of the same matrix (other seeds), then every attempt of
    Step 3 builds 8 candidate children and the best-scoring one goes on to the
    tabu check and exact evaluation.  A step is one screened generation.
    Training, the held-out ranking quality and the plain-vs-screened
    comparison (1,000 generations each, same seed) run outside the timed
    region."""
    name = "generations-screened"
    DEFAULT_STEPS = 1000
    V = 8
    TRAIN_SEEDS = (1001, 1002)       # 2 plain runs x 1,001 generations x 600 = 1.2M pairs
    HOLDOUT_SEED = 1003
    STEPS, BATCH, LR = 3000, 4096, 1e-3

    def config(self):
        c = super().config()
        c.update({"workload": "generations-screened-1000x100-P600-L3-20-V8",
                  "oversample": self.V,
                  "step": "one screened generation (candidate children, surrogate forward, "
                          "pick, Steps 2-5) as a replayed CUDA graph",
                  "surrogate": "bf16 MLP 80-256-256-1 on sum-pooled column embeddings + "
                               "column mean/sd + length",
                  "training": getattr(self, "train_info", None)})
        return c

    def _params(self, iterations, seed):
        kw = self.params_kw(iterations)
        kw["seed"] = seed
        return self.eb.ebic_default_params(**kw)

    def _plain_run(self, seed, track=False):
        eb = self.eb
        eb.ebic_run_screen(self.h, None, 1, eb.SCREEN_OFF)
        eb.ebic_run_init(self.h, self._params(self.GENS, seed))
        if not track:
            eb.ebic_run_step(self.h, self.GENS)
            return None
        return self._tracked(self.GENS)

    def _tracked(self, gens):
        eb = self.eb
        best = []
        for _ in range(gens):
            eb.ebic_run_step(self.h, 1)
            _, fit, _ = eb.ebic_get_toprank(self.h, 1, self.LMAX)
            best.append(float(fit[0]) if len(fit) else 0.0)
        return best

    def setup_gpu(self, torch, eb, capacity: int):
        self.eb = eb
        self.h = eb.ebic_load_matrix(self.prob.A)
        t0 = time.perf_counter()
        self.sur = eb.ebic_surrogate_create(self.h, self.LMAX, self.rank)
        n = 0
        for seed in self.TRAIN_SEEDS:
            self._plain_run(seed)
            n = eb.ebic_surrogate_log(self.sur, self.h)
        t_log = time.perf_counter() - t0
        first = eb.ebic_surrogate_train(self.sur, 1, self.BATCH, self.LR)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        last = eb.ebic_surrogate_train(self.sur, self.STEPS - 1, self.BATCH, self.LR)
        t_train = time.perf_counter() - t1
        self.train_info = {"pairs": n, "runs": list(self.TRAIN_SEEDS), "steps": self.STEPS,
                           "batch": self.BATCH, "lr": self.LR, "loss_first": first,
                           "loss_last": last, "train_s": round(t_train, 3),
                           "train_steps_per_s": round((self.STEPS - 1) / t_train, 1),
                           "logging_runs_s": round(t_log, 3)}
        self.quality = self._holdout_quality(torch)
        eb.ebic_run_screen(self.h, self.sur, self.V, eb.SCREEN_SURROGATE)
        eb.ebic_set_kernel_timing(self.h, capacity)
        eb.ebic_run_init(self.h, self._params(capacity, self.rank))
        eb.ebic_set_kernel_timing(self.h, 0)
        self.tuning = eb.ebic_get_eval_tuning(self.h)
        self.capacity = capacity

    def _holdout_quality(self, torch):
        """Spearman correlation and top-10% recall of the predictions on the
        populations of a held-out plain run (every 10th generation)."""
        eb = self.eb
        eb.ebic_run_screen(self.h, None, 1, eb.SCREEN_OFF)
        eb.ebic_run_init(self.h, self._params(self.GENS, self.HOLDOUT_SEED))
        seqs, fit = [], []
        for g in range(0, self.GENS + 1, 10):
            if g:
                eb.ebic_run_step(self.h, 10)
            pop = eb.ebic_get_population(self.h, self.P, self.LMAX)
            seqs += pop["seqs"]
            fit.append(pop["f"])
        fit = np.concatenate(fit)
        n = len(seqs)
        arr = np.zeros((n, self.LMAX), np.int16)
        lens = np.zeros(n, np.int32)
        for i, x in enumerate(seqs):
            arr[i, :len(x)] = x
            lens[i] = len(x)
        d_seq = torch.from_numpy(arr).cuda()
        d_len = torch.from_numpy(lens).cuda()
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        eb.ebic_surrogate_predict(self.sur, d_seq, d_len, self.LMAX, n, out)
        pred = out.cpu().numpy().astype(np.float64)
        target = np.log1p(fit)
        ra = np.argsort(np.argsort(pred)).astype(np.float64)
        rb = np.argsort(np.argsort(target)).astype(np.float64)
        rho = float(np.corrcoef(ra, rb)[0, 1])
        k = max(1, n // 10)
        top_true = set(np.argsort(-target, kind="stable")[:k].tolist())
        top_pred = set(np.argsort(-pred, kind="stable")[:k].tolist())
        return {"pairs": n, "spearman": rho, "top10pct_recall": len(top_true & top_pred) / k,
                "source": f"plain run seed {self.HOLDOUT_SEED}, populations of every 10th "
                          "generation (not in the training log)"}

    FWD_ROWS = 1 << 17
    FWD_FLOPS = 2 * (80 * 256 + 256 * 256 + 256)      # multiply-adds of the three layers

    def forward_throughput(self, torch, eb) -> dict:
        """The surrogate's scoring kernels alone on a large batch of random
        series of one length (131,072 rows, two 65,536-row launches a call):
        CUDA events around 10 back-to-back ebic_surrogate_predict calls on one
        stream, for the tcgen05 kernel and the mma.sync one.  TFLOP/s counts
        the three layers' multiply-adds (172,544 flops a series); the feature
        gather (embedding sums) is work on top that the count leaves out."""
        peaks = load_peaks()
        peak = peaks.get("bf16_tflops")
        n, C = self.FWD_ROWS, self.prob.A.shape[1]
        rng = np.random.default_rng(7)
        st = torch.cuda.current_stream()
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        rows = {}
        for L in (3, 12, 20):
            arr = np.zeros((n, self.LMAX), np.int16)
            arr[:, :L] = np.argsort(rng.random((n, C)), axis=1)[:, :L]
            d_seq = torch.from_numpy(arr).cuda()
            d_len = torch.full((n,), L, dtype=torch.int32, device="cuda")
            row = {}
            for kind, name in ((eb.FORWARD_TCGEN05, "tcgen05"), (eb.FORWARD_MMA_SYNC, "mma_sync")):
                eb.ebic_surrogate_forward_kernel(self.sur, kind)
                for _ in range(3):
                    eb.ebic_surrogate_predict(self.sur, d_seq, d_len, self.LMAX, n, out, st)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(st)
                for _ in range(10):
                    eb.ebic_surrogate_predict(self.sur, d_seq, d_len, self.LMAX, n, out, st)
                b.record(st)
                torch.cuda.synchronize()
                us = a.elapsed_time(b) * 1e3 / 10
                tf = n * self.FWD_FLOPS / us / 1e6
                row[name] = {"us": round(us, 1), "tflops": round(tf, 1),
                             "frac_of_bf16_peak": round(tf / peak, 3) if peak else None}
            rows[f"L{L}"] = row
        eb.ebic_surrogate_forward_kernel(self.sur, eb.FORWARD_TCGEN05)
        return {"rows": n, "per_length": rows, "peak_tflops": peak,
                "peak_source": f"bf16 burst, of {peaks['source']}",
                "flops_per_series": self.FWD_FLOPS}

    COMPARE_SEEDS = 3

    def compare(self) -> dict:
        """1,000-generation runs with the same seeds in three arms: plain EBIC,
        screening with the trained surrogate, and screening with random
        (Philox) scores -- the same oversampling and the same preference for
        candidates outside the tabu list, without the model.  Per arm: wall
        time, final best exact fitness, and the generation at which the run
        first reaches 99% of the plain run's final best."""
        eb = self.eb
        arms = (("plain", None, 1, eb.SCREEN_OFF),
                ("screened", self.sur, self.V, eb.SCREEN_SURROGATE),
                ("random_scores", None, self.V, eb.SCREEN_PSEUDO))
        per_seed = []
        for i in range(self.COMPARE_SEEDS):
            seed = 10 * self.rank + i
            row = {"seed": seed}
            for name, sur, V, mode in arms:
                eb.ebic_run_screen(self.h, sur, V, mode)
                eb.ebic_run_init(self.h, self._params(self.GENS, seed))
                t0 = time.perf_counter()
                st = eb.ebic_run_step(self.h, self.GENS)
                dt = time.perf_counter() - t0
                _, fit, _ = eb.ebic_get_toprank(self.h, self.T, self.LMAX)
                eb.ebic_run_init(self.h, self._params(self.GENS, seed))
                curve = self._tracked(self.GENS)
                row[name] = {"generations_per_s": round(st["generations_done"] / dt, 1),
                             "generations": st["generations_done"],
                             "final_best_fitness": float(fit[0]),
                             "tabu_hits": st["tabu_hits_total"], "curve": curve}
            per_seed.append(self.score_seed(row, [name for name, *_ in arms]))
        eb.ebic_run_screen(self.h, None, 1, eb.SCREEN_OFF)
        out = self.summarize(per_seed, [name for name, *_ in arms])
        out["holdout"] = self.quality
        return out

    @staticmethod
    def score_seed(row: dict, arms) -> dict:
        """One seed's arms, each with its best-so-far curve: the generation
        (and the time at the arm's rate) at which it first reaches 99% of the
        plain run's final best, and the screened / plain final-best ratio."""
        target = 0.99 * row["plain"]["final_best_fitness"]
        for name in arms:
            curve = row[name].pop("curve")
            hit = next((g + 1 for g, b in enumerate(curve) if b >= target), None)
            row[name]["generations_to_99pct_of_plain_best"] = hit
            row[name]["seconds_to_99pct_of_plain_best"] = (
                None if hit is None else hit / row[name]["generations_per_s"])
        row["screened_best_over_plain_best"] = (row["screened"]["final_best_fitness"] /
                                                row["plain"]["final_best_fitness"])
        return row

    @staticmethod
    def summarize(per_seed, arms) -> dict:
        summary = {}
        for name in arms:
            secs = [r[name]["seconds_to_99pct_of_plain_best"] for r in per_seed]
            summary[name] = {
                "mean_generations_per_s": statistics.mean(r[name]["generations_per_s"] for r in per_seed),
                "mean_final_best_fitness": statistics.mean(r[name]["final_best_fitness"] for r in per_seed),
                "seeds_reaching_99pct_of_plain_best": sum(x is not None for x in secs),
                "mean_seconds_to_99pct_of_plain_best": (
                    statistics.mean(secs) if all(x is not None for x in secs) else None)}
        ratios = [r["screened_best_over_plain_best"] for r in per_seed]
        return {"per_seed": per_seed, "summary": summary,
                "screened_best_over_plain_best_min": min(ratios),
                "within_1pct_every_seed": all(x >= 0.99 for x in ratios)}

    def e2e_gpu(self, torch, eb, steps: int) -> dict:
        """A whole screened user run through the host API with the trained
        surrogate: attach it, Step 1 + 1,000 screened generations, read the
        top-rank list back."""
        h = eb.ebic_load_matrix(self.prob.A)
        t0 = time.perf_counter()
        eb.ebic_run_screen(h, self.sur, self.V, eb.SCREEN_SURROGATE)
        top, fit, st = eb.ebic_run_generations(h, self._params(self.GENS, self.rank))
        dt = time.perf_counter() - t0
        eb.ebic_free(h)
        gens = st["generations_done"]
        return {"value": self.units_per_step() * gens / dt, "unit": "tests/s",
                "generations_per_s": gens / dt, "generations": gens,
                "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(sum(len(t) for t in top) * 4 + len(fit) * 12),
                "scope": "ebic_run_screen + ebic_run_generations (Step 1 + 1,000 screened "
                         "generations, top-rank read back), wall clock; the matrix was "
                         "loaded before the timer started"}


class EvalBatch:
    """64 independent problems of uneven size (rows 500-50,000, columns
    20-500, populations 256-2,048, lengths 3-30): one step is one persistent
    launch over all of them (graph replay)."""
    name = "eval-batch"
    DEFAULT_STEPS = 300

    def __init__(self, rank: int):
        from paper_1801_03039_gb300 import synth
        self.items = synth.batch_uneven(seed=rank, n=64)
        self.P = sum(len(it.offsets) - 1 for it in self.items)
        self.R = None

    def config(self):
        return {"workload": "eval-batch-64-uneven", "problems": len(self.items),
                "rows": [500, 50000], "cols": [20, 500], "population": [256, 2048],
                "series_total": self.P, "series_len": [3, 30],
                "paths": getattr(self, "paths", None),
                "step": "one persistent launch over all problems (CUDA graph replay)",
                "l2": getattr(self, "l2_desc", None)}

    def units_per_step(self) -> int:
        return sum((len(it.offsets) - 1) * it.problem.A.shape[0] for it in self.items)

    def setup_gpu(self, torch, eb):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.handles, bitems, self.outs = [], [], []
        for it in self.items:
            h = eb.ebic_load_matrix(it.problem.A)
            P = len(it.offsets) - 1
            off = torch.from_numpy(it.offsets).to(dev)
            cols = torch.from_numpy(it.cols).to(dev)
            inc = torch.zeros(P, dtype=torch.int32, device=dev)
            fit = torch.zeros(P, dtype=torch.float64, device=dev)
            self.handles.append(h)
            self.outs.append((off, cols, inc, fit))
            bitems.append((off, cols, P, len(it.cols), it.problem.sigma, inc, fit))
        self.b = eb.ebic_batch_create(self.handles, bitems, eb.BATCH_BUILD_TABLES |
                                      eb.BATCH_AUTOTUNE | eb.BATCH_GRAPH)
        d = [eb.ebic_batch_describe(self.b, k) for k in range(len(self.items))]
        self.path_of = [x["path"] for x in d]
        self.paths = {"bitmask": sum(x["path"] == 2 for x in d),
                      "gather": sum(x["path"] == 1 for x in d),
                      "work_items": d[0]["work_items"], "grid": d[0]["grid"]}
        torch.cuda.synchronize()

    def step_gpu(self, torch, eb, stream):
        eb.ebic_batch_eval(self.b, stream)

    def e2e_gpu(self, torch, eb, steps: int) -> dict:
        """Per step: every population's CBF copied in from pinned host memory,
        one batch launch, every result copied back to pinned host memory."""
        host_in = [(torch.from_numpy(it.offsets).pin_memory(), torch.from_numpy(it.cols).pin_memory())
                   for it in self.items]
        host_out = [(torch.empty(o[2].shape, dtype=o[2].dtype).pin_memory(),
                     torch.empty(o[3].shape, dtype=o[3].dtype).pin_memory()) for o in self.outs]
        s = torch.cuda.current_stream()

        def one():
            for (ho, hc), (off, cols, _, _) in zip(host_in, self.outs):
                off.copy_(ho, non_blocking=True)
                cols.copy_(hc, non_blocking=True)
            eb.ebic_batch_eval(self.b, s)
            for (hi, hf), (_, _, inc, fit) in zip(host_out, self.outs):
                hi.copy_(inc, non_blocking=True)
                hf.copy_(fit, non_blocking=True)
            s.synchronize()

        one()
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        dt = time.perf_counter() - t0
        h2d = sum(a.nbytes + b.nbytes for a, b in ((it.offsets, it.cols) for it in self.items))
        d2h = sum(o[2].numel() * 4 + o[3].numel() * 8 for o in self.outs)
        return {"value": self.units_per_step() * steps / dt, "unit": "tests/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    def algorithmic_bytes(self, paths) -> tuple[int, str]:
        """Sum over the problems of support_bytes on each problem's path (as the
        batch autotuner chose it), plus every CBF in and the counts and fitness
        out."""
        total = 0
        for it, path in zip(self.items, paths):
            total += support_bytes(it.problem.A, it.offsets, it.cols,
                                   "bitmask" if path == 2 else "gather")
            total += it.offsets.nbytes + it.cols.nbytes + (len(it.offsets) - 1) * 12
        return total, ("per problem as the single-problem pass: bitmask 16 B per (series, "
                       "128-row block, AND step) while alive, gather 16 B per (series, 4-row "
                       "group, column read) while alive; + CBF in + inc/fitness out")

    def oracle_sample(self, oracle, budget_s: float, nthreads: int):
        it = max(self.items, key=lambda x: x.problem.A.shape[0])
        n = 16
        while True:
            off = it.offsets[:n + 1]
            cols = it.cols[:off[-1]]
            t0 = time.perf_counter()
            oracle.support(it.problem.A, off, cols, nthreads=nthreads)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or n >= len(it.offsets) - 1:
                self.R = it.problem.A.shape[0]
                return n, dt
            n = min(len(it.offsets) - 1, n * 4)


WORKLOADS = {"eval-expression": EvalExpression, "generations-paper": GenerationsPaper,
             "eval-batch": EvalBatch, "generations-screened": GenerationsScreened}


# ---------------------------------------------------------------------------
def time_workload(torch, eb, wl, steps: int, warmup: int, flush, clocks=None, ws: int = 1):
    """W warm-up steps, then `steps` steps each timed with CUDA events on the
    launching stream, the L2 flushed before each outside the timed interval.
    Returns (per-step ms list, this library's kernel launches in the timed
    region, clock summary or None)."""
    gens = isinstance(wl, GenerationsPaper)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        wl.step_gpu(torch, eb, stream)
    torch.cuda.synchronize()
    if gens:
        eb.ebic_read_kernel_timing(wl.h, reset=True)   # drop the warm-up replays
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
    barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    l0 = eb.ebic_kernel_launches()
    for i in range(steps):
        flush(i)
        events[i][0].record(stream)
        wl.step_gpu(torch, eb, stream)
        events[i][1].record(stream)
    torch.cuda.synchronize()
    launches = eb.ebic_kernel_launches() - l0
    clk = clocks.stop() if clocks else None
    return [x.elapsed_time(y) for x, y in events], launches, clk


def warm_pass_us(torch, eb, wl, steps: int = 200) -> float:
    """Mean event time of the fitness pass with the workload left in L2 (no
    flush): the table (100 MB) fits the 126 MB L2."""
    stream = torch.cuda.current_stream()
    for _ in range(5):
        wl.step_gpu(torch, eb, stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        wl.step_gpu(torch, eb, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return 1e3 * statistics.mean(x.elapsed_time(y) for x, y in ev)


def l2_probe(torch, eb, local: int) -> dict:
    """L2 size (device properties) and the read bandwidth of a buffer of half
    of it and of one of 2 GiB (the library's read probe, best of 20 passes)."""
    props = torch.cuda.get_device_properties(local)
    l2 = int(getattr(props, "L2_cache_size", 0) or 0)
    out = {"l2_bytes": l2}
    for name, nbytes in (("l2_read", (l2 // 2) // 16 * 16 if l2 else 32 << 20),
                         ("hbm_read", 2 << 30)):
        buf = torch.ones(nbytes // 4, dtype=torch.int32, device="cuda")
        us = eb.ebic_probe_read_bandwidth(buf, nbytes, 20, torch.cuda.current_stream())
        out[f"{name}_gbs"] = nbytes / us / 1e3
        out[f"{name}_buffer_bytes"] = nbytes
        del buf
    out["method"] = ("ebic_probe_read_bandwidth: one kernel reads every 16-byte vector of the "
                     "buffer once; a warm-up pass, then the fastest of 20 passes by CUDA events")
    return out


def generations_block(torch, eb, args, flush, rank: int) -> dict:
    """The 1000 x 100 generation workload (configs' paper-scale case) measured
    in the same run: 1,000 timed generations with the L2 flushed before each,
    the per-kernel breakdown, Step 3's builder against one SM's issue rate,
    the host-API run, and the sequential oracle."""
    wl = GenerationsPaper(rank)
    wl.l2_desc = flush.desc
    steps = GenerationsPaper.DEFAULT_STEPS
    wl.setup_gpu(torch, eb, capacity=args.warmup + steps + 16)
    per_step_ms, launches, _ = time_workload(torch, eb, wl, steps, args.warmup, flush)
    kb_us, kb_n = eb.ebic_read_kernel_timing(wl.h)
    if kb_n != steps:
        raise RuntimeError(f"k_build timed {kb_n} times in {steps} steps")
    st = wl.check_gpu(torch, eb, args.warmup + steps)
    kern = {k: round(v, 2) for k, v in wl.profile_gpu(eb).items()}
    total_s = sum(per_step_ms) / 1e3
    out = {"workload": wl.config()["workload"], "config": wl.config(),
           "steps": steps, "warmup": args.warmup,
           "generations_per_s": steps / total_s,
           "value": wl.units_per_step() * steps / total_s, "unit": "tests/s",
           "ms_per_step": 1e3 * total_s / steps, "gpu_launches": int(launches),
           "run_stats": st, "kernel_us": kern, "k_build_us_timed": kb_us}
    out["roofline"] = kbuild_roofline(kb_us, kern, load_peaks())
    out["e2e"] = wl.e2e_gpu(torch, eb, steps)
    out["cpu_baseline"] = cpu_baseline(wl, budget_s=8.0)
    eb.ebic_free(wl.h)
    return out


def run_ours(args, ws, rank, local):
    import torch
    import paper_1801_03039_gb300 as eb
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    eb.build()
    wl = WORKLOADS[args.workload](rank)
    if getattr(args, "tuning", None):
        wl.forced_tuning = json.loads(args.tuning)
    flush = L2Flush(torch)
    wl.l2_desc = flush.desc
    gens = isinstance(wl, GenerationsPaper)
    if gens:
        wl.setup_gpu(torch, eb, capacity=args.warmup + args.steps + 16)
    else:
        wl.setup_gpu(torch, eb)
    props = torch.cuda.get_device_properties(local)
    bus = getattr(props, "pci_bus_id", None)
    clocks = ClockSampler(bus if isinstance(bus, str) else None) if rank == 0 else None
    per_step_ms, launches, clk = time_workload(torch, eb, wl, args.steps, args.warmup, flush,
                                               clocks, ws)
    total_s = sum(per_step_ms) / 1e3
    extra = {}
    if gens:
        kb_us, kb_n = eb.ebic_read_kernel_timing(wl.h)
        if kb_n != args.steps:
            raise RuntimeError(f"k_build timed {kb_n} times in {args.steps} steps")
        extra["k_build_us_timed"] = kb_us
        extra["run_stats"] = wl.check_gpu(torch, eb, args.warmup + args.steps)
        extra["kernel_us"] = {k: round(v, 2) for k, v in wl.profile_gpu(eb).items()}
        if isinstance(wl, GenerationsScreened):
            extra["surrogate"] = wl.compare()
            extra["surrogate"]["forward"] = wl.forward_throughput(torch, eb)
    barrier(ws)
    slowest = aggregate_max(total_s, ws, device=torch.device("cuda", local))
    e2e = wl.e2e_gpu(torch, eb, max(3, args.steps))
    if ws > 1:
        e2e_val = aggregate_max(1.0 / e2e["value"], ws, device=torch.device("cuda", local))
        e2e["value"] = ws / e2e_val
    peaks = load_peaks()
    warm_us = warm_pass_us(torch, eb, wl) if isinstance(wl, EvalExpression) else None
    probe = l2_probe(torch, eb, local) if rank == 0 and not gens else None
    gen_block = None
    if rank == 0 and isinstance(wl, EvalExpression):
        gen_block = generations_block(torch, eb, args, flush, rank)
    barrier(ws)
    if rank != 0:
        return None
    value = ws * wl.units_per_step() * args.steps / slowest
    out = {
        "metric": METRIC, "value": value, "unit": "tests/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * slowest / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-compare/u32-count/f64-fitness",
        "data": "synthetic (seeded; stands in for the paper's benchmark data)",
        "config": wl.config(),
        "e2e": e2e,
        "gpu_launches": int(launches),
    }
    if gens:
        out["generations_per_s"] = ws * args.steps / slowest
    out.update(extra)
    if gens:
        out["roofline"] = kbuild_roofline(extra["k_build_us_timed"], extra["kernel_us"], peaks)
    elif isinstance(wl, EvalBatch):
        out["roofline"] = hbm_roofline(wl, per_step_ms, peaks, *wl.algorithmic_bytes(wl.path_of),
                                       kernel="k_support_batch")
    else:
        out["roofline"] = hbm_roofline(wl, per_step_ms, peaks, *wl.algorithmic_bytes(),
                                       kernel=kernel_name(wl.tuning),
                                       full=wl.full_table_bytes(), warm_us=warm_us, probe=probe)
    if probe is not None:
        out["l2_probe"] = probe
    if gen_block is not None:
        out["generations"] = gen_block
    out["clocks"] = clk
    if ws == 1:
        out["cpu_baseline"] = cpu_baseline(wl, budget_s=12.0)
    return out


def kernel_name(tuning) -> str:
    k = (tuning or {}).get("kernel", 0)
    return {4: "k_support_phased", 3: "k_support_staged",
            1: "k_support_bitmask_lane"}.get(k, "k_support_bitmask_warp")


def hbm_roofline(wl, per_step_ms, peaks, alg_bytes, alg_def, kernel, full=None, warm_us=None,
                 probe=None):
    """Achieved = algorithmic bytes per launch / mean CUDA-event time of a step
    (one launch), against the measured HBM copy bandwidth."""
    kernel_s = statistics.mean(per_step_ms) / 1e3
    achieved = alg_bytes / kernel_s / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / peaks["hbm_gbs"],
           "traffic": read_traffic(wl.name, kernel, getattr(wl, "tuning", None)),
           "algorithmic_bytes": alg_bytes, "algorithmic_def": alg_def, "kernel": kernel,
           "duration_us": 1e3 * statistics.mean(per_step_ms),
           "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peaks['source']}; burst copy, "
                          "the kernel is timed alone)"}
    if full is not None:
        out["bytes_without_early_exit"] = full
    if warm_us is not None:
        out["warm_l2"] = {"duration_us": warm_us, "achieved": alg_bytes / warm_us / 1e3,
                          "unit": "GB/s", "note": "no flush between passes: the 100 MB table "
                                                  "stays in L2"}
        if probe and probe.get("l2_read_gbs"):
            out["warm_l2"]["peak"] = probe["l2_read_gbs"]
            out["warm_l2"]["frac"] = out["warm_l2"]["achieved"] / probe["l2_read_gbs"]
            out["warm_l2"]["peak_source"] = "l2_probe.l2_read_gbs (measured in this run)"
    return out


def kbuild_roofline(kb_us, kern, peaks):
    dom = max(kern, key=kern.get)
    if dom != "k_build":
        return {"dominant_kernel": dom, "kernel_us": kern}
    # The Step 3 builder is sequential and runs in one CTA (one SM).  Its
    # bound is that SM's issue rate: four warp-instructions per cycle (one
    # per sub-partition) at the SM clock.  Work per launch = the kernel's
    # warp-instructions, from ncu samples of single launches across a
    # 1,000-generation run (committed under profiles/).  Duration: the mean
    # of the CUDA events that bracket k_build inside the replayed graph, over
    # the timed steps.
    prof = read_profile("k_build-generations-paper-1000x100.json")
    inst = prof.get("smsp__inst_executed.sum") if prof else None
    mhz = peaks.get("sm_max_mhz") or 2070.0
    peak = 4 * mhz * 1e6 / 1e9                   # G warp-instructions / s
    dur = kb_us * 1e-6
    achieved = inst / dur / 1e9 if inst else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G warp-inst/s",
            "frac": achieved / peak if achieved else None,
            "traffic": prof.get("dram_bytes_per_launch") if prof else None,
            "kernel": "k_build (Step 3 builder, one CTA of eight warps on one SM)",
            "work_per_launch": inst,
            "work_def": prof.get("work_def") if prof else None,
            "peak_source": "4 warp-instructions/cycle (one SM) x the maximum SM clock",
            "duration_us": kb_us,
            "duration_source": "CUDA events on the launching stream, recorded by event nodes "
                               "around k_build in the replayed graph, mean over the timed steps",
            "kernel_us": kern}


def read_profile(name: str):
    try:
        return json.load(open(os.path.join(ROOT, "profiles", name)))
    except (OSError, ValueError):
        return None


def read_traffic(workload: str, kernel: str, tuning=None):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary,
    if one exists for this workload, this kernel and (for the staged and the
    phased kernel) this number of staged steps (else null).  The summary holds
    one entry, or a list of entries under "kernels", one per kernel."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    try:
        top = json.load(open(p))
    except (OSError, ValueError):
        return None
    entries = top.get("kernels", [top])
    d = next((e for e in entries if str(e.get("kernel", "")).startswith(kernel)), None)
    if d is None:
        return None
    by_dense = d.get("dram_bytes_per_launch_by_dense_steps")
    if by_dense is not None:
        dense = (tuning or {}).get("dense_steps") or (5 if kernel == "k_support_phased" else 4)
        return by_dense.get(str(dense))
    return d.get("dram_bytes_per_launch")


def cpu_baseline(wl, budget_s: float):
    import oracle
    if isinstance(wl, GenerationsPaper):
        g, dt = wl.oracle_generations(oracle, budget_s)
        return {"value": wl.units_per_step() * (g + 1) / dt, "unit": "tests/s",
                "generations_per_s": (g + 1) / dt, "cores": 1, "kind": "oracle",
                "sample": f"Step 1 + {g} generations of the same run, sequential oracle on one "
                          f"core ({dt:.2f} s)"}
    cores = os.cpu_count() or 1
    n, dt = wl.oracle_sample(oracle, budget_s, cores)
    where = "the largest problem" if isinstance(wl, EvalBatch) else "the population"
    return {"value": n * wl.R / dt, "unit": "tests/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} series x all {wl.R} rows of {where} (the first series, whole "
                      f"passes repeated), OpenMP over series on {cores} threads ({dt:.2f} s)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    wl = WORKLOADS[args.workload](0)
    cores = os.cpu_count() or 1
    per_step = min(1.0, max(0.02, 120.0 / max(args.steps, 1)))   # seconds of oracle work
    if isinstance(wl, GenerationsPaper):
        g, _ = wl.oracle_generations(oracle, 4.0 * per_step)
        for _ in range(args.warmup):
            oracle.run(wl.prob.A, **wl.params_kw(1))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.run(wl.prob.A, **wl.params_kw(g))
        dt = time.perf_counter() - t0
        value = wl.units_per_step() * (g + 1) * args.steps / dt
        sample = f"each step: Step 1 + {g} generations, sequential oracle on one core"
        used = 1
    else:
        n, _ = wl.oracle_sample(oracle, 4.0 * per_step, cores)
        if isinstance(wl, EvalExpression):
            n = min(n, wl.P)                  # repeated whole passes count once per step
        if isinstance(wl, EvalBatch):
            big = max(wl.items, key=lambda x: x.problem.A.shape[0])
            A, off, cols = big.problem.A, big.offsets[:n + 1], big.cols[:big.offsets[n]]
            where = "the largest problem"
        else:
            A, off, cols = wl.prob.A, wl.off[:n + 1], wl.cols[:wl.off[n]]
            where = "the population"
        for _ in range(args.warmup):
            oracle.support(A, off, cols, nthreads=cores)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.support(A, off, cols, nthreads=cores)
        dt = time.perf_counter() - t0
        value = n * A.shape[0] * args.steps / dt
        sample = (f"first {n} series x all {A.shape[0]} rows of {where} per step, "
                  f"OpenMP on {cores} threads")
        used = cores
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "tests/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-compare/u32-count/f64-fitness",
            "data": "synthetic", "config": wl.config(),
            "cpu_baseline": {"value": value, "unit": "tests/s", "cores": used,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "tests/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the configured 1,000 generations for the "
                         "generation workloads, about half a second of GPU work for the "
                         "others; 20 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="eval-expression")
    ap.add_argument("--tuning", default=None,
                    help="eval-expression: a JSON launch shape for ebic_set_eval_tuning instead "
                         "of the autotuner (e.g. for a profiler run of one shape)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else WORKLOADS[args.workload].DEFAULT_STEPS
    if args.steps < 1:
        ap.error("--steps must be at least 1")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
