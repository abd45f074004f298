"""Seeded synthetic inputs shaped like the workloads of arXiv 1801.03039.

This module only draws random numbers: matrices with planted biclusters and
populations of column series.  It holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.

The paper evaluates on the synthetic benchmark of Wang et al. (2016) and on
GEO expression sets; neither is available offline, so these generators stand in
for them with the shapes the paper states (section "Pattern discovery on
synthetic datasets": 150x100 .. 1000x100 matrices; "Scalability": up to 25,000
rows x 100 columns) and the patterns it names (shift, scale, order-preserving).

Planted order-preserving rows: the row's values on the bicluster columns are
sorted random draws laid along a random column order, plus N(0, noise^2) noise
(noise is a standard deviation).  A reversed plant lays them in decreasing
order.  Every plant records ``order``: its columns in the order along which its
rows increase.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Plant:
    rows: np.ndarray          # planted row indices
    order: np.ndarray         # columns in increasing-value order
    kind: str                 # "op", "shift", "scale", or a benchmark pattern name
    reversed: bool = False
    cols: np.ndarray = None   # the plant's columns, ascending (when order is empty)


@dataclass
class Problem:
    name: str
    A: np.ndarray             # row-major float32 [R, C]
    plants: list = field(default_factory=list)
    sigma: int = 10

    @property
    def shape(self):
        return self.A.shape


def _plant_op(rng, A, rows, cols, noise, reverse=False, draw=None):
    """Order-preserving plant: sorted draws along the random column order ``cols``."""
    k = len(cols)
    for r in rows:
        v = np.sort(draw(k) if draw is not None else rng.standard_normal(k))
        if reverse:
            v = v[::-1]
        A[r, cols] = v + (rng.standard_normal(k) * noise if noise > 0 else 0.0)
    order = cols[::-1].copy() if reverse else cols.copy()
    return Plant(rows=np.sort(np.asarray(rows)), order=np.asarray(order), kind="op",
                 reversed=reverse)


def matrix_tiny(seed: int = 0, noise: float = 0.01) -> Problem:
    """200 x 20, N(0,1) background, two disjoint planted 20 x 5 order-preserving
    biclusters."""
    rng = np.random.default_rng(seed)
    R, C = 200, 20
    A = rng.standard_normal((R, C)).astype(np.float64)
    rows = rng.permutation(R)
    cols = rng.permutation(C)
    plants = []
    for b in range(2):
        pr = rows[b * 20:(b + 1) * 20]
        pc = cols[b * 5:(b + 1) * 5]
        plants.append(_plant_op(rng, A, pr, pc, noise))
    return Problem("tiny-200x20", A.astype(np.float32), plants, sigma=10)


def matrix_paper(seed: int = 0, noise: float = 0.01) -> Problem:
    """1000 x 100, N(0,1) background with three disjoint 50 x 10 biclusters:
    shift (b_i + c_j), scale (b_i * c_j, positive factors) and order-preserving."""
    rng = np.random.default_rng(seed)
    R, C = 1000, 100
    A = rng.standard_normal((R, C)).astype(np.float64)
    rows = rng.permutation(R)
    cols = rng.permutation(C)
    plants = []
    for b, kind in enumerate(("shift", "scale", "op")):
        pr = rows[b * 50:(b + 1) * 50]
        pc = cols[b * 10:(b + 1) * 10]
        if kind == "op":
            plants.append(_plant_op(rng, A, pr, pc, noise))
            continue
        if kind == "shift":
            bi = rng.standard_normal(50)
            cj = rng.standard_normal(10)
            A[np.ix_(pr, pc)] = bi[:, None] + cj[None, :]
        else:
            bi = rng.uniform(0.5, 2.0, 50)
            cj = rng.uniform(0.5, 2.0, 10)
            A[np.ix_(pr, pc)] = bi[:, None] * cj[None, :]
        plants.append(Plant(rows=np.sort(pr), order=pc[np.argsort(cj, kind="stable")],
                            kind=kind))
    return Problem("paper-1000x100", A.astype(np.float32), plants, sigma=25)


def matrix_overlap(seed: int = 0, overlap: int = 0, noise: float = 0.01) -> Problem:
    """200 x 150 (rows x columns), N(0,1) background with three 20 x 20
    order-preserving biclusters, each sharing ``overlap`` rows and
    ``overlap`` columns with the next (the paper's overlap benchmark shape:
    0x0, 3x3, 6x6, 9x9).  A later plant overwrites an earlier one in the
    shared cells."""
    rng = np.random.default_rng(seed)
    R, C = 200, 150
    A = rng.standard_normal((R, C)).astype(np.float64)
    rows = rng.permutation(R)
    cols = rng.permutation(C)
    plants = []
    r0 = c0 = 0
    for b in range(3):
        pr = rows[r0:r0 + 20]
        pc = cols[c0:c0 + 20]
        plants.append(_plant_op(rng, A, pr, pc, noise))
        r0 += 20 - overlap
        c0 += 20 - overlap
    return Problem(f"overlap-200x150-{overlap}", A.astype(np.float32), plants, sigma=10)


PATTERNS = ("trend-preserving", "column-constant", "row-constant", "shift", "scale",
            "shift-scale")
PATTERN_SIZES = {"150x100": (150, 100, 3, 15), "200x150": (200, 150, 4, 20),
                 "300x200": (300, 200, 5, 25)}


def _plant_pattern(rng, A, pr, pc, pattern):
    """Cells of one bicluster of the given pattern; returns its Plant (``order``:
    the columns along which its rows rise; empty for row-constant, whose rows
    are flat)."""
    nr, nc = len(pr), len(pc)
    if pattern == "trend-preserving":
        plant = _plant_op(rng, A, pr, pc, 0.0)
        plant.kind = pattern
        return plant
    cj = rng.standard_normal(nc)
    if pattern == "column-constant":
        A[np.ix_(pr, pc)] = np.broadcast_to(cj[None, :], (nr, nc))
    elif pattern == "row-constant":
        A[np.ix_(pr, pc)] = np.broadcast_to(rng.standard_normal(nr)[:, None], (nr, nc))
        return Plant(rows=np.sort(pr), order=np.zeros(0, np.int64), kind=pattern,
                     cols=np.sort(pc))
    elif pattern == "shift":
        A[np.ix_(pr, pc)] = rng.standard_normal(nr)[:, None] + cj[None, :]
    elif pattern == "scale":
        A[np.ix_(pr, pc)] = rng.uniform(0.5, 2.0, nr)[:, None] * cj[None, :]
    elif pattern == "shift-scale":
        A[np.ix_(pr, pc)] = (rng.uniform(0.5, 2.0, nr)[:, None] * cj[None, :] +
                             rng.standard_normal(nr)[:, None])
    else:
        raise ValueError(pattern)
    return Plant(rows=np.sort(pr), order=pc[np.argsort(cj, kind="stable")], kind=pattern)


def matrix_pattern(seed: int = 0, pattern: str = "trend-preserving", size: str = "150x100",
                   noise: float = 0.0) -> Problem:
    """The pattern-discovery shapes of the paper's synthetic benchmark: N(0,1)
    background with disjoint square biclusters of one pattern -- 3 of 15 x 15
    in 150 x 100, 4 of 20 x 20 in 200 x 150, 5 of 25 x 25 in 300 x 200.
    Patterns: trend-preserving (sorted draws along a random column order),
    column-constant (c_j), row-constant (r_i: no column order), shift
    (r_i + c_j), scale (r_i c_j, r_i in [0.5, 2]), shift-scale (r_i c_j + s_i).
    N(0, noise^2) is added to every cell of the matrix afterwards (the noise
    sweep; noise is a standard deviation)."""
    R, C, n, w = PATTERN_SIZES[size]
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((R, C)).astype(np.float64)
    rows = rng.permutation(R)
    cols = rng.permutation(C)
    plants = [_plant_pattern(rng, A, rows[b * w:(b + 1) * w], cols[b * w:(b + 1) * w], pattern)
              for b in range(n)]
    if noise > 0:
        A += rng.standard_normal(A.shape) * noise
    return Problem(f"{pattern}-{size}", A.astype(np.float32), plants, sigma=max(5, w // 2))


def matrix_narrow(seed: int = 0, width: int = 10, noise: float = 0.0) -> Problem:
    """The narrow-bicluster shape of the paper's benchmark: 1000 x 100, N(0,1)
    background, three disjoint trend-preserving biclusters of 100 rows and
    ``width`` (10, 20 or 30) columns."""
    rng = np.random.default_rng(seed)
    R, C = 1000, 100
    A = rng.standard_normal((R, C)).astype(np.float64)
    rows = rng.permutation(R)
    cols = rng.permutation(C)
    plants = [_plant_op(rng, A, rows[b * 100:(b + 1) * 100], cols[b * width:(b + 1) * width], 0.0)
              for b in range(3)]
    if noise > 0:
        A += rng.standard_normal(A.shape) * noise
    return Problem(f"narrow-1000x100-{width}", A.astype(np.float32), plants, sigma=50)


def matrix_expression(seed: int = 0, R: int = 20000, C: int = 200, n_plants: int = 10,
                      noise: float = 0.05) -> Problem:
    """Expression-shaped: log-normal(0, 1) background, ``n_plants`` order-preserving
    plants of 100-500 rows x 8-30 columns.  Each plant shares about a quarter of
    its rows and columns with the one before it (a later plant overwrites the
    overlap); every second plant is reversed (decreasing)."""
    rng = np.random.default_rng(seed)
    A = rng.lognormal(0.0, 1.0, (R, C))
    plants = []
    prev_rows = prev_cols = None
    for b in range(n_plants):
        nr = int(rng.integers(100, 501))
        nc = int(rng.integers(8, 31))
        if prev_rows is None:
            pr = rng.choice(R, nr, replace=False)
            pc = rng.choice(C, nc, replace=False)
        else:
            kr = min(len(prev_rows), nr // 4)
            kc = min(len(prev_cols), nc // 4)
            keep_r = rng.choice(prev_rows, kr, replace=False)
            keep_c = rng.choice(prev_cols, kc, replace=False)
            rest_r = rng.choice(np.setdiff1d(np.arange(R), keep_r), nr - kr, replace=False)
            rest_c = rng.choice(np.setdiff1d(np.arange(C), keep_c), nc - kc, replace=False)
            pr = np.concatenate([keep_r, rest_r])
            pc = rng.permutation(np.concatenate([keep_c, rest_c]))
        plants.append(_plant_op(rng, A, pr, pc, noise, reverse=(b % 2 == 1),
                                draw=lambda k: rng.lognormal(0.0, 1.0, k)))
        prev_rows, prev_cols = pr, pc
    return Problem(f"expression-{R}x{C}", A.astype(np.float32), plants, sigma=50)


def matrix_random(seed: int, R: int, C: int, n_plants: int = 0, noise: float = 0.0,
                  plant_rows=(20, 60), plant_cols=(3, 8)) -> Problem:
    """N(0,1) matrix with ``n_plants`` order-preserving plants (for tests)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((R, C)).astype(np.float64)
    plants = []
    for _ in range(n_plants):
        nr = int(rng.integers(plant_rows[0], min(plant_rows[1], R) + 1))
        nc = int(rng.integers(plant_cols[0], min(plant_cols[1], C) + 1))
        pr = rng.choice(R, nr, replace=False)
        pc = rng.choice(C, nc, replace=False)
        plants.append(_plant_op(rng, A, pr, pc, noise))
    return Problem(f"random-{R}x{C}", A.astype(np.float32), plants,
                   sigma=max(10, R // 100))


@dataclass
class BatchItem:
    problem: Problem
    offsets: np.ndarray
    cols: np.ndarray


def batch_uneven(seed: int = 0, n: int = 64, rows=(500, 50000), cols=(20, 500),
                 pop=(256, 2048), max_len: int = 30) -> list:
    """``n`` independent problems of uneven size: rows uniform in ``rows``,
    columns uniform in ``cols``, N(0,1) with 1-5 order-preserving plants, each
    with its own population (size uniform in ``pop``, lengths 3..min(max_len, C)).
    Problem i is drawn from seed ``seed * 100000 + 1000 + i``."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed * 100000 + 1000 + i)
        R = int(rng.integers(rows[0], rows[1] + 1))
        C = int(rng.integers(cols[0], cols[1] + 1))
        n_pl = int(rng.integers(1, 6))
        prob = matrix_random(int(rng.integers(1 << 31)), R, C, n_plants=n_pl, noise=0.0,
                             plant_rows=(max(10, R // 200), max(20, R // 40)),
                             plant_cols=(4, min(30, C // 2)))
        P = int(rng.integers(pop[0], pop[1] + 1))
        off, cl = population(int(rng.integers(1 << 31)), P, C, 3, min(max_len, C),
                             plants=prob.plants)
        out.append(BatchItem(prob, off, cl))
    return out


def population(seed: int, P: int, C: int, Lmin: int, Lmax: int, plants=None,
               frac_planted: float = 0.5, duplicates: bool = False):
    """A CBF population (offsets[P+1], cols) of distinct-column series.

    With ``plants``, a fraction ``frac_planted`` of the series are ordered
    subsequences of a plant's increasing order (a third of them with one
    foreign column inserted) -- shaped like an evolved population, whose members
    match many rows.  The rest are uniform random series.  ``duplicates=True``
    lets random series repeat a column (the evaluator must then report 0)."""
    rng = np.random.default_rng(seed)
    seqs = []
    for _ in range(P):
        use_plant = plants and rng.random() < frac_planted
        if use_plant:
            pl = plants[int(rng.integers(len(plants)))]
            width = len(pl.order)
            hi = max(min(Lmax, width), 1)
            lo = min(Lmin, hi)
            L = int(rng.integers(lo, hi + 1))
            idx = np.sort(rng.choice(width, L, replace=False))
            s = pl.order[idx].tolist()
            if rng.random() < 1 / 3 and len(s) < Lmax and len(s) < C:
                foreign = [c for c in range(C) if c not in s]
                s.insert(int(rng.integers(len(s) + 1)), int(rng.choice(foreign)))
        else:
            L = int(rng.integers(Lmin, Lmax + 1))
            if duplicates:
                s = rng.integers(0, C, L).tolist()
            else:
                s = rng.choice(C, L, replace=False).tolist()
        seqs.append(s)
    offsets = np.zeros(P + 1, np.int32)
    offsets[1:] = np.cumsum([len(s) for s in seqs])
    cols = np.asarray([c for s in seqs for c in s], np.int32)
    return offsets, cols
