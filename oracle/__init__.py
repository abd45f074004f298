"""EBIC CPU oracle -- test infrastructure only.

A plain C++ restatement of the method of arXiv 1801.03039 (support from the
"Motivation" section, Eq. (1), the CBF of Fig. 3 and Steps 1-5 of the "EBIC
Algorithm" section), loaded through ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the CUDA library neither imports nor links it.

``build()`` compiles ``ebic_oracle.cpp`` with ``-O2 -fno-fast-math
-ffp-contract=off`` (IEEE binary32/binary64, no fused multiply-add) and OpenMP
into ``oracle/_build/libebic_oracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebic_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libebic_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-std=c++17",
          "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["g++", *CFLAGS, _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("pop_size", ctypes.c_int32), ("len_min", ctypes.c_int32),
        ("len_max", ctypes.c_int32), ("iterations", ctypes.c_int32),
        ("sigma", ctypes.c_int32), ("toprank_size", ctypes.c_int32),
        ("tournament_k", ctypes.c_int32), ("fitness_support", ctypes.c_int32),
        ("overlap_tau", ctypes.c_double), ("elite_frac", ctypes.c_double),
        ("penalty_base", ctypes.c_double), ("p_crossover", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("oversample", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("generations_done", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
        ("tabu_hits_total", ctypes.c_int64), ("attempts_total", ctypes.c_int64),
        ("evaluations_total", ctypes.c_int64), ("last_gen_hits", ctypes.c_int32),
        ("toprank_n", ctypes.c_int32),
    ]


_P = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_philox4x32_10.argtypes = [_P, _P, _P]
            lib.or_draw.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
            lib.or_draw.restype = ctypes.c_uint32
            lib.or_support.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                       ctypes.c_int32, _P, _P, ctypes.c_int32]
            lib.or_rows.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                    ctypes.c_int32, _P]
            lib.or_rows.restype = ctypes.c_int32
            lib.or_fitness.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
            lib.or_fitness.restype = ctypes.c_double
            lib.or_omp_max_threads.restype = ctypes.c_int32
            lib.or_random_series.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]
            lib.or_random_series.restype = ctypes.c_int32
            lib.or_crossover.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, _P]
            lib.or_crossover.restype = ctypes.c_int32
            lib.or_mutate.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, _P, _P]
            lib.or_mutate.restype = ctypes.c_int32
            lib.or_penalized.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_double]
            lib.or_penalized.restype = ctypes.c_double
            lib.or_tournament.argtypes = [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P,
                                          ctypes.c_int32, ctypes.c_double]
            lib.or_tournament.restype = ctypes.c_int32
            lib.or_toprank_update.argtypes = [_P, _P, _P, ctypes.c_int32, _P, _P, _P,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                              _P, _P, _P]
            lib.or_toprank_update.restype = ctypes.c_int32
            lib.or_rows_approx.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, _P]
            lib.or_rows_approx.restype = ctypes.c_int32
            lib.or_screen_attempt.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              _P, _P, ctypes.c_int32, _P, _P, _P, _P,
                                              ctypes.c_int32, _P, _P, _P, _P, _P, _P]
            lib.or_screen_attempt.restype = ctypes.c_int32
            lib.or_run.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Params),
                                   _P, _P, _P, _P, ctypes.POINTER(Stats),
                                   _P, _P, _P, _P, _P, _P, _P, _P, _P]
            lib.or_run.restype = ctypes.c_int32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox-4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed: int, g: int, j: int, d: int) -> int:
    """Draw number d of attempt j in generation g."""
    return int(_load().or_draw(seed, g, j, d))


def support(A, offsets, cols, nthreads: int = 1):
    """(inc, dec) for each series of a CBF population over row-major A."""
    A = _c(A, np.float32)
    R, C = A.shape
    offsets = _c(offsets, np.int32)
    cols = _c(cols, np.int32)
    P = offsets.shape[0] - 1
    inc = np.zeros(P, np.uint32)
    dec = np.zeros(P, np.uint32)
    _load().or_support(_ptr(A), R, C, _ptr(offsets), _ptr(cols), P, _ptr(inc), _ptr(dec),
                       nthreads)
    return inc, dec


def fitness(n: int, J: int, sigma: int) -> float:
    """Eq. (1) for one bicluster with n rows and J columns."""
    return float(_load().or_fitness(int(n), int(J), int(sigma)))


def fitness_array(n, J, sigma):
    n = np.asarray(n)
    J = np.asarray(J)
    return np.array([fitness(int(a), int(b), sigma) for a, b in zip(n.ravel(), J.ravel())],
                    dtype=np.float64).reshape(n.shape)


def omp_max_threads() -> int:
    return int(_load().or_omp_max_threads())


def random_series(seed, g, j, C, Lmin, Lmax):
    out = np.zeros(Lmax, np.int32)
    n = _load().or_random_series(seed, g, j, C, Lmin, Lmax, _ptr(out))
    return out[:n].copy()


def crossover(a, b, cut_a, cut_b, Lmax):
    a = _c(a, np.int32)
    b = _c(b, np.int32)
    out = np.zeros(len(a) + len(b) + 1, np.int32)
    n = _load().or_crossover(_ptr(a), len(a), _ptr(b), len(b), cut_a, cut_b, Lmax, _ptr(out))
    return out[:n].copy()


MUT_NAMES = ("insert", "delete", "swap", "substitute", "none")


def mutate(s, C, Lmin, Lmax, r_type, r1, r2):
    s = _c(s, np.int32)
    out = np.zeros(len(s) + 1, np.int32)
    kind = np.zeros(1, np.int32)
    n = _load().or_mutate(_ptr(s), len(s), C, Lmin, Lmax, r_type, r1, r2, _ptr(out), _ptr(kind))
    return out[:n].copy(), MUT_NAMES[int(kind[0])]


def penalized(f, S, L, base):
    return float(_load().or_penalized(f, S, L, base))


def to_cbf(seqs):
    """List of column sequences -> (offsets[P+1], cols)."""
    offsets = np.zeros(len(seqs) + 1, np.int32)
    for i, s in enumerate(seqs):
        offsets[i + 1] = offsets[i] + len(s)
    cols = np.concatenate([np.asarray(s, np.int32) for s in seqs]) if seqs else np.zeros(0, np.int32)
    return offsets, cols.astype(np.int32)


def tournament(entrants, seqs, f, pen, base):
    off, cols = to_cbf(seqs)
    e = _c(entrants, np.int32)
    f = _c(f, np.float64)
    pen = _c(pen, np.int64)
    return int(_load().or_tournament(_ptr(e), len(e), _ptr(off), _ptr(cols), len(seqs), _ptr(f),
                                     _ptr(pen), len(pen), base))


def toprank_update(list_seqs, list_f, pop_seqs, pop_f, T, tau):
    loff, lcols = to_cbf(list_seqs)
    poff, pcols = to_cbf(pop_seqs)
    lf = _c(list_f, np.float64)
    pf = _c(pop_f, np.float64)
    cap = len(list_seqs) + len(pop_seqs)
    ooff = np.zeros(cap + 1, np.int32)
    ocols = np.zeros(max(1, len(lcols) + len(pcols)), np.int32)
    of = np.zeros(max(1, cap), np.float64)
    n = _load().or_toprank_update(_ptr(loff), _ptr(lcols), _ptr(lf), len(list_seqs), _ptr(poff),
                                  _ptr(pcols), _ptr(pf), len(pop_seqs), T, tau, _ptr(ooff),
                                  _ptr(ocols), _ptr(of))
    seqs = [ocols[ooff[i]:ooff[i + 1]].tolist() for i in range(n)]
    return seqs, of[:n].copy()


def rows(A, seq, mode: int = 0) -> np.ndarray:
    """Step 6: rows rising strictly along seq (mode 0); with Step 7's
    negative-trend expansion, rows rising or falling strictly (mode 1)."""
    A = _c(A, np.float32)
    R, C = A.shape
    s = np.ascontiguousarray(seq, np.int32)
    out = np.zeros(R, np.int32)
    n = _load().or_rows(_ptr(A), R, C, _ptr(s), len(s), int(mode), _ptr(out))
    return out[:n].copy()


def rows_approx(A, seq, e: int, mode: int = 0) -> np.ndarray:
    """Step 7 by approximate trends (reading: at most e adjacent pairs of a
    row break the order): mode 0 rising, mode 1 rising or falling."""
    A = _c(A, np.float32)
    R, C = A.shape
    s = np.ascontiguousarray(seq, np.int32)
    out = np.zeros(R, np.int32)
    n = _load().or_rows_approx(_ptr(A), R, C, _ptr(s), len(s), int(e), int(mode), _ptr(out))
    return out[:n].copy()


def recovery_relevance(expected, found):
    """Eq. (2)-(3): a bicluster is the set of cells rows x cols; the Jaccard
    index of two biclusters is |e & f| / |e | f| over cells.  Recovery is the
    mean over expected biclusters of the best Jaccard index against the found
    ones, relevance the mean over found biclusters of the best against the
    expected ones (reading: the sums of Eq. (2)-(3) divided by the number of
    terms, which puts both in [0, 1]; no found bicluster gives 0 and 0)."""
    def jac(e, f):
        er, ec = set(map(int, e[0])), set(map(int, e[1]))
        fr, fc = set(map(int, f[0])), set(map(int, f[1]))
        inter = len(er & fr) * len(ec & fc)
        union = len(er) * len(ec) + len(fr) * len(fc) - inter
        return inter / union if union else 0.0
    if not expected or not found:
        return 0.0, 0.0
    J = [[jac(e, f) for f in found] for e in expected]
    rec = sum(max(row) for row in J) / len(expected)
    rel = sum(max(J[i][j] for i in range(len(expected))) for j in range(len(found))) / len(found)
    return rec, rel


def make_params(**kw) -> Params:
    d = dict(pop_size=100, len_min=2, len_max=6, iterations=10, sigma=10, toprank_size=100,
             tournament_k=2, fitness_support=0, overlap_tau=0.5, elite_frac=0.25,
             penalty_base=1.2, p_crossover=0.5, seed=0, oversample=1)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def screen_attempt(C, g, j, seqs, f, pen, tabu=(), **kw):
    """One attempt of Step 3 with offspring screening (make_child): attempt j
    of generation g drawn from the population `seqs` (fitness f, penalty
    counts pen[C]) against the tabu list `tabu` as it stood at the
    generation's start.  Returns the candidates, their pseudo scores (V > 1),
    the tournament outcome and the child."""
    p = make_params(**kw)
    V, L = max(1, p.oversample), p.len_max
    off, cols = to_cbf(seqs)
    toff, tcols = to_cbf(list(tabu)) if len(tabu) else (np.zeros(1, np.int32),
                                                        np.zeros(1, np.int32))
    f = _c(f, np.float64)
    pen = _c(pen, np.int64)
    cl = np.zeros(V, np.int32)
    cc = np.zeros(V * L, np.int32)
    sc = np.zeros(V, np.uint32)
    oc = np.zeros(1, np.int32)
    chl = np.zeros(1, np.int32)
    chc = np.zeros(L, np.int32)
    rc = _load().or_screen_attempt(ctypes.byref(p), C, g, j, _ptr(off), _ptr(cols), len(seqs),
                                   _ptr(f), _ptr(pen), _ptr(toff), _ptr(tcols), len(tabu),
                                   _ptr(cl), _ptr(cc), _ptr(sc), _ptr(oc), _ptr(chl), _ptr(chc))
    if rc < 0:
        raise ValueError("invalid parameters")
    cands = [cc[v * L:v * L + cl[v]].tolist() for v in range(V)]
    return {"cands": cands, "scores": sc.tolist(), "outcome": int(oc[0]),
            "child": chc[:chl[0]].tolist()}


def run(A, trace: bool = False, **kw):
    """Run the sequential EA.  Returns a dict with the final top-rank list,
    stats and (when trace=True) the per-generation populations and lists."""
    A = _c(A, np.float32)
    R, C = A.shape
    p = make_params(**kw)
    P, T, L, G = p.pop_size, p.toprank_size, p.len_max, p.iterations
    top_len = np.zeros(T, np.int32)
    top_cols = np.zeros(T * L, np.int32)
    top_f = np.zeros(T, np.float64)
    top_inc = np.zeros(T, np.uint32)
    st = Stats()
    tr = {}
    if trace:
        tr = dict(pop_len=np.zeros((G + 1) * P, np.int32),
                  pop_cols=np.zeros((G + 1) * P * L, np.int32),
                  pop_inc=np.zeros((G + 1) * P, np.uint32),
                  pop_dec=np.zeros((G + 1) * P, np.uint32),
                  pop_f=np.zeros((G + 1) * P, np.float64),
                  top_n=np.zeros(G + 1, np.int32),
                  top_len=np.zeros((G + 1) * T, np.int32),
                  top_cols=np.zeros((G + 1) * T * L, np.int32),
                  top_f=np.zeros((G + 1) * T, np.float64))
    rc = _load().or_run(_ptr(A), R, C, ctypes.byref(p), _ptr(top_len), _ptr(top_cols),
                        _ptr(top_f), _ptr(top_inc), ctypes.byref(st),
                        _ptr(tr.get("pop_len")), _ptr(tr.get("pop_cols")),
                        _ptr(tr.get("pop_inc")), _ptr(tr.get("pop_dec")),
                        _ptr(tr.get("pop_f")), _ptr(tr.get("top_n")),
                        _ptr(tr.get("top_len")), _ptr(tr.get("top_cols")),
                        _ptr(tr.get("top_f")))
    if rc != 0:
        raise ValueError("oracle rejected the EA parameters")
    n = st.toprank_n
    out = dict(
        toprank=[top_cols[i * L:i * L + top_len[i]].tolist() for i in range(n)],
        toprank_f=top_f[:n].copy(), toprank_inc=top_inc[:n].copy(),
        stats={f: getattr(st, f) for f, _ in Stats._fields_})
    if trace:
        gens = st.generations_done + 1
        pops, tops = [], []
        for g in range(gens):
            pl = tr["pop_len"][g * P:(g + 1) * P]
            pc = tr["pop_cols"][g * P * L:(g + 1) * P * L].reshape(P, L)
            pops.append(dict(seqs=[pc[i, :pl[i]].tolist() for i in range(P)],
                             inc=tr["pop_inc"][g * P:(g + 1) * P].copy(),
                             dec=tr["pop_dec"][g * P:(g + 1) * P].copy(),
                             f=tr["pop_f"][g * P:(g + 1) * P].copy()))
            tn = tr["top_n"][g]
            tl = tr["top_len"][g * T:(g + 1) * T]
            tc = tr["top_cols"][g * T * L:(g + 1) * T * L].reshape(T, L)
            tops.append(dict(seqs=[tc[i, :tl[i]].tolist() for i in range(tn)],
                             f=tr["top_f"][g * T:g * T + tn].copy()))
        out["trace_pop"] = pops
        out["trace_top"] = tops
    return out
