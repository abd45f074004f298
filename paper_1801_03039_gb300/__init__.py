"""GB300 (sm_103a) implementation of the EBIC hot path (arXiv 1801.03039).

A thin ctypes binding over ``libebic.so``, whose C ABI is declared in
``include/ebic.h``.  The functions below carry the C names and only marshal
arguments: every step of support counting, Eq. (1) and the generation loop
runs in the library's CUDA kernels.  There is no CPU fallback -- if the
library is missing or no GPU is visible the calls raise.

Device buffers may be given as torch CUDA tensors (or raw integer device
pointers); host buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "EbicError", "build", "lib", "ebic_kernel_launches", "ebic_load_matrix", "ebic_load_matrix_dev", "ebic_free",
    "ebic_matrix_shape", "ebic_build_pair_table", "ebic_pair_table_bytes",
    "ebic_read_pair_words", "ebic_set_path", "ebic_set_eval_tuning", "ebic_get_eval_tuning",
    "TUNE_COLD_L2", "ebic_probe_read_bandwidth",
    "ebic_autotune_eval", "ebic_eval_population",
    "ebic_eval_population_dev", "ebic_eval_population_dev_noalloc", "ebic_check_device_error", "ebic_default_params",
    "ebic_batch_create", "ebic_batch_eval", "ebic_batch_describe", "ebic_batch_free",
    "BATCH_AUTOTUNE", "BATCH_GRAPH", "BATCH_BUILD_TABLES",
    "ebic_run_init", "ebic_run_step", "ebic_run_step_async", "ebic_run_step_profiled",
    "ebic_set_kernel_timing", "ebic_read_kernel_timing",
    "ebic_get_toprank", "ebic_get_population",
    "ebic_run_generations", "Params", "Stats", "PATH_AUTO", "PATH_GATHER", "PATH_BITMASK",
    "SUPPORT_INC", "SUPPORT_INC_PLUS_DEC",
    "ebic_surrogate_create", "ebic_surrogate_free", "ebic_surrogate_params", "ebic_surrogate_grads",
    "ebic_surrogate_colstats", "ebic_surrogate_step", "ebic_surrogate_log", "ebic_surrogate_train",
    "ebic_surrogate_target_norm", "ebic_surrogate_predict", "ebic_run_screen",
    "ebic_surrogate_forward_kernel", "FORWARD_TCGEN05", "FORWARD_MMA_SYNC",
    "ebic_surrogate_train_kernel",
    "SCREEN_OFF", "SCREEN_SURROGATE", "SCREEN_PSEUDO",
    "ebic_extract_rows", "ebic_extract_rows_approx", "ebic_recovery_relevance", "ROWS_RISING", "ROWS_RISING_OR_FALLING",
]

PATH_AUTO, PATH_GATHER, PATH_BITMASK = 0, 1, 2
SUPPORT_INC, SUPPORT_INC_PLUS_DEC = 0, 1
SCREEN_OFF, SCREEN_SURROGATE, SCREEN_PSEUDO = 0, 1, 2
ROWS_RISING, ROWS_RISING_OR_FALLING = 0, 1
STATUS = {0: "EBIC_OK", 1: "EBIC_ERR_ARG", 2: "EBIC_ERR_CUDA", 3: "EBIC_ERR_OOM",
          4: "EBIC_ERR_TIMEOUT", 5: "EBIC_ERR_STATE", 6: "EBIC_ERR_CANCELLED",
          7: "EBIC_ERR_DEVICE"}


class EbicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("pop_size", ctypes.c_int32), ("len_min", ctypes.c_int32),
        ("len_max", ctypes.c_int32), ("iterations", ctypes.c_int32),
        ("sigma", ctypes.c_int32), ("toprank_size", ctypes.c_int32),
        ("tournament_k", ctypes.c_int32), ("support_mode", ctypes.c_int32),
        ("overlap_tau", ctypes.c_double), ("elite_frac", ctypes.c_double),
        ("penalty_base", ctypes.c_double), ("p_crossover", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("generations_done", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
        ("tabu_hits_total", ctypes.c_int64), ("attempts_total", ctypes.c_int64),
        ("evaluations_total", ctypes.c_int64), ("last_gen_hits", ctypes.c_int32),
        ("toprank_n", ctypes.c_int32), ("exact_tournaments", ctypes.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIGS = {
    "ebic_last_error": ([], ctypes.c_char_p),
    "ebic_abi_version": ([], _I32),
    "ebic_kernel_launches": ([], ctypes.c_uint64),
    "ebic_probe_read_bandwidth": ([_P, ctypes.c_uint64, _I32, _P, _P], _I32),
    "ebic_load_matrix": ([_P, _I32, _I32, _P], _I32),
    "ebic_load_matrix_dev": ([_P, _I32, _I32, _P, _P], _I32),
    "ebic_free": ([_P], None),
    "ebic_matrix_shape": ([_P, _P, _P], _I32),
    "ebic_build_pair_table": ([_P, _P], _I32),
    "ebic_pair_table_bytes": ([_P, _P, _P], _I32),
    "ebic_read_pair_words": ([_P, _I32, _I32, _I32, _I32, _P], _I32),
    "ebic_set_path": ([_P, _I32], _I32),
    "ebic_set_eval_tuning": ([_P, _P], _I32),
    "ebic_get_eval_tuning": ([_P, _P], _I32),
    "ebic_autotune_eval": ([_P, _P, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P, _I32, _P, _P],
                           _I32),
    "ebic_eval_population": ([_P, _P, _P, _I32, _I32, _I32, _P, _P, _P], _I32),
    "ebic_eval_population_dev": ([_P, _P, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P], _I32),
    "ebic_check_device_error": ([_P], _I32),
    "ebic_eval_population_dev_noalloc": ([_P, _P, _P, _I32, _I32, _I32, _P, _P, _P], _I32),
    "ebic_default_params": ([_P], None),
    "ebic_batch_create": ([_P, _P, _I32, _I32, _P, _P], _I32),
    "ebic_batch_eval": ([_P, _P], _I32),
    "ebic_batch_describe": ([_P, _I32, _P, _P, _P, _P, _P], _I32),
    "ebic_batch_free": ([_P], None),
    "ebic_run_init": ([_P, _P], _I32),
    "ebic_run_step": ([_P, _I32, _P], _I32),
    "ebic_run_step_async": ([_P, _I32, _P], _I32),
    "ebic_run_step_profiled": ([_P, _P], _I32),
    "ebic_set_kernel_timing": ([_P, _I32], _I32),
    "ebic_read_kernel_timing": ([_P, _I32, _P, _P], _I32),
    "ebic_get_toprank": ([_P, _P, _P, _P, _P, _P], _I32),
    "ebic_get_population": ([_P, _P, _P, _P, _P, _P, _P], _I32),
    "ebic_run_generations": ([_P, _P, _P, _P, _P, _P, _P], _I32),
    "ebic_surrogate_create": ([_P, _I32, ctypes.c_uint64, _P], _I32),
    "ebic_surrogate_free": ([_P], _I32),
    "ebic_surrogate_params": ([_P, _P, _P, _I32], _I32),
    "ebic_surrogate_grads": ([_P, _P, ctypes.c_int64], _I32),
    "ebic_surrogate_colstats": ([_P, _P, _P], _I32),
    "ebic_surrogate_step": ([_P, _P, _P, _I32, _P, _P, _I32, ctypes.c_float, _I32, _P], _I32),
    "ebic_surrogate_log": ([_P, _P, _P], _I32),
    "ebic_surrogate_train": ([_P, _P, _P, _I32, _P, ctypes.c_int64, _I32, _I32, ctypes.c_float,
                              _P], _I32),
    "ebic_surrogate_target_norm": ([_P, _P, _P], _I32),
    "ebic_surrogate_predict": ([_P, _P, _P, _I32, ctypes.c_int64, _P, _P], _I32),
    "ebic_surrogate_forward_kernel": ([_P, _I32], _I32),
    "ebic_surrogate_train_kernel": ([_P, _I32], _I32),
    "ebic_run_screen": ([_P, _P, _I32, _I32], _I32),
    "ebic_extract_rows": ([_P, _P, _P, _I32, _I32, _P, _P, _P], _I32),
    "ebic_extract_rows_approx": ([_P, _P, _P, _I32, _I32, _I32, _P, _P, _P], _I32),
    "ebic_recovery_relevance": ([_I32, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P], _I32),
}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (no-op when up to date)."""
    return _build.build(force=force)


def lib():
    """The loaded ``libebic.so``.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(
                    "libebic.so is missing: the CUDA library must be built (build()); "
                    "there is no CPU fallback")
            L = ctypes.CDLL(_build.LIB)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise EbicError(status, lib().ebic_last_error().decode(errors="replace"))


def _host(a, dtype):
    """A contiguous array of `dtype` and its address (a plain int, which the
    c_void_p argument types take as is and which is cheaper to get than a
    ctypes pointer object)."""
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _dev(x):
    """Device pointer of a torch CUDA tensor (or an int / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if not getattr(x, "is_cuda", False):
        raise TypeError("expected a CUDA tensor for a device buffer")
    if not x.is_contiguous():
        raise ValueError("device buffers must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
def ebic_load_matrix(A) -> ctypes.c_void_p:
    A, p = _host(A, np.float32)
    if A.ndim != 2:
        raise ValueError("A must be 2-D (rows x cols)")
    h = ctypes.c_void_p()
    _check(lib().ebic_load_matrix(p, A.shape[0], A.shape[1], ctypes.byref(h)))
    return h


def ebic_load_matrix_dev(A, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().ebic_load_matrix_dev(_dev(A), A.shape[0], A.shape[1], _stream(stream),
                                      ctypes.byref(h)))
    return h


def ebic_kernel_launches() -> int:
    return int(lib().ebic_kernel_launches())


def ebic_probe_read_bandwidth(d_buf, nbytes: int, reps: int = 20, stream=None) -> float:
    """Fastest of `reps` timed read passes over a device buffer, in us."""
    us = ctypes.c_float()
    _check(lib().ebic_probe_read_bandwidth(_dev(d_buf), int(nbytes), int(reps), _stream(stream),
                                           ctypes.byref(us)))
    return us.value


def ebic_free(h):
    if h is not None and h.value:
        lib().ebic_free(h)
        h.value = None


def ebic_matrix_shape(h):
    r, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().ebic_matrix_shape(h, ctypes.byref(r), ctypes.byref(c)))
    return r.value, c.value


def ebic_build_pair_table(h, stream=None):
    _check(lib().ebic_build_pair_table(h, _stream(stream)))


def ebic_pair_table_bytes(h):
    b, built = ctypes.c_uint64(), ctypes.c_int32()
    _check(lib().ebic_pair_table_bytes(h, ctypes.byref(b), ctypes.byref(built)))
    return b.value, bool(built.value)


def ebic_read_pair_words(h, p, q, w0, n):
    out = np.zeros(n, np.uint32)
    _check(lib().ebic_read_pair_words(h, p, q, w0, n, out.ctypes.data))
    return out


def ebic_set_path(h, path: int):
    _check(lib().ebic_set_path(h, path))


class EvalTuning(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("vecs_per_part_bitmask", ctypes.c_int32),
                ("vecs_per_part_gather", ctypes.c_int32), ("batch_steps", ctypes.c_int32),
                ("vecs_per_lane", ctypes.c_int32), ("dense_steps", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("dynamic_rounds", ctypes.c_int32)]


def ebic_set_eval_tuning(h, kernel: int = 0, vecs_per_part_bitmask: int = 0,
                         vecs_per_part_gather: int = 0, batch_steps: int = 0,
                         vecs_per_lane: int = 0, dense_steps: int = 0, stages: int = 0,
                         groups: int = 0, dynamic_rounds: int = 0):
    t = EvalTuning(kernel, vecs_per_part_bitmask, vecs_per_part_gather, batch_steps,
                   vecs_per_lane, dense_steps, stages, groups, dynamic_rounds)
    _check(lib().ebic_set_eval_tuning(h, ctypes.byref(t)))


def ebic_get_eval_tuning(h) -> dict:
    t = EvalTuning()
    _check(lib().ebic_get_eval_tuning(h, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in EvalTuning._fields_}


TUNE_COLD_L2 = 1


def ebic_autotune_eval(h, d_offsets, d_cols, P: int, total_cols: int, sigma: int,
                       support_mode: int, d_inc, d_dec, d_fitness, stream=None, flags: int = 0):
    """Times launch shapes on this device population; returns (shape dict, us).
    flags=TUNE_COLD_L2 times every launch with the L2 emptied first."""
    t = EvalTuning()
    us = ctypes.c_float()
    _check(lib().ebic_autotune_eval(h, _dev(d_offsets), _dev(d_cols), int(P), int(total_cols),
                                    int(sigma), int(support_mode), _dev(d_inc), _dev(d_dec),
                                    _dev(d_fitness), _stream(stream), int(flags), ctypes.byref(t),
                                    ctypes.byref(us)))
    return {f: getattr(t, f) for f, _ in EvalTuning._fields_}, us.value


def ebic_eval_population(h, offsets, cols, sigma: int, support_mode: int = SUPPORT_INC,
                         want_dec: bool = True):
    """Host-buffer evaluation.  Returns (inc, dec or None, fitness)."""
    off, po = _host(offsets, np.int32)
    cl, pc = _host(cols, np.int32)
    P = off.shape[0] - 1
    inc = np.empty(P, np.uint32)
    dec = np.empty(P, np.uint32) if want_dec else None
    fit = np.empty(P, np.float64)
    _check(lib().ebic_eval_population(
        h, po, pc, P, int(sigma), int(support_mode), inc.ctypes.data,
        dec.ctypes.data if dec is not None else None, fit.ctypes.data))
    return inc, dec, fit


def ebic_eval_population_dev(h, d_offsets, d_cols, P: int, total_cols: int, sigma: int,
                             support_mode: int, d_inc, d_dec, d_fitness, stream=None):
    """Device-buffer evaluation, queued on ``stream`` (torch stream or handle)."""
    _check(lib().ebic_eval_population_dev(h, _dev(d_offsets), _dev(d_cols), int(P),
                                          int(total_cols), int(sigma), int(support_mode),
                                          _dev(d_inc), _dev(d_dec), _dev(d_fitness),
                                          _stream(stream)))


def ebic_eval_population_dev_noalloc(h, d_offsets, d_cols, P: int, total_cols: int,
                                     sigma: int, d_inc, d_fitness, stream=None):
    """Rising support and Eq. (1) on device buffers without any allocation by
    the library (fixed static scratch; see include/ebic.h)."""
    _check(lib().ebic_eval_population_dev_noalloc(h, _dev(d_offsets), _dev(d_cols), int(P),
                                                  int(total_cols), int(sigma), _dev(d_inc),
                                                  _dev(d_fitness), _stream(stream)))


def ebic_check_device_error(h):
    _check(lib().ebic_check_device_error(h))


BATCH_AUTOTUNE, BATCH_GRAPH, BATCH_BUILD_TABLES = 1, 2, 4


class BatchItem(ctypes.Structure):
    _fields_ = [("d_offsets", ctypes.c_void_p), ("d_cols", ctypes.c_void_p),
                ("P", ctypes.c_int32), ("total_cols", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("d_inc", ctypes.c_void_p), ("d_fitness", ctypes.c_void_p)]


def ebic_batch_create(handles, items, flags: int, stream=None):
    """items: sequence of (d_offsets, d_cols, P, total_cols, sigma, d_inc, d_fitness)
    with torch CUDA tensors for the device buffers.  Returns the batch handle."""
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value for h in handles])
    arr = (BatchItem * n)()
    for k, (off, cols, P, total, sigma, inc, fit) in enumerate(items):
        arr[k] = BatchItem(_dev(off).value, _dev(cols).value, int(P), int(total), int(sigma),
                           _dev(inc).value, _dev(fit).value)
    b = ctypes.c_void_p()
    _check(lib().ebic_batch_create(H, arr, n, int(flags), _stream(stream), ctypes.byref(b)))
    return b


def ebic_batch_eval(b, stream=None):
    _check(lib().ebic_batch_eval(b, _stream(stream)))


def ebic_batch_describe(b, problem: int) -> dict:
    path, vpp, parts, grid = (ctypes.c_int32() for _ in range(4))
    items = ctypes.c_int64()
    _check(lib().ebic_batch_describe(b, int(problem), ctypes.byref(path), ctypes.byref(vpp),
                                     ctypes.byref(parts), ctypes.byref(items),
                                     ctypes.byref(grid)))
    return dict(path=path.value, vecs_per_part=vpp.value, parts=parts.value,
                work_items=items.value, grid=grid.value)


def ebic_batch_free(b):
    if b is not None and b.value:
        lib().ebic_batch_free(b)
        b.value = None


def ebic_default_params(**overrides) -> Params:
    p = Params()
    lib().ebic_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def ebic_run_init(h, params: Params):
    _check(lib().ebic_run_init(h, ctypes.byref(params)))


def ebic_run_step(h, generations: int) -> dict:
    st = Stats()
    _check(lib().ebic_run_step(h, int(generations), ctypes.byref(st)))
    return st.as_dict()


def ebic_run_step_async(h, generations: int, stream=None):
    _check(lib().ebic_run_step_async(h, int(generations), _stream(stream)))


KERNELS = ("k_spec", "k_build", "k_tabu_insert", "eval", "k_rank",
           "screen_candidates", "screen_scores", "screen_pick")


def ebic_run_step_profiled(h) -> dict:
    us = (ctypes.c_float * 8)()
    _check(lib().ebic_run_step_profiled(h, us))
    out = dict(zip(KERNELS, list(us)))
    if not any(out[k] for k in KERNELS[5:]):          # no screening
        for k in KERNELS[5:]:
            out.pop(k)
    return out


def ebic_set_kernel_timing(h, slots: int) -> None:
    _check(lib().ebic_set_kernel_timing(h, int(slots)))


def ebic_read_kernel_timing(h, reset: bool = False):
    """(mean k_build microseconds, replays covered) of the in-graph timing."""
    us, n = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().ebic_read_kernel_timing(h, int(bool(reset)), ctypes.byref(us), ctypes.byref(n)))
    return us.value, n.value


def _records(off, cols, n):
    return [cols[off[i]:off[i + 1]].tolist() for i in range(n)]


def ebic_get_toprank(h, capacity: int, len_max: int):
    off = np.zeros(capacity + 1, np.int32)
    cols = np.zeros(max(1, capacity * len_max), np.int32)
    fit = np.zeros(max(1, capacity), np.float64)
    inc = np.zeros(max(1, capacity), np.uint32)
    n = ctypes.c_int32(capacity)
    _check(lib().ebic_get_toprank(h, off.ctypes.data, cols.ctypes.data,
                                  fit.ctypes.data, inc.ctypes.data,
                                  ctypes.byref(n)))
    k = n.value
    return _records(off, cols, k), fit[:k].copy(), inc[:k].copy()


def ebic_get_population(h, capacity: int, len_max: int):
    off = np.zeros(capacity + 1, np.int32)
    cols = np.zeros(max(1, capacity * len_max), np.int32)
    inc = np.zeros(max(1, capacity), np.uint32)
    dec = np.zeros(max(1, capacity), np.uint32)
    fit = np.zeros(max(1, capacity), np.float64)
    n = ctypes.c_int32(capacity)
    _check(lib().ebic_get_population(h, off.ctypes.data, cols.ctypes.data,
                                     inc.ctypes.data, dec.ctypes.data,
                                     fit.ctypes.data, ctypes.byref(n)))
    k = n.value
    return dict(seqs=_records(off, cols, k), inc=inc[:k].copy(), dec=dec[:k].copy(),
                f=fit[:k].copy())


def ebic_run_generations(h, params: Params, capacity: int | None = None):
    """Steps 1-5 for params.iterations generations; returns (toprank, fitness, stats)."""
    cap = params.toprank_size if capacity is None else capacity
    off = np.zeros(cap + 1, np.int32)
    cols = np.zeros(max(1, cap * params.len_max), np.int32)
    fit = np.zeros(max(1, cap), np.float64)
    n = ctypes.c_int32(cap)
    st = Stats()
    _check(lib().ebic_run_generations(h, ctypes.byref(params), off.ctypes.data,
                                      cols.ctypes.data, fit.ctypes.data,
                                      ctypes.byref(n), ctypes.byref(st)))
    k = n.value
    return _records(off, cols, k), fit[:k].copy(), st.as_dict()


# ---------------------------------------------------------------------------
# Fitness surrogate and offspring screening (no counterpart in the paper)
SUR_F, SUR_EMB, SUR_H = 80, 64, 256


def ebic_surrogate_create(h, len_scale: int = 64, seed: int = 0) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(lib().ebic_surrogate_create(h, int(len_scale), int(seed), ctypes.byref(out)))
    return out


def ebic_surrogate_free(s):
    _check(lib().ebic_surrogate_free(s))


def ebic_surrogate_params(s, values=None) -> np.ndarray:
    """Reads the flat fp32 parameters, or replaces them with `values`."""
    n = ctypes.c_int64(0)
    _check(lib().ebic_surrogate_params(s, None, ctypes.byref(n), 0))
    if values is None:
        out = np.zeros(n.value, np.float32)
        _check(lib().ebic_surrogate_params(s, out.ctypes.data, ctypes.byref(n), 0))
        return out
    v, p = _host(values, np.float32)
    if v.size != n.value:
        raise ValueError(f"expected {n.value} parameters, got {v.size}")
    _check(lib().ebic_surrogate_params(s, p, ctypes.byref(n), 1))
    return v


def ebic_surrogate_split(flat: np.ndarray, C: int) -> dict:
    """Views of the flat parameter vector by name (Emb, W1, b1, W2, b2, w3, b3)."""
    shapes = [("Emb", (C, SUR_EMB)), ("W1", (SUR_F, SUR_H)), ("b1", (SUR_H,)),
              ("W2", (SUR_H, SUR_H)), ("b2", (SUR_H,)), ("w3", (SUR_H,)), ("b3", ())]
    out, o = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp)) if shp else 1
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def ebic_surrogate_grads(s) -> np.ndarray:
    n = ctypes.c_int64(0)
    _check(lib().ebic_surrogate_params(s, None, ctypes.byref(n), 0))
    out = np.zeros(n.value, np.float32)
    _check(lib().ebic_surrogate_grads(s, out.ctypes.data, n.value))
    return out


def ebic_surrogate_colstats(s, C: int):
    m = np.zeros(C, np.float32)
    d = np.zeros(C, np.float32)
    _check(lib().ebic_surrogate_colstats(s, m.ctypes.data, d.ctypes.data))
    return m, d


def ebic_surrogate_step(s, d_seq, d_len, stride: int, d_target, batch: int, lr: float = 0.0,
                        update: bool = False, d_idx=None) -> float:
    loss = ctypes.c_float(0)
    _check(lib().ebic_surrogate_step(s, _dev(d_seq), _dev(d_len), int(stride), _dev(d_target),
                                     _dev(d_idx), int(batch), float(lr), int(bool(update)),
                                     ctypes.byref(loss)))
    return loss.value


def ebic_surrogate_log(s, h) -> int:
    n = ctypes.c_int64(0)
    _check(lib().ebic_surrogate_log(s, h, ctypes.byref(n)))
    return n.value


def ebic_surrogate_train(s, steps: int, batch: int, lr: float, d_seq=None, d_len=None,
                         stride: int = 0, d_fitness=None, n: int = 0) -> float:
    """Adam steps on device pairs (or on the log when no arrays are given)."""
    loss = ctypes.c_float(0)
    _check(lib().ebic_surrogate_train(s, _dev(d_seq), _dev(d_len), int(stride), _dev(d_fitness),
                                      int(n), int(steps), int(batch), float(lr),
                                      ctypes.byref(loss)))
    return loss.value


def ebic_surrogate_target_norm(s):
    m, d = ctypes.c_float(0), ctypes.c_float(0)
    _check(lib().ebic_surrogate_target_norm(s, ctypes.byref(m), ctypes.byref(d)))
    return m.value, d.value


FORWARD_TCGEN05, FORWARD_MMA_SYNC = 0, 1


def ebic_surrogate_forward_kernel(s, kind: int):
    """Scoring kernel: FORWARD_TCGEN05 (default) or FORWARD_MMA_SYNC."""
    _check(lib().ebic_surrogate_forward_kernel(s, int(kind)))


def ebic_surrogate_train_kernel(s, kind: int):
    """Training GEMMs: FORWARD_TCGEN05 (default) or FORWARD_MMA_SYNC."""
    _check(lib().ebic_surrogate_train_kernel(s, int(kind)))


def ebic_surrogate_predict(s, d_seq, d_len, stride: int, n: int, d_out, stream=None):
    _check(lib().ebic_surrogate_predict(s, _dev(d_seq), _dev(d_len), int(stride), int(n),
                                        _dev(d_out), _stream(stream)))


def ebic_run_screen(h, s=None, oversample: int = 1, mode: int = SCREEN_OFF):
    _check(lib().ebic_run_screen(h, s, int(oversample), int(mode)))


# ---------------------------------------------------------------------------
# Step 6 rows and Step 7 negative-trend expansion; Eq. (2)-(3)
def _extract(call, offsets, cols):
    """Two calls of a rows entry point: the first sizes the buffer."""
    off, po = _host(offsets, np.int32)
    c, pc = _host(cols, np.int32)
    P = len(off) - 1
    roff = np.zeros(P + 1, np.int64)
    cap = ctypes.c_int64(0)
    st = call(po, pc, P, roff.ctypes.data, None, ctypes.byref(cap))
    if st != 0 and cap.value == 0 and P > 0:
        _check(st)
    rows = np.zeros(max(1, cap.value), np.int32)
    _check(call(po, pc, P, roff.ctypes.data, rows.ctypes.data, ctypes.byref(cap)))
    return [rows[roff[i]:roff[i + 1]].copy() for i in range(P)]


def ebic_extract_rows(h, offsets, cols, mode: int = ROWS_RISING):
    """Rows matching each series of a CBF population: list of int32 arrays."""
    return _extract(lambda po, pc, P, ro, rw, cap: lib().ebic_extract_rows(
        h, po, pc, P, int(mode), ro, rw, cap), offsets, cols)


def ebic_extract_rows_approx(h, offsets, cols, max_breaks: int, mode: int = ROWS_RISING):
    """Rows following each series with at most max_breaks broken adjacent
    pairs (Step 7 by approximate trends): list of int32 arrays."""
    return _extract(lambda po, pc, P, ro, rw, cap: lib().ebic_extract_rows_approx(
        h, po, pc, P, int(max_breaks), int(mode), ro, rw, cap), offsets, cols)


def _csr(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    for i, x in enumerate(lists):
        off[i + 1] = off[i] + len(x)
    v = np.concatenate([np.asarray(x, np.int32) for x in lists]) if lists else np.zeros(0, np.int32)
    return off, np.ascontiguousarray(v if len(v) else np.zeros(1, np.int32), np.int32)


def ebic_recovery_relevance(expected, found, want_jaccard: bool = False):
    """expected / found: lists of (rows, cols) with ascending distinct indices."""
    E, F = len(expected), len(found)
    er, ev = _csr([e[0] for e in expected])
    ec, ecv = _csr([e[1] for e in expected])
    fr, fv = _csr([f[0] for f in found])
    fc, fcv = _csr([f[1] for f in found])
    rec, rel = ctypes.c_double(0), ctypes.c_double(0)
    J = np.zeros(max(1, E * F), np.float64)
    p = lambda a: a.ctypes.data
    _check(lib().ebic_recovery_relevance(E, p(er), p(ev), p(ec), p(ecv), F, p(fr), p(fv), p(fc),
                                         p(fcv), ctypes.byref(rec), ctypes.byref(rel),
                                         p(J) if want_jaccard else None))
    if want_jaccard:
        return rec.value, rel.value, J[:E * F].reshape(E, F)
    return rec.value, rel.value
