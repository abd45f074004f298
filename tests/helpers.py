"""Shared helpers for the parity tests (CUDA path vs the oracle)."""
import os
import re

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    """Names of the functions declared in include/ebic.h."""
    text = open(os.path.join(ROOT, "include", "ebic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ebic_[a-z_0-9]+)\s*\(", text)))


def oracle_eval(A, off, cols, sigma, mode=0, nthreads=None):
    """Oracle support and Eq. (1) fitness for a CBF population."""
    nthreads = nthreads or oracle.omp_max_threads()
    inc, dec = oracle.support(A, off, cols, nthreads=nthreads)
    lens = np.diff(np.asarray(off))
    n = inc.astype(np.int64) + (dec.astype(np.int64) if mode == 1 else 0)
    fit = np.array([oracle.fitness(int(a), int(b), sigma) for a, b in zip(n, lens)], np.float64)
    return inc, dec, fit


def assert_bits_equal(got, want, what):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if got.dtype.kind == "f":
        assert got.dtype == want.dtype, (what, got.dtype, want.dtype)
        u = np.dtype(f"u{got.dtype.itemsize}")
        same = got.view(u) == want.view(u)
    else:
        same = got == want
    if not same.all():
        bad = np.flatnonzero(~same)[:8]
        raise AssertionError(f"{what}: {len(np.flatnonzero(~same))} mismatches, first at "
                             f"{bad.tolist()}: got {got[bad].tolist()} want {want[bad].tolist()}")
