"""Parity of the multi-problem persistent launch with the oracle: every
problem's counts and fitness, bit for bit, on repeated evaluations (graph
replay and self-resetting split scratch)."""
import numpy as np
import pytest

import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth
from helpers import assert_bits_equal, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    eb.build()
    return t


def _setup(torch, items):
    dev = torch.device("cuda:0")
    handles, bitems, outs = [], [], []
    for it in items:
        h = eb.ebic_load_matrix(it.problem.A)
        P = len(it.offsets) - 1
        inc = torch.full((P,), -1, dtype=torch.int32, device=dev)
        fit = torch.full((P,), -1.0, dtype=torch.float64, device=dev)
        off = torch.from_numpy(it.offsets).to(dev)
        cols = torch.from_numpy(it.cols).to(dev)
        handles.append(h)
        outs.append((inc, fit, off, cols))
        bitems.append((off, cols, P, len(it.cols), it.problem.sigma, inc, fit))
    return handles, bitems, outs


@pytest.mark.parametrize("flags", [eb.BATCH_BUILD_TABLES | eb.BATCH_AUTOTUNE | eb.BATCH_GRAPH,
                                   eb.BATCH_GRAPH])
def test_small_batch_full_parity(torch, flags):
    items = synth.batch_uneven(seed=3, n=12, rows=(200, 8000), cols=(8, 120), pop=(50, 400),
                               max_len=12)
    handles, bitems, outs = _setup(torch, items)
    try:
        b = eb.ebic_batch_create(handles, bitems, flags)
        try:
            for rep in range(3):
                for inc, fit, _, _ in outs:
                    inc.fill_(-1)
                    fit.fill_(-1.0)
                eb.ebic_batch_eval(b)
                torch.cuda.synchronize()
                for k, it in enumerate(items):
                    eb.ebic_check_device_error(handles[k])
                    oinc, _, ofit = oracle_eval(it.problem.A, it.offsets, it.cols,
                                                it.problem.sigma)
                    inc, fit = outs[k][0], outs[k][1]
                    assert_bits_equal(inc.cpu().numpy().view(np.uint32), oinc, f"inc p{k} r{rep}")
                    assert_bits_equal(fit.cpu().numpy(), ofit, f"fit p{k} r{rep}")
            descr = [eb.ebic_batch_describe(b, k) for k in range(len(items))]
            assert all(d["work_items"] > 0 and d["grid"] > 0 for d in descr)
        finally:
            eb.ebic_batch_free(b)
    finally:
        for h in handles:
            eb.ebic_free(h)


def test_uneven_64_problem_batch_full_parity(torch):
    # the full-size uneven batch: 64 problems of 500-50,000 rows and 20-500
    # columns with 256-2,048 series each, every series of every problem
    # against the oracle (about 20 s of oracle time)
    items = synth.batch_uneven(seed=0, n=64)
    handles, bitems, outs = _setup(torch, items)
    try:
        b = eb.ebic_batch_create(handles, bitems, eb.BATCH_BUILD_TABLES | eb.BATCH_AUTOTUNE |
                                 eb.BATCH_GRAPH)
        try:
            for rep in range(2):
                eb.ebic_batch_eval(b)
                torch.cuda.synchronize()
            for k, it in enumerate(items):
                eb.ebic_check_device_error(handles[k])
                oinc, _, ofit = oracle_eval(it.problem.A, it.offsets, it.cols, it.problem.sigma)
                inc = outs[k][0].cpu().numpy().view(np.uint32)
                fit = outs[k][1].cpu().numpy()
                assert_bits_equal(inc, oinc, f"inc problem {k}")
                assert_bits_equal(fit, ofit, f"fit problem {k}")
        finally:
            eb.ebic_batch_free(b)
    finally:
        for h in handles:
            eb.ebic_free(h)
