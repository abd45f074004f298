"""The evaluation entry point that allocates nothing, for callers whose device
memory is owned by someone else (a framework's pool) or who cannot take the
synchronisation an allocation may bring.  It must give the same rising
counts and fitness as the regular device entry point, call after call, while
its per-series scratch lives in a fixed static array shared by all calls."""
import numpy as np
import pytest

import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth
from helpers import assert_bits_equal, oracle_eval

pytestmark = pytest.mark.gpu

NOALLOC_MAX_SERIES = 65536     # EBIC_NOALLOC_MAX_SERIES in include/ebic.h


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    eb.build()
    return t


@pytest.mark.parametrize("use_table", [False, True])
def test_matches_the_regular_entry_point_on_two_calls(torch, use_table):
    # few series over many rows: every series is split across warps, so the
    # partial counts go through the static scratch array
    prob = synth.matrix_random(21, 30000, 40, n_plants=3, plant_rows=(1500, 3000),
                               plant_cols=(3, 8))
    off, cols = synth.population(22, 50, 40, 2, 12, plants=prob.plants)
    P, sigma = len(off) - 1, 300
    dev = torch.device("cuda:0")
    h = eb.ebic_load_matrix(prob.A)
    try:
        if use_table:
            eb.ebic_build_pair_table(h)
        d_off = torch.from_numpy(off).to(dev)
        d_cols = torch.from_numpy(cols).to(dev)
        want_inc = torch.zeros(P, dtype=torch.int32, device=dev)
        want_fit = torch.zeros(P, dtype=torch.float64, device=dev)
        eb.ebic_eval_population_dev(h, d_off, d_cols, P, len(cols), sigma, eb.SUPPORT_INC,
                                    want_inc, None, want_fit)
        torch.cuda.synchronize()
        for call in range(2):
            inc = torch.full((P,), -1, dtype=torch.int32, device=dev)
            fit = torch.full((P,), -1.0, dtype=torch.float64, device=dev)
            eb.ebic_eval_population_dev_noalloc(h, d_off, d_cols, P, len(cols), sigma, inc, fit)
            torch.cuda.synchronize()
            eb.ebic_check_device_error(h)
            assert torch.equal(inc, want_inc), f"call {call}: counts differ"
            assert np.array_equal(fit.cpu().numpy().view(np.uint64),
                                  want_fit.cpu().numpy().view(np.uint64)), f"call {call}: fitness"
        assert int(want_inc.max()) >= 1500          # the planted series were counted
        # and both equal the oracle's counts and Eq. (1) values
        oinc, _, ofit = oracle_eval(prob.A, off, cols, sigma)
        assert_bits_equal(inc.cpu().numpy().view(np.uint32), oinc, "inc vs oracle")
        assert_bits_equal(fit.cpu().numpy(), ofit, "fitness vs oracle")
    finally:
        eb.ebic_free(h)


def test_rejects_more_series_than_its_scratch_holds(torch):
    A = np.random.default_rng(0).standard_normal((100, 5)).astype(np.float32)
    dev = torch.device("cuda:0")
    h = eb.ebic_load_matrix(A)
    try:
        off = torch.zeros(2, dtype=torch.int32, device=dev)
        buf = torch.zeros(1, dtype=torch.int32, device=dev)
        fit = torch.zeros(1, dtype=torch.float64, device=dev)
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_eval_population_dev_noalloc(h, off, buf, NOALLOC_MAX_SERIES + 1, 0, 3, buf,
                                                fit)
        assert e.value.status == 1 and "EBIC_NOALLOC_MAX_SERIES" in str(e.value)
    finally:
        eb.ebic_free(h)
