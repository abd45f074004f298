"""Parity of the CUDA evaluation path (K1 placement, K2 pair table, K3 support
+ Eq. (1)) with the oracle, through the C ABI.  Counts and fitness must be
bit-identical: integers exactly, binary64 fitness bit for bit."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth
from helpers import assert_bits_equal, oracle_eval

pytestmark = pytest.mark.gpu

PATHS = [eb.PATH_GATHER, eb.PATH_BITMASK]


@pytest.fixture(scope="module", autouse=True)
def built():
    eb.build()
    yield


def _check(A, off, cols, sigma, path, mode=0, want_dec=True):
    h = eb.ebic_load_matrix(A)
    try:
        eb.ebic_set_path(h, path)
        inc, dec, fit = eb.ebic_eval_population(h, off, cols, sigma, mode, want_dec)
    finally:
        eb.ebic_free(h)
    oinc, odec, ofit = oracle_eval(A, off, cols, sigma, mode)
    assert_bits_equal(inc, oinc, "inc")
    if want_dec:
        assert_bits_equal(dec, odec, "dec")
    assert_bits_equal(fit, ofit, "fitness")
    return inc, dec, fit


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_200x20(path, mode):
    prob = synth.matrix_tiny(seed=0)
    off, cols = synth.population(0, 100, 20, 2, 6, plants=prob.plants)
    _check(prob.A, off, cols, 10, path, mode)


@pytest.mark.parametrize("path", PATHS)
def test_paper_1000x100(path):
    prob = synth.matrix_paper(seed=0)
    off, cols = synth.population(1, 600, 100, 3, 20, plants=prob.plants)
    inc, _, _ = _check(prob.A, off, cols, 25, path)
    assert inc.max() >= 50           # planted series are found


@pytest.mark.parametrize("path", PATHS)
def test_expression_20000x200_full(path):
    prob = synth.matrix_expression(seed=0)
    off, cols = synth.population(2, 4096, 200, 3, 30, plants=prob.plants)
    _check(prob.A, off, cols, 50, path, mode=1)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("R,C", [(1, 3), (31, 5), (33, 7), (127, 9), (129, 4), (1001, 13),
                                 (4097, 6), (5000, 40)])
def test_ragged_shapes(path, R, C):
    rng = np.random.default_rng(R * 100 + C)
    A = rng.standard_normal((R, C)).astype(np.float32)
    off, cols = synth.population(R + C, 300, C, 1, min(C, 8))
    _check(A, off, cols, 5, path, mode=1)


@pytest.mark.parametrize("path", PATHS)
def test_ties_nan_signed_zero(path):
    rng = np.random.default_rng(11)
    A = rng.integers(-2, 3, (700, 10)).astype(np.float32)
    A[rng.random(A.shape) < 0.05] = np.nan
    A[rng.random(A.shape) < 0.1] = -0.0
    off, cols = synth.population(3, 500, 10, 1, 6, duplicates=True)
    _check(A, off, cols, 7, path, mode=1)


@pytest.mark.parametrize("path", PATHS)
def test_single_column_duplicates_and_long_series(path):
    rng = np.random.default_rng(12)
    A = rng.standard_normal((300, 1100)).astype(np.float32)
    seqs = [[5], [5, 5], [0, 1, 0], list(range(1024)), rng.permutation(1100)[:1024].tolist(),
            list(range(1023, -1, -1)), [7] * 1024]
    off, cols = oracle.to_cbf(seqs)
    inc, dec, fit = _check(A, off, cols, 3, path, mode=1)
    assert inc[0] == dec[0] == 300 and inc[1] == dec[1] == 0 and inc[2] == 0


@pytest.mark.parametrize("path", PATHS)
def test_few_series_many_rows_split_into_parts(path):
    # Few series over many rows: each series is split across warps and the
    # last-arriving part writes Eq. (1).  Run twice (arrival counters reset).
    prob = synth.matrix_random(5, 60000, 12, n_plants=2, plant_rows=(3000, 6000),
                               plant_cols=(3, 6))
    off, cols = synth.population(4, 5, 12, 2, 5, plants=prob.plants, frac_planted=1.0)
    for _ in range(2):
        _check(prob.A, off, cols, 100, path, mode=1)


@pytest.mark.parametrize("path", PATHS)
def test_fitness_underflow_region(path):
    prob = synth.matrix_paper(seed=3)
    off, cols = synth.population(5, 600, 100, 2, 4, plants=prob.plants)
    for sigma in (1000, 1100, 1500, 3000):
        _check(prob.A, off, cols, sigma, path)


def test_empty_population():
    h = eb.ebic_load_matrix(np.zeros((10, 3), np.float32))
    inc, dec, fit = eb.ebic_eval_population(h, np.zeros(1, np.int32), np.zeros(0, np.int32), 3)
    assert len(inc) == len(fit) == 0
    eb.ebic_free(h)


def test_pair_table_words_match_numpy():
    rng = np.random.default_rng(13)
    R, C = 1000, 9
    A = rng.integers(-3, 4, (R, C)).astype(np.float32)
    A[rng.random(A.shape) < 0.03] = np.nan
    h = eb.ebic_load_matrix(A)
    eb.ebic_build_pair_table(h)
    nbytes, built = eb.ebic_pair_table_bytes(h)
    W = 1024 // 32
    assert built and nbytes == C * C * W * 4
    for p in range(C):
        for q in range(C):
            bits = np.zeros(W * 32, bool)
            bits[:R] = A[:, p] < A[:, q]
            # word 4b + i, bit l  <->  row 128 b + 4 l + i
            blk = bits.reshape(W // 4, 32, 4)                  # [b][l][i]
            want = np.zeros(W, np.uint64)
            for i in range(4):
                want[i::4] = (blk[:, :, i] * (1 << np.arange(32, dtype=np.uint64))).sum(1)
            want = want.astype(np.uint32)
            got = eb.ebic_read_pair_words(h, p, q, 0, W)
            assert np.array_equal(got, want), (p, q)
    eb.ebic_free(h)


@pytest.mark.parametrize("path", PATHS)
def test_device_buffers_on_a_torch_stream(path):
    torch = pytest.importorskip("torch")
    prob = synth.matrix_paper(seed=4)
    off, cols = synth.population(6, 600, 100, 3, 20, plants=prob.plants)
    dev = torch.device("cuda:0")
    s = torch.cuda.Stream()
    dA = torch.from_numpy(prob.A).to(dev)
    h = eb.ebic_load_matrix_dev(dA, stream=s)
    eb.ebic_set_path(h, path)
    d_off = torch.from_numpy(off).to(dev)
    d_cols = torch.from_numpy(cols).to(dev)
    d_inc = torch.zeros(600, dtype=torch.int32, device=dev)
    d_dec = torch.zeros(600, dtype=torch.int32, device=dev)
    d_fit = torch.zeros(600, dtype=torch.float64, device=dev)
    with torch.cuda.stream(s):
        eb.ebic_eval_population_dev(h, d_off, d_cols, 600, len(cols), 25, 0, d_inc, d_dec,
                                    d_fit, stream=s)
    s.synchronize()
    eb.ebic_check_device_error(h)
    oinc, odec, ofit = oracle_eval(prob.A, off, cols, 25)
    assert_bits_equal(d_inc.cpu().numpy().view(np.uint32), oinc, "inc")
    assert_bits_equal(d_dec.cpu().numpy().view(np.uint32), odec, "dec")
    assert_bits_equal(d_fit.cpu().numpy(), ofit, "fitness")
    eb.ebic_free(h)


def test_host_variant_rejects_invalid_cbf():
    A = np.random.default_rng(0).standard_normal((50, 4)).astype(np.float32)
    h = eb.ebic_load_matrix(A)
    for off, cols in [([0, 2], [0, 4]), ([0, 2], [-1, 1]), ([1, 3], [0, 1, 2]),
                      ([0, 0], []), ([0, 2, 1], [0, 1]), ([0, 2, 5], [0, 1, 2, 3, 9]),
                      ([0, 3, 2, 5], [0, 1, 2, 3, 1]), ([0, 1, 1, 3], [0, 1, 2]),
                      ([0, 2000], list(range(4)) * 500)]:
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_eval_population(h, np.array(off), np.array(cols), 3)
        assert e.value.status == 1
        eb.ebic_check_device_error(h)       # no device error left behind
    # a length check that runs beside the device work also leaves the
    # caller's buffers untouched
    off = np.array([0, 2, 2, 4], np.int32)
    cols = np.array([0, 1, 2, 3], np.int32)
    inc = np.full(3, 7, np.uint32)
    fit = np.full(3, 7.0)
    P_ = ctypes.c_void_p
    st = eb.lib().ebic_eval_population(h, off.ctypes.data_as(P_), cols.ctypes.data_as(P_), 3, 3, 0,
                                       inc.ctypes.data_as(P_), None, fit.ctypes.data_as(P_))
    assert st == 1 and b"series 1" in eb.lib().ebic_last_error()
    assert (inc == 7).all() and (fit == 7.0).all()
    eb.ebic_check_device_error(h)
    # column indices are checked while the device runs: a bad one leaves the
    # caller's buffers untouched and no device error behind
    off = np.array([0, 2, 4], np.int32)
    cols = np.array([0, 1, 2, 7], np.int32)
    inc = np.full(2, 7, np.uint32)
    dec = np.full(2, 7, np.uint32)
    fit = np.full(2, 7.0)
    P_ = ctypes.c_void_p
    st = eb.lib().ebic_eval_population(h, off.ctypes.data_as(P_), cols.ctypes.data_as(P_), 2, 3, 0,
                                       inc.ctypes.data_as(P_), dec.ctypes.data_as(P_),
                                       fit.ctypes.data_as(P_))
    assert st == 1
    assert (inc == 7).all() and (dec == 7).all() and (fit == 7.0).all()
    eb.ebic_check_device_error(h)
    cols[3] = 3
    oinc, odec, ofit = oracle_eval(A, off, cols, 3)
    ginc, gdec, gfit = eb.ebic_eval_population(h, off, cols, 3)
    assert_bits_equal(ginc, oinc, "inc")
    assert_bits_equal(gdec, odec, "dec")
    assert_bits_equal(gfit, ofit, "fitness")
    eb.ebic_free(h)


@pytest.mark.parametrize("path", PATHS)
def test_device_variant_flags_invalid_series(path):
    torch = pytest.importorskip("torch")
    A = np.random.default_rng(1).standard_normal((300, 6)).astype(np.float32)
    h = eb.ebic_load_matrix(A)
    eb.ebic_set_path(h, path)
    dev = torch.device("cuda:0")
    # series 1 has a column out of range; series 3 has offsets past the end
    off = torch.tensor([0, 2, 4, 6, 99], dtype=torch.int32, device=dev)
    cols = torch.tensor([0, 1, 2, 6, 3, 4], dtype=torch.int32, device=dev)
    inc = torch.full((4,), 7, dtype=torch.int32, device=dev)
    fit = torch.full((4,), 7.0, dtype=torch.float64, device=dev)
    eb.ebic_eval_population_dev(h, off, cols, 4, 6, 3, 0, inc, None, fit)
    with pytest.raises(eb.EbicError) as e:
        eb.ebic_check_device_error(h)
    assert e.value.status == 7
    got = inc.cpu().numpy()
    oinc, _, ofit = oracle_eval(A, np.array([0, 2, 4]), np.array([0, 1, 3, 4]), 3)
    assert got[1] == 0 and got[3] == 0 and fit.cpu().numpy()[1] == 0.0
    assert got[0] == oinc[0] and got[2] == oinc[1]
    eb.ebic_check_device_error(h)      # flag was cleared
    eb.ebic_free(h)


@pytest.mark.parametrize("shape", [(200, 20), (1000, 100), (4097, 30), (20000, 60)])
@pytest.mark.parametrize("tune", [dict(), dict(kernel=1), dict(kernel=2),
                                  dict(kernel=2, vecs_per_part_bitmask=32, vecs_per_part_gather=32),
                                  dict(kernel=2, batch_steps=4, vecs_per_lane=1),
                                  dict(kernel=2, batch_steps=8, vecs_per_lane=1),
                                  dict(kernel=2, batch_steps=4, vecs_per_lane=2),
                                  dict(kernel=2, batch_steps=8, vecs_per_lane=2),
                                  dict(kernel=2, batch_steps=4, vecs_per_lane=4,
                                       vecs_per_part_bitmask=64),
                                  dict(kernel=3), dict(kernel=3, dense_steps=2, stages=2),
                                  dict(kernel=4), dict(kernel=4, dense_steps=2, stages=2)])
def test_launch_shapes_do_not_change_results(shape, tune):
    # lane-per-vector kernel, warp kernel, and forced splits of each series
    R, C = shape
    prob = synth.matrix_random(R + C, R, C, n_plants=3, plant_rows=(R // 20, R // 8),
                               plant_cols=(3, 8))
    off, cols = synth.population(R, 257, C, 2, 12, plants=prob.plants)
    oinc, odec, ofit = oracle_eval(prob.A, off, cols, max(10, R // 100), 1)
    h = eb.ebic_load_matrix(prob.A)
    try:
        for path in PATHS:
            eb.ebic_set_path(h, path)
            eb.ebic_set_eval_tuning(h, **tune)
            for mode in (0, 1):
                inc, dec, fit = eb.ebic_eval_population(h, off, cols, max(10, R // 100), mode,
                                                        want_dec=(mode == 1))
                eb.ebic_check_device_error(h)
                assert_bits_equal(inc, oinc, f"inc {path} {tune}")
                if mode == 1:
                    assert_bits_equal(dec, odec, f"dec {path} {tune}")
                    assert_bits_equal(fit, ofit, f"fit {path} {tune}")
    finally:
        eb.ebic_free(h)


@pytest.mark.parametrize("kernel,batch_steps,nv", [(2, 4, 1), (2, 8, 1), (2, 4, 2), (2, 8, 2),
                                                   (2, 4, 4)])
def test_long_series_batches(kernel, batch_steps, nv):
    """Series of 30-45 columns: several 32-step windows per series."""
    R, C = 3000, 60
    prob = synth.matrix_random(7, R, C, n_plants=2, plant_rows=(300, 600), plant_cols=(40, 50))
    off, cols = synth.population(8, 300, C, 30, 45, plants=prob.plants)
    oinc, _, ofit = oracle_eval(prob.A, off, cols, 30)
    h = eb.ebic_load_matrix(prob.A)
    try:
        eb.ebic_set_path(h, eb.PATH_BITMASK)
        eb.ebic_set_eval_tuning(h, kernel=kernel, batch_steps=batch_steps, vecs_per_lane=nv)
        inc, _, fit = eb.ebic_eval_population(h, off, cols, 30)
        assert_bits_equal(inc, oinc, "inc")
        assert_bits_equal(fit, ofit, "fit")
        assert (oinc > 0).sum() > 10      # planted series survive all windows
    finally:
        eb.ebic_free(h)


def test_autotuner_rejects_unknown_flags():
    torch = pytest.importorskip("torch")
    prob = synth.matrix_tiny(seed=0)
    off, cols = synth.population(0, 10, 20, 2, 6)
    dev = torch.device("cuda:0")
    h = eb.ebic_load_matrix(prob.A)
    try:
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_autotune_eval(h, torch.from_numpy(off).to(dev), torch.from_numpy(cols).to(dev),
                                  10, len(cols), 10, 0, torch.zeros(10, dtype=torch.int32, device=dev),
                                  None, torch.zeros(10, dtype=torch.float64, device=dev), flags=2)
        assert e.value.status == 1
    finally:
        eb.ebic_free(h)


def test_tuning_rejects_bad_batch():
    prob = synth.matrix_tiny(seed=0)
    h = eb.ebic_load_matrix(prob.A)
    try:
        with pytest.raises(eb.EbicError):
            eb.ebic_set_eval_tuning(h, kernel=2, batch_steps=8, vecs_per_lane=4)
        with pytest.raises(eb.EbicError):
            eb.ebic_set_eval_tuning(h, kernel=2, batch_steps=12)
        with pytest.raises(eb.EbicError):
            eb.ebic_set_eval_tuning(h, kernel=5)
    finally:
        eb.ebic_free(h)


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("which", ["paper", "expression"])
def test_autotuner_keeps_results_exact(which, flags):
    torch = pytest.importorskip("torch")
    if which == "paper":
        prob, P, lo, hi, sig = synth.matrix_paper(seed=7), 600, 3, 20, 25
    else:
        prob, P, lo, hi, sig = synth.matrix_expression(seed=7), 4096, 3, 30, 50
    off, cols = synth.population(8, P, prob.A.shape[1], lo, hi, plants=prob.plants)
    oinc, _, ofit = oracle_eval(prob.A, off, cols, sig)
    dev = torch.device("cuda:0")
    h = eb.ebic_load_matrix(prob.A)
    try:
        for path in PATHS:
            eb.ebic_set_path(h, path)
            d_off = torch.from_numpy(off).to(dev)
            d_cols = torch.from_numpy(cols).to(dev)
            inc = torch.zeros(P, dtype=torch.int32, device=dev)
            fit = torch.zeros(P, dtype=torch.float64, device=dev)
            shape, us = eb.ebic_autotune_eval(h, d_off, d_cols, P, len(cols), sig, 0, inc, None,
                                              fit, flags=flags)
            assert us > 0 and shape == eb.ebic_get_eval_tuning(h)
            assert_bits_equal(inc.cpu().numpy().view(np.uint32), oinc, f"inc {path}")
            assert_bits_equal(fit.cpu().numpy(), ofit, f"fit {path}")
            inc2, _, fit2 = eb.ebic_eval_population(h, off, cols, sig)
            assert_bits_equal(inc2, oinc, "inc after tuning")
            assert_bits_equal(fit2, ofit, "fit after tuning")
    finally:
        eb.ebic_free(h)


# ---------------------------------------------------------------------------
# The staged kernel (launch shape kernel 3): dense AND steps brought into
# shared memory by bulk copies, the rest by per-vector loads.  Rising counts.
# ---------------------------------------------------------------------------
STAGED = [dict(kernel=3), dict(kernel=3, dense_steps=1, stages=2),
          dict(kernel=3, dense_steps=8, stages=4, groups=1),
          dict(kernel=3, dense_steps=3, stages=3, groups=2, vecs_per_lane=1),
          dict(kernel=3, dense_steps=5, stages=2, vecs_per_lane=2),
          dict(kernel=3, vecs_per_lane=1), dict(kernel=3, vecs_per_lane=3),
          dict(kernel=3, vecs_per_lane=3, dense_steps=6, stages=3),
          dict(kernel=3, dynamic_rounds=1), dict(kernel=3, dynamic_rounds=3),
          dict(kernel=3, dynamic_rounds=64, groups=1),
          dict(kernel=3, vecs_per_part_bitmask=64), dict(kernel=3, vecs_per_part_bitmask=20,
                                                        vecs_per_lane=1, stages=4)]


def _staged_case(name):
    rng = np.random.default_rng(sum(map(ord, name)))
    if name == "tiny":
        prob = synth.matrix_tiny(seed=0)
        return prob.A, *synth.population(0, 100, 20, 2, 6, plants=prob.plants), 10
    if name == "ragged_4097x30":
        prob = synth.matrix_random(41, 4097, 30, n_plants=3, plant_rows=(200, 500),
                                   plant_cols=(3, 8))
        return prob.A, *synth.population(9, 257, 30, 2, 12, plants=prob.plants), 40
    if name == "windows_3000x60_L30_45":
        prob = synth.matrix_random(7, 3000, 60, n_plants=2, plant_rows=(300, 600),
                                   plant_cols=(40, 50))
        return prob.A, *synth.population(8, 300, 60, 30, 45, plants=prob.plants), 30
    if name == "long_300x1100":
        A = rng.standard_normal((300, 1100)).astype(np.float32)
        A[:40] = np.sort(A[:40], axis=1)                 # rows rising along 0, 1, 2, ...
        seqs = [[5], [5, 5], [0, 1, 0], list(range(1024)), list(range(65)), list(range(66)),
                list(range(64)), rng.permutation(1100)[:1024].tolist(),
                list(range(1023, -1, -1)), [7] * 1024, list(range(0, 1100, 11))]
        off, cols = oracle.to_cbf(seqs)
        return A, off, cols, 3
    if name == "parts_60000x12":
        prob = synth.matrix_random(5, 60000, 12, n_plants=2, plant_rows=(3000, 6000),
                                   plant_cols=(3, 6))
        return prob.A, *synth.population(4, 37, 12, 1, 5, plants=prob.plants, frac_planted=0.6), 100
    if name == "ties_nan":
        A = rng.integers(-2, 3, (5000, 10)).astype(np.float32)
        A[rng.random(A.shape) < 0.05] = np.nan
        A[rng.random(A.shape) < 0.1] = -0.0
        return A, *synth.population(3, 500, 10, 1, 6, duplicates=True), 7
    raise KeyError(name)


@pytest.mark.parametrize("tune", STAGED)
@pytest.mark.parametrize("case", ["tiny", "ragged_4097x30", "windows_3000x60_L30_45",
                                  "long_300x1100", "parts_60000x12", "ties_nan"])
def test_staged_kernel_exact(case, tune):
    A, off, cols, sigma = _staged_case(case)
    oinc, _, ofit = oracle_eval(A, off, cols, sigma)
    h = eb.ebic_load_matrix(A)
    try:
        eb.ebic_set_path(h, eb.PATH_BITMASK)
        eb.ebic_set_eval_tuning(h, **tune)
        for rep in range(3):               # the work counter is back to zero after each launch
            inc, _, fit = eb.ebic_eval_population(h, off, cols, sigma, want_dec=False)
            eb.ebic_check_device_error(h)
            assert_bits_equal(inc, oinc, f"inc {case} {tune} launch {rep}")
            assert_bits_equal(fit, ofit, f"fit {case} {tune} launch {rep}")
    finally:
        eb.ebic_free(h)


@pytest.mark.parametrize("tune", STAGED[:2] + [dict(kernel=3, vecs_per_part_bitmask=80)])
def test_staged_kernel_expression_full(tune):
    """The expression-shaped workload at full size, 20,000 x 200, P = 4,096."""
    prob = synth.matrix_expression(seed=0)
    off, cols = synth.population(2, 4096, 200, 3, 30, plants=prob.plants)
    oinc, _, ofit = oracle_eval(prob.A, off, cols, 50)
    h = eb.ebic_load_matrix(prob.A)
    try:
        eb.ebic_set_path(h, eb.PATH_BITMASK)
        eb.ebic_set_eval_tuning(h, **tune)
        for _ in range(2):
            inc, _, fit = eb.ebic_eval_population(h, off, cols, 50, want_dec=False)
            assert_bits_equal(inc, oinc, "inc")
            assert_bits_equal(fit, ofit, "fit")
    finally:
        eb.ebic_free(h)


def test_staged_kernel_flags_invalid_series():
    torch = pytest.importorskip("torch")
    A = np.random.default_rng(1).standard_normal((5000, 6)).astype(np.float32)
    h = eb.ebic_load_matrix(A)
    eb.ebic_set_path(h, eb.PATH_BITMASK)
    eb.ebic_set_eval_tuning(h, kernel=3)
    dev = torch.device("cuda:0")
    off = torch.tensor([0, 2, 4, 6, 99], dtype=torch.int32, device=dev)
    cols = torch.tensor([0, 1, 2, 6, 3, 4], dtype=torch.int32, device=dev)
    inc = torch.full((4,), 7, dtype=torch.int32, device=dev)
    fit = torch.full((4,), 7.0, dtype=torch.float64, device=dev)
    eb.ebic_eval_population_dev(h, off, cols, 4, 6, 3, 0, inc, None, fit)
    with pytest.raises(eb.EbicError) as e:
        eb.ebic_check_device_error(h)
    assert e.value.status == 7
    got = inc.cpu().numpy()
    oinc, _, ofit = oracle_eval(A, np.array([0, 2, 4]), np.array([0, 1, 3, 4]), 3)
    assert got[1] == 0 and got[3] == 0 and fit.cpu().numpy()[1] == 0.0
    assert got[0] == oinc[0] and got[2] == oinc[1]
    # a valid launch afterwards is exact (the work counter was reset)
    off2, cols2 = synth.population(3, 200, 6, 2, 5)
    oinc2, _, ofit2 = oracle_eval(A, off2, cols2, 3)
    inc2, _, fit2 = eb.ebic_eval_population(h, off2, cols2, 3, want_dec=False)
    assert_bits_equal(inc2, oinc2, "inc")
    assert_bits_equal(fit2, ofit2, "fit")
    eb.ebic_check_device_error(h)
    eb.ebic_free(h)


# ---------------------------------------------------------------------------
# The phased kernel (launch shape kernel 4): per-CTA chunks of series, their
# dense steps streamed through a ring of shared-memory slots, the live
# vectors' remaining steps walked by the whole CTA.  Rising counts.
# ---------------------------------------------------------------------------
PHASED = [dict(kernel=4), dict(kernel=4, dense_steps=1), dict(kernel=4, dense_steps=3, stages=2),
          dict(kernel=4, dense_steps=4), dict(kernel=4, dense_steps=6, stages=3),
          dict(kernel=4, dense_steps=8)]


def _rising_case():
    """Rows that rise along every column (a sorted matrix): every 128-row
    block of a series in increasing column order stays alive through all its
    steps, so the live-vector and survivor lists of a chunk overflow and the
    walking threads finish those vectors themselves."""
    rng = np.random.default_rng(11)
    A = np.sort(rng.standard_normal((20000, 40)).astype(np.float32), axis=1)
    seqs = [sorted(rng.choice(40, size=int(rng.integers(2, 31)), replace=False).tolist())
            for _ in range(2000)]
    seqs += [rng.permutation(40)[:int(rng.integers(2, 20))].tolist() for _ in range(200)]
    off, cols = oracle.to_cbf(seqs)
    return A, off, cols, 100


@pytest.mark.parametrize("tune", PHASED)
@pytest.mark.parametrize("case", ["tiny", "ragged_4097x30", "windows_3000x60_L30_45",
                                  "long_300x1100", "parts_60000x12", "ties_nan", "rising"])
def test_phased_kernel_exact(case, tune):
    A, off, cols, sigma = _rising_case() if case == "rising" else _staged_case(case)
    oinc, _, ofit = oracle_eval(A, off, cols, sigma)
    h = eb.ebic_load_matrix(A)
    try:
        eb.ebic_set_path(h, eb.PATH_BITMASK)
        eb.ebic_set_eval_tuning(h, **tune)
        for rep in range(2):
            inc, _, fit = eb.ebic_eval_population(h, off, cols, sigma, want_dec=False)
            eb.ebic_check_device_error(h)
            assert_bits_equal(inc, oinc, f"inc {case} {tune} launch {rep}")
            assert_bits_equal(fit, ofit, f"fit {case} {tune} launch {rep}")
    finally:
        eb.ebic_free(h)


@pytest.mark.parametrize("tune", PHASED[:1] + PHASED[3:5])
def test_phased_kernel_expression_full(tune):
    """The expression-shaped workload at full size, 20,000 x 200, P = 4,096."""
    prob = synth.matrix_expression(seed=0)
    off, cols = synth.population(2, 4096, 200, 3, 30, plants=prob.plants)
    oinc, _, ofit = oracle_eval(prob.A, off, cols, 50)
    h = eb.ebic_load_matrix(prob.A)
    try:
        eb.ebic_set_path(h, eb.PATH_BITMASK)
        eb.ebic_set_eval_tuning(h, **tune)
        for _ in range(2):
            inc, _, fit = eb.ebic_eval_population(h, off, cols, 50, want_dec=False)
            assert_bits_equal(inc, oinc, "inc")
            assert_bits_equal(fit, ofit, "fit")
        eb.ebic_check_device_error(h)
    finally:
        eb.ebic_free(h)


def test_phased_kernel_flags_invalid_series():
    torch = pytest.importorskip("torch")
    A = np.random.default_rng(1).standard_normal((5000, 6)).astype(np.float32)
    h = eb.ebic_load_matrix(A)
    eb.ebic_set_path(h, eb.PATH_BITMASK)
    eb.ebic_set_eval_tuning(h, kernel=4)
    dev = torch.device("cuda:0")
    off = torch.tensor([0, 2, 4, 6, 99], dtype=torch.int32, device=dev)
    cols = torch.tensor([0, 1, 2, 6, 3, 4], dtype=torch.int32, device=dev)
    inc = torch.full((4,), 7, dtype=torch.int32, device=dev)
    fit = torch.full((4,), 7.0, dtype=torch.float64, device=dev)
    eb.ebic_eval_population_dev(h, off, cols, 4, 6, 3, 0, inc, None, fit)
    with pytest.raises(eb.EbicError) as e:
        eb.ebic_check_device_error(h)
    assert e.value.status == 7
    got = inc.cpu().numpy()
    oinc, _, ofit = oracle_eval(A, np.array([0, 2, 4]), np.array([0, 1, 3, 4]), 3)
    assert got[1] == 0 and got[3] == 0 and fit.cpu().numpy()[1] == 0.0
    assert got[0] == oinc[0] and got[2] == oinc[1]
    off2, cols2 = synth.population(3, 200, 6, 2, 5)
    oinc2, _, ofit2 = oracle_eval(A, off2, cols2, 3)
    inc2, _, fit2 = eb.ebic_eval_population(h, off2, cols2, 3, want_dec=False)
    assert_bits_equal(inc2, oinc2, "inc")
    assert_bits_equal(fit2, ofit2, "fit")
    eb.ebic_check_device_error(h)
    eb.ebic_free(h)


def test_staged_kernel_rejects_bad_tuning():
    h = eb.ebic_load_matrix(synth.matrix_tiny(seed=0).A)
    try:
        for bad in (dict(kernel=3, dense_steps=9), dict(kernel=3, stages=1),
                    dict(kernel=3, stages=5), dict(kernel=3, groups=16),
                    dict(kernel=3, dynamic_rounds=-2), dict(kernel=3, dynamic_rounds=65),
                    dict(kernel=5), dict(kernel=4, dense_steps=9)):
            with pytest.raises(eb.EbicError):
                eb.ebic_set_eval_tuning(h, **bad)
    finally:
        eb.ebic_free(h)
