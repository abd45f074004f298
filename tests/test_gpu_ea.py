"""Parity of the device generation loop (Steps 1-5) with the oracle: the
same seed gives the same populations, fitness and top-rank lists, generation
by generation, bit for bit."""
import numpy as np
import pytest

import oracle
import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth
from helpers import assert_bits_equal

pytestmark = pytest.mark.gpu

BASE = dict(pop_size=100, len_min=2, len_max=6, iterations=10, sigma=10, toprank_size=100,
            tournament_k=2, overlap_tau=0.5, elite_frac=0.25, penalty_base=1.2,
            p_crossover=0.5, seed=0)


@pytest.fixture(scope="module", autouse=True)
def built():
    eb.build()
    yield


def _device_params(kw):
    d = dict(kw)
    d.pop("oversample", None)
    mode = d.pop("fitness_support", 0)
    p = eb.ebic_default_params(**d)
    p.support_mode = mode
    return p


def run_both(A, gens_to_check=None, tuning=None, **kw):
    """Runs the oracle and the device loop with the same parameters and compares
    them generation by generation.  oversample > 1 screens offspring with
    pseudo scores on both sides; `tuning` fixes the evaluation's launch shape."""
    kw = {**BASE, **kw}
    ref = oracle.run(A, trace=True, **kw)
    h = eb.ebic_load_matrix(A)
    try:
        if tuning:
            eb.ebic_set_path(h, eb.PATH_BITMASK)
            eb.ebic_set_eval_tuning(h, **tuning)
        p = _device_params(kw)
        V = kw.get("oversample", 1)
        if V > 1:
            eb.ebic_run_screen(h, None, V, eb.SCREEN_PSEUDO)
        eb.ebic_run_init(h, p)
        P, T, L = kw["pop_size"], kw["toprank_size"], kw["len_max"]
        done = ref["stats"]["generations_done"]
        checks = range(done + 1) if gens_to_check is None else gens_to_check
        if ref["stats"]["stop_reason"] == 2:        # Step 1 never completed
            checks = ()
            assert eb.ebic_get_population(h, P, L)["seqs"] == []
        stats = None
        for g in range(done + 1):
            if g > 0:
                stats = eb.ebic_run_step(h, 1)
            if g in checks:
                _compare_generation(h, ref, g, P, T, L, kw)
        # the run stops (or ends) exactly where the oracle's does
        rest = kw["iterations"] - done
        if rest:
            stats = eb.ebic_run_step(h, rest)
        if stats is None:
            stats = eb.ebic_run_step(h, 0)
        rs = ref["stats"]
        for key in ("generations_done", "stop_reason", "tabu_hits_total", "attempts_total",
                    "evaluations_total", "last_gen_hits", "toprank_n"):
            assert stats[key] == rs[key], (key, stats[key], rs[key])
        top, fit, inc = eb.ebic_get_toprank(h, T, L)
        assert top == ref["toprank"]
        assert_bits_equal(fit, ref["toprank_f"], "final toprank fitness")
        assert_bits_equal(inc, ref["toprank_inc"], "final toprank inc")
        return stats
    finally:
        eb.ebic_free(h)


def _compare_generation(h, ref, g, P, T, L, kw):
    pop = eb.ebic_get_population(h, P, L)
    rp = ref["trace_pop"][g]
    if pop["seqs"] != rp["seqs"]:
        bad = [i for i in range(P) if pop["seqs"][i] != rp["seqs"][i]][:5]
        raise AssertionError(f"generation {g}: population differs at {bad}: "
                             f"{[pop['seqs'][i] for i in bad]} vs {[rp['seqs'][i] for i in bad]}")
    assert_bits_equal(pop["inc"], rp["inc"], f"gen {g} inc")
    if kw.get("fitness_support", 0) == 1:
        assert_bits_equal(pop["dec"], rp["dec"], f"gen {g} dec")
    assert_bits_equal(pop["f"], rp["f"], f"gen {g} fitness")
    top, fit, _ = eb.ebic_get_toprank(h, T, L)
    rt = ref["trace_top"][g]
    assert top == rt["seqs"], f"generation {g}: top-rank list differs"
    assert_bits_equal(fit, rt["f"], f"gen {g} toprank fitness")


def test_tiny_200x20_ten_generations():
    prob = synth.matrix_tiny(seed=0)
    st = run_both(prob.A)
    assert st["generations_done"] == 10


def test_paper_1000x100_population_600():
    prob = synth.matrix_paper(seed=0)
    run_both(prob.A, gens_to_check={0, 1, 2, 10, 30}, pop_size=600, len_min=3, len_max=20,
             sigma=25, iterations=30)


def test_paper_1000x100_thousand_generations():
    """The benchmark's generation workload over its whole run length: 1,000
    generations of the 1000 x 100 matrix (P = 600, lengths 3-20, sigma 25),
    populations and top-rank lists compared at generations 1, 250, 500, 999
    and 1,000, and the run statistics at the end."""
    prob = synth.matrix_paper(seed=0)
    st = run_both(prob.A, gens_to_check={1, 250, 500, 999, 1000}, pop_size=600, len_min=3,
                  len_max=20, sigma=25, iterations=1000)
    assert st["generations_done"] == 1000 and st["tabu_hits_total"] > 0


def test_paper_1000x100_screened_two_hundred_generations():
    """Screening with pseudo scores (8 candidates per attempt) on the same
    workload for 200 generations."""
    prob = synth.matrix_paper(seed=0)
    st = run_both(prob.A, gens_to_check={1, 100, 199, 200}, pop_size=600, len_min=3,
                  len_max=20, sigma=25, iterations=200, oversample=8)
    assert st["generations_done"] == 200


@pytest.mark.parametrize("variant", [
    dict(tournament_k=1), dict(tournament_k=3), dict(tournament_k=4),
    dict(p_crossover=0.0), dict(p_crossover=1.0), dict(fitness_support=1),
    dict(penalty_base=1.0), dict(penalty_base=2.5), dict(elite_frac=0.0), dict(elite_frac=1.0),
    dict(toprank_size=5), dict(overlap_tau=0.75), dict(overlap_tau=0.0), dict(seed=12345),
    dict(len_min=3, len_max=3), dict(sigma=1000)])
def test_parameter_variants(variant):
    prob = synth.matrix_tiny(seed=1)
    run_both(prob.A, iterations=8, **variant)


def test_ties_and_nan_matrix():
    rng = np.random.default_rng(2)
    A = rng.integers(-2, 3, (300, 12)).astype(np.float32)
    A[rng.random(A.shape) < 0.03] = np.nan
    run_both(A, iterations=8, len_max=5)


def test_tabu_stop_matches():
    A = np.random.default_rng(0).standard_normal((50, 3)).astype(np.float32)
    st = run_both(A, iterations=100, pop_size=6, len_min=2, len_max=3, sigma=2, toprank_size=10)
    assert st["stop_reason"] == 1 and st["generations_done"] < 100


def test_step1_failure_matches():
    A = np.random.default_rng(0).standard_normal((20, 2)).astype(np.float32)
    st = run_both(A, iterations=3, pop_size=3, len_min=2, len_max=2, sigma=2, toprank_size=4)
    assert st["stop_reason"] == 2


def test_one_call_run_generations_equals_stepping():
    prob = synth.matrix_tiny(seed=3)
    kw = {**BASE, "iterations": 12, "seed": 7}
    ref = oracle.run(prob.A, **kw)
    h = eb.ebic_load_matrix(prob.A)
    try:
        top, fit, st = eb.ebic_run_generations(h, _device_params(kw))
    finally:
        eb.ebic_free(h)
    assert top == ref["toprank"] and st["generations_done"] == 12
    assert_bits_equal(fit, ref["toprank_f"], "toprank fitness")


def test_in_graph_kernel_timing_leaves_the_run_unchanged():
    """Event nodes around k_build in the replayed graph: the run is the
    oracle's, every replay is timed, and a ring of three event pairs wraps."""
    prob = synth.matrix_tiny(seed=3)
    kw = {**BASE, "iterations": 12, "seed": 7}
    ref = oracle.run(prob.A, **kw)
    h = eb.ebic_load_matrix(prob.A)
    try:
        with pytest.raises(eb.EbicError):
            eb.ebic_set_kernel_timing(h, -1)
        eb.ebic_run_init(h, _device_params(kw))
        with pytest.raises(eb.EbicError):               # started without timing
            eb.ebic_read_kernel_timing(h)
        eb.ebic_set_kernel_timing(h, 3)
        eb.ebic_run_init(h, _device_params(kw))
        eb.ebic_run_step(h, 5)
        us, n = eb.ebic_read_kernel_timing(h, reset=True)
        assert n == 5 and 0 < us < 1e5
        eb.ebic_run_step(h, 7)
        us, n = eb.ebic_read_kernel_timing(h)
        assert n == 7 and 0 < us < 1e5
        top, fit, _ = eb.ebic_get_toprank(h, kw["toprank_size"], kw["len_max"])
        st = eb.ebic_run_step(h, 0)
    finally:
        eb.ebic_free(h)
    assert top == ref["toprank"] and st["generations_done"] == 12
    assert_bits_equal(fit, ref["toprank_f"], "toprank fitness")


def test_state_errors():
    prob = synth.matrix_tiny(seed=0)
    h = eb.ebic_load_matrix(prob.A)
    try:
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_run_step(h, 1)
        assert e.value.status == 5
        eb.ebic_run_init(h, _device_params({**BASE, "iterations": 2}))
        eb.ebic_run_step(h, 2)
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_run_step(h, 1)
        assert e.value.status == 5
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_run_init(h, _device_params({**BASE, "len_max": 21}))
        assert e.value.status == 1
    finally:
        eb.ebic_free(h)


def test_expression_shape_three_generations():
    prob = synth.matrix_expression(seed=0)
    run_both(prob.A, gens_to_check={0, 3}, pop_size=4096, len_min=3, len_max=30, sigma=50,
             iterations=3)


@pytest.mark.parametrize("tuning", [dict(kernel=2), dict(kernel=3, dense_steps=6),
                                    dict(kernel=4), dict(kernel=4, dense_steps=3)])
def test_expression_shape_each_launch_shape(tuning):
    """The EA's own population view (the archive) through each bitmask launch
    shape, set by hand so that the run keeps it."""
    prob = synth.matrix_expression(seed=1)
    run_both(prob.A, gens_to_check={0, 2, 5}, tuning=tuning, pop_size=600, len_min=3,
             len_max=30, sigma=50, iterations=5)


# ---------------------------------------------------------------------------
# offspring screening with pseudo scores: the candidate generation, the pick
# and the record completion against the oracle, bit for bit
@pytest.mark.parametrize("variant", [
    dict(oversample=2), dict(oversample=4, tournament_k=1), dict(oversample=8, tournament_k=3),
    dict(oversample=16, p_crossover=1.0), dict(oversample=3, p_crossover=0.0),
    dict(oversample=5, tournament_k=4, fitness_support=1)])
def test_pseudo_screening_matches_oracle(variant):
    prob = synth.matrix_tiny(seed=3)
    run_both(prob.A, iterations=8, **variant)


def test_pseudo_screening_paper_shape():
    prob = synth.matrix_paper(seed=1)
    run_both(prob.A, gens_to_check={0, 1, 5, 20}, pop_size=600, len_min=3, len_max=20,
             sigma=25, iterations=20, oversample=8)


def test_pseudo_screening_changes_the_run_but_not_step1():
    prob = synth.matrix_tiny(seed=4)
    plain = oracle.run(prob.A, trace=True, **{**BASE, "iterations": 3})
    scr = oracle.run(prob.A, trace=True, **{**BASE, "iterations": 3, "oversample": 4})
    assert plain["trace_pop"][0]["seqs"] == scr["trace_pop"][0]["seqs"]
    assert plain["trace_pop"][3]["seqs"] != scr["trace_pop"][3]["seqs"]


def test_screen_argument_errors():
    prob = synth.matrix_tiny(seed=0)
    h = eb.ebic_load_matrix(prob.A)
    try:
        for bad in [dict(oversample=0, mode=eb.SCREEN_PSEUDO), dict(oversample=17, mode=eb.SCREEN_PSEUDO),
                    dict(oversample=4, mode=7), dict(oversample=4, mode=eb.SCREEN_SURROGATE)]:
            with pytest.raises(eb.EbicError) as e:
                eb.ebic_run_screen(h, None, **bad)
            assert e.value.status == 1
        # screening off again: the plain trajectory
        eb.ebic_run_screen(h, None, 4, eb.SCREEN_PSEUDO)
        eb.ebic_run_screen(h, None, 1, eb.SCREEN_OFF)
    finally:
        eb.ebic_free(h)


def test_wide_matrix_generic_paths():
    """More than 256 columns: the builder's generic consumer and the CTA-wide
    Step 5 (the bitset paths need at most 256 columns)."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((300, 300)).astype(np.float32)
    run_both(A, iterations=6, len_max=8)


def test_eight_word_bitsets():
    """129-256 columns: the builder's fast path and Step 5's warp visit with
    eight-word column bitsets (two 16-byte vectors per series)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((400, 160)).astype(np.float32)
    run_both(A, gens_to_check={0, 1, 6, 12}, iterations=12, pop_size=300, len_min=2,
             len_max=10, sigma=8)


@pytest.mark.parametrize("P,T", [(37, 3), (300, 250), (1024, 1), (2000, 50)])
def test_population_and_list_sizes(P, T):
    """Populations that are not powers of two, lists shorter and longer than
    a warp's chunk, a list of one; Step 5's sort with one, two and four keys
    per thread (P up to 512, 1,024 and 2,048)."""
    prob = synth.matrix_tiny(seed=5)
    run_both(prob.A, iterations=5, pop_size=P, toprank_size=T, len_max=6)


def test_profiled_step_splits_the_screened_records_stage():
    """ebic_run_step_profiled: with screening, the records stage is also given
    as candidates + scores + pick, which add up to it; without, those keys are
    absent."""
    prob = synth.matrix_tiny(seed=0)
    h = eb.ebic_load_matrix(prob.A)
    try:
        p = _device_params({**BASE, "iterations": 6})
        eb.ebic_run_init(h, p)
        eb.ebic_run_step(h, 2)
        plain = eb.ebic_run_step_profiled(h)
        assert set(plain) == set(eb.KERNELS[:5]) and plain["k_build"] > 0
        eb.ebic_run_screen(h, None, 8, eb.SCREEN_PSEUDO)
        eb.ebic_run_init(h, p)
        eb.ebic_run_step(h, 2)
        scr = eb.ebic_run_step_profiled(h)
        parts = scr["screen_candidates"] + scr["screen_scores"] + scr["screen_pick"]
        assert min(scr["screen_candidates"], scr["screen_scores"], scr["screen_pick"]) > 0
        assert abs(parts - scr["k_spec"]) <= 1e-3 * scr["k_spec"] + 0.01
    finally:
        eb.ebic_free(h)
