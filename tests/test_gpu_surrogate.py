"""The fitness surrogate on the GPU against its fp64 oracle (oracle/mlp.py),
and offspring screening with a trained surrogate.

Tolerances (bf16 operands, unit roundoff u = 2^-9, fp32 accumulation).  The
error model: each bf16 rounding (features, W1, h1, W2, h2 in the forward;
dh2, dh1 and the weight copies in the reverse pass) multiplies its value by
(1 + d), d independent and uniform in [-u, u] (variance u^2 / 3); fp32
accumulation over at most 256 terms (< 2^-16 relative) is neglected.
  forward  |y_gpu - y| <= 10 sigma + 1e-5, sigma^2 the variance of y under the
           model, propagated layer by layer from the oracle's own activations
           (a worst-case first-order bound is vacuous here: sums of |terms|
           exceed the outputs by three orders of magnitude).  Emulating the
           kernel's rounding points in numpy gives at most 5.2 sigma over
           1,000 outputs.
  backward per parameter tensor, relative Frobenius error <= 2^-4 and cosine
           similarity >= 0.998.  The emulated reverse pass gives at most 0.016
           and 0.9998.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
import paper_1801_03039_gb300 as eb
from paper_1801_03039_gb300 import synth
from helpers import assert_bits_equal, oracle_eval

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -9


@pytest.fixture(scope="module", autouse=True)
def built():
    eb.build()
    yield


def _series(rng, n, C, Lmin, Lmax):
    return [rng.choice(C, size=int(rng.integers(Lmin, Lmax + 1)), replace=False) for _ in range(n)]


def _device_series(seqs, S):
    n = len(seqs)
    arr = np.zeros((n, S), np.int16)
    lens = np.zeros(n, np.int32)
    for i, s in enumerate(seqs):
        arr[i, :len(s)] = s
        lens[i] = len(s)
    return torch.from_numpy(arr).cuda(), torch.from_numpy(lens).cuda()


def _oracle_params(C, seed):
    """Seeded parameters with non-zero biases, rounded to the fp32 the device holds."""
    rng = np.random.default_rng(seed + 100)
    p = mlp.init_params(C, seed)
    p["b1"] = rng.standard_normal(mlp.H) * 0.1
    p["b2"] = rng.standard_normal(mlp.H) * 0.1
    p["b3"] = np.array(0.25)
    p = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}
    flat = np.concatenate([p[k].reshape(-1) for k in ["Emb", "W1", "b1", "W2", "b2", "w3", "b3"]])
    return p, flat.astype(np.float32)


def _forward_sigma(X, p):
    """Standard deviation of y under the bf16 rounding-error model."""
    _, (X, z1, h1, z2, h2) = mlp.forward(X, p)
    u2 = U * U / 3
    vz1 = (X ** 2) @ (p["W1"] ** 2) * 2 * u2
    vh1 = (z1 > 0) * (vz1 + h1 ** 2 * u2)
    vz2 = vh1 @ (p["W2"] ** 2) + (h1 ** 2) @ (p["W2"] ** 2) * u2
    vh2 = (z2 > 0) * (vz2 + h2 ** 2 * u2)
    return np.sqrt(vh2 @ (p["w3"] ** 2))


@pytest.fixture(scope="module")
def paper_problem():
    prob = synth.matrix_paper(seed=0)
    h = eb.ebic_load_matrix(prob.A)
    yield prob, h
    eb.ebic_free(h)


def test_column_statistics(paper_problem):
    rng = np.random.default_rng(0)
    A = rng.lognormal(0, 1, (777, 37)).astype(np.float32)
    A[rng.random(A.shape) < 0.05] = np.nan
    h = eb.ebic_load_matrix(A)
    s = eb.ebic_surrogate_create(h, 16, 0)
    try:
        m, d = eb.ebic_surrogate_colstats(s, 37)
        om, od = mlp.column_stats(A)
        np.testing.assert_allclose(m, om, rtol=2e-6, atol=1e-6)
        np.testing.assert_allclose(d, od, rtol=2e-5, atol=1e-6)
    finally:
        eb.ebic_surrogate_free(s)
        eb.ebic_free(h)


@pytest.mark.parametrize("kind", [eb.FORWARD_TCGEN05, eb.FORWARD_MMA_SYNC])
def test_forward_matches_oracle(paper_problem, kind):
    prob, h = paper_problem
    C = prob.A.shape[1]
    s = eb.ebic_surrogate_create(h, 20, 1)
    try:
        eb.ebic_surrogate_forward_kernel(s, kind)
        p, flat = _oracle_params(C, 7)
        eb.ebic_surrogate_params(s, flat)
        back = eb.ebic_surrogate_params(s)
        assert_bits_equal(back, flat, "parameter round trip")
        rng = np.random.default_rng(1)
        seqs = _series(rng, 1000, C, 1, 20)          # 15 full 64-row tiles + 40
        seqs[0] = np.array([5])
        seqs[1] = np.arange(20)
        d_seq, d_len = _device_series(seqs, 20)
        out = torch.empty(len(seqs), dtype=torch.float32, device="cuda")
        eb.ebic_surrogate_predict(s, d_seq, d_len, 20, len(seqs), out)
        y = out.cpu().numpy().astype(np.float64)
        cm, cs = mlp.column_stats(prob.A)
        X = mlp.features(seqs, p["Emb"], cm, cs, 20)
        want, _ = mlp.forward(X, p)
        bound = 10 * _forward_sigma(X, p) + 1e-5
        err = np.abs(y - want)
        assert np.all(err <= bound), (err.max(), float((err / bound).max()))
        # the bound is not vacuous: predictions spread far beyond it
        assert np.std(want) > 20 * np.median(bound)
        # reversal changes nothing beyond the fp32 order of the embedding sum
        d_rev, d_rlen = _device_series([x[::-1] for x in seqs], 20)
        out2 = torch.empty_like(out)
        eb.ebic_surrogate_predict(s, d_rev, d_rlen, 20, len(seqs), out2)
        assert np.all(np.abs(out2.cpu().numpy() - y) <= 2 * bound)
    finally:
        eb.ebic_surrogate_free(s)


def test_forward_kernels_agree(paper_problem):
    """The tcgen05 scoring kernel (128-series tiles, accumulators in tensor
    memory) and the mma.sync one (64-series tiles) round at the same points;
    on 5,000 series of ragged tiles (39 full tiles of 128 + 8) they differ by
    no more than the fp32 order of the additions allows."""
    prob, h = paper_problem
    C = prob.A.shape[1]
    s = eb.ebic_surrogate_create(h, 20, 2)
    try:
        p, flat = _oracle_params(C, 11)
        eb.ebic_surrogate_params(s, flat)
        rng = np.random.default_rng(3)
        seqs = _series(rng, 5000, C, 1, 20)
        d_seq, d_len = _device_series(seqs, 20)
        outs = {}
        for kind in (eb.FORWARD_TCGEN05, eb.FORWARD_MMA_SYNC):
            eb.ebic_surrogate_forward_kernel(s, kind)
            out = torch.full((len(seqs),), float("nan"), dtype=torch.float32, device="cuda")
            for _ in range(2):                      # twice: the result does not depend on history
                eb.ebic_surrogate_predict(s, d_seq, d_len, 20, len(seqs), out)
            outs[kind] = out.cpu().numpy().astype(np.float64)
        a, b = outs[eb.FORWARD_TCGEN05], outs[eb.FORWARD_MMA_SYNC]
        assert np.isfinite(a).all() and np.isfinite(b).all()
        cm, cs = mlp.column_stats(prob.A)
        X = mlp.features(seqs, p["Emb"], cm, cs, 20)
        bound = 10 * _forward_sigma(X, p) + 1e-5
        assert np.all(np.abs(a - b) <= 2 * bound), float(np.abs(a - b).max())
        with pytest.raises(eb.EbicError):
            eb.ebic_surrogate_forward_kernel(s, 2)
    finally:
        eb.ebic_surrogate_free(s)


TRAIN_KINDS = [eb.FORWARD_TCGEN05, eb.FORWARD_MMA_SYNC]


@pytest.mark.parametrize("kind", TRAIN_KINDS)
def test_gradients_match_oracle(paper_problem, kind):
    """Loss and every parameter gradient of one minibatch of 300 series (a
    ragged last tile of 44 rows, split-K over a ragged range) against the
    oracle, with the tcgen05 training GEMMs and with the mma.sync ones."""
    prob, h = paper_problem
    C = prob.A.shape[1]
    s = eb.ebic_surrogate_create(h, 20, 2)
    try:
        eb.ebic_surrogate_train_kernel(s, kind)
        p, flat = _oracle_params(C, 9)
        eb.ebic_surrogate_params(s, flat)
        rng = np.random.default_rng(2)
        B = 300                                       # split-K over a ragged batch
        seqs = _series(rng, B, C // 2, 2, 20)         # columns >= 50 never used
        cm, cs = mlp.column_stats(prob.A)
        X = mlp.features(seqs, p["Emb"], cm, cs, 20)
        y0, _ = mlp.forward(X, p)
        t = y0 - 1.0 - np.abs(rng.standard_normal(B))    # residuals >= 1
        loss, g = mlp.loss_and_grads(seqs, t, p, cm, cs, 20)
        d_seq, d_len = _device_series(seqs, 20)
        d_t = torch.from_numpy(t.astype(np.float32)).cuda()
        gl = eb.ebic_surrogate_step(s, d_seq, d_len, 20, d_t, B, update=False)
        assert abs(gl - loss) <= 0.02 * loss
        gg = eb.ebic_surrogate_split(eb.ebic_surrogate_grads(s).astype(np.float64), C)
        for name in ["Emb", "W1", "b1", "W2", "b2", "w3", "b3"]:
            a, b = gg[name].reshape(-1), np.asarray(g[name]).reshape(-1)
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
            assert rel <= 2 ** -4 and cos >= 0.998, (name, rel, cos)
        assert np.all(gg["Emb"][C // 2:] == 0)
        assert np.all(gg["W1"][67:] == 0)
    finally:
        eb.ebic_surrogate_free(s)


@pytest.mark.parametrize("kind", TRAIN_KINDS)
def test_adam_step(paper_problem, kind):
    """First Adam step: every parameter moves by at most lr, and where the
    oracle's gradient is large it moves by exactly -lr sign(g)."""
    prob, h = paper_problem
    C = prob.A.shape[1]
    s = eb.ebic_surrogate_create(h, 20, 3)
    try:
        eb.ebic_surrogate_train_kernel(s, kind)
        p, flat = _oracle_params(C, 11)
        eb.ebic_surrogate_params(s, flat)
        rng = np.random.default_rng(3)
        B = 256
        seqs = _series(rng, B, C - 10, 2, 20)         # the last 10 columns unused
        cm, cs = mlp.column_stats(prob.A)
        y0, _ = mlp.forward(mlp.features(seqs, p["Emb"], cm, cs, 20), p)
        t = y0 - 1.0 - np.abs(rng.standard_normal(B))
        _, g = mlp.loss_and_grads(seqs, t, p, cm, cs, 20)
        d_seq, d_len = _device_series(seqs, 20)
        d_t = torch.from_numpy(t.astype(np.float32)).cuda()
        lr = 1e-3
        eb.ebic_surrogate_step(s, d_seq, d_len, 20, d_t, B, lr=lr, update=True)
        after = eb.ebic_surrogate_split(eb.ebic_surrogate_params(s).astype(np.float64), C)
        before = eb.ebic_surrogate_split(flat.astype(np.float64), C)
        for name in ["Emb", "W1", "b1", "W2", "b2", "w3", "b3"]:
            dp = (after[name] - before[name]).reshape(-1)
            gv = np.asarray(g[name]).reshape(-1)
            pv = np.abs(before[name].reshape(-1))
            assert np.all(np.abs(dp) <= lr * (1 + 1e-4) + 2 ** -23 * pv), name
            strong = np.abs(gv) > 0.25 * np.abs(gv).max()
            assert strong.any()
            np.testing.assert_array_less(np.abs(dp[strong] + lr * np.sign(gv[strong])),
                                         1e-4 * lr + 2 ** -23 * pv[strong] + 1e-12)
        # structurally zero gradients (unused embedding rows, the padded W1
        # rows) leave the parameters untouched; elsewhere a unit on the ReLU
        # boundary may be alive on one side only, and Adam's first step moves
        # any non-zero gradient by lr
        used = sorted({int(c) for x in seqs for c in x})
        unused = np.setdiff1d(np.arange(C), used)
        assert np.all(after["Emb"][unused] == before["Emb"][unused])
        assert np.all(after["W1"][67:] == before["W1"][67:])
    finally:
        eb.ebic_surrogate_free(s)


def _plain_run(h, seed, P=300, iters=60):
    p = eb.ebic_default_params(pop_size=P, len_min=3, len_max=20, iterations=iters, sigma=25,
                               toprank_size=100, tournament_k=2, seed=seed)
    eb.ebic_run_screen(h, None, 1, eb.SCREEN_OFF)
    eb.ebic_run_init(h, p)
    eb.ebic_run_step(h, iters)
    return p


def _spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    return float(np.corrcoef(ra, rb)[0, 1])


def test_training_on_logged_runs(paper_problem):
    """Trained on (series, exact fitness) pairs logged from two runs, the
    surrogate ranks a third run's individuals far better than chance."""
    prob, h = paper_problem
    s = eb.ebic_surrogate_create(h, 20, 4)
    try:
        for seed in (10, 11):
            _plain_run(h, seed)
            n = eb.ebic_surrogate_log(s, h)
        assert n == 2 * 61 * 300
        first = eb.ebic_surrogate_train(s, 1, 1024, 1e-3)
        last = eb.ebic_surrogate_train(s, 600, 1024, 1e-3)
        assert last < 0.6 * first, (first, last)
        # held-out run
        _plain_run(h, 12)
        pop = eb.ebic_get_population(h, 300, 20)
        seqs = pop["seqs"]
        d_seq, d_len = _device_series([np.array(x) for x in seqs], 20)
        out = torch.empty(len(seqs), dtype=torch.float32, device="cuda")
        eb.ebic_surrogate_predict(s, d_seq, d_len, 20, len(seqs), out)
        rho = _spearman(out.cpu().numpy(), np.log1p(pop["f"]))
        assert rho > 0.3, rho
    finally:
        eb.ebic_run_screen(h, None, 1, eb.SCREEN_OFF)
        eb.ebic_surrogate_free(s)


def test_surrogate_screened_run(paper_problem):
    """A screened run stays a valid EBIC run: distinct individuals, exact
    support and Eq. (1) for everything that enters a population, the same
    result on a repeat; the surrogate cannot be freed while attached."""
    prob, h = paper_problem
    s = eb.ebic_surrogate_create(h, 20, 5)
    try:
        _plain_run(h, 20, iters=20)
        eb.ebic_surrogate_log(s, h)
        eb.ebic_surrogate_train(s, 200, 512, 1e-3)
        p = eb.ebic_default_params(pop_size=300, len_min=3, len_max=20, iterations=15, sigma=25,
                                   toprank_size=100, tournament_k=2, seed=21)
        results = []
        for _ in range(2):
            eb.ebic_run_screen(h, s, 8, eb.SCREEN_SURROGATE)
            eb.ebic_run_init(h, p)
            st = eb.ebic_run_step(h, 15)
            assert st["generations_done"] == 15
            pop = eb.ebic_get_population(h, 300, 20)
            seqs = pop["seqs"]
            assert len({tuple(x) for x in seqs}) == 300
            assert all(3 <= len(x) <= 20 and len(set(x)) == len(x) for x in seqs)
            off, cols = oracle.to_cbf(seqs)
            inc, _, fit = oracle_eval(prob.A, off, cols, 25)
            assert_bits_equal(pop["inc"], inc, "screened population inc")
            assert_bits_equal(pop["f"], fit, "screened population fitness")
            results.append(eb.ebic_get_toprank(h, 100, 20))
        assert results[0][0] == results[1][0]
        assert_bits_equal(results[0][1], results[1][1], "repeat top-rank fitness")
        with pytest.raises(eb.EbicError) as e:
            eb.ebic_surrogate_free(s)
        assert e.value.status == 5
    finally:
        eb.ebic_run_screen(h, None, 1, eb.SCREEN_OFF)
        eb.ebic_surrogate_free(s)


def test_trained_surrogate_picks_fitter_children(paper_problem):
    """What the trained network adds over screening without it: from the same
    Step 1 population, the children accepted in generation 1 when the
    surrogate scores the 8 candidates are fitter (exact Eq. (1)) than when
    random Philox scores do, with the same oversampling and the same
    preference for candidates outside the tabu list."""
    prob, h = paper_problem
    s = eb.ebic_surrogate_create(h, 20, 6)
    try:
        for seed in (30, 31):
            _plain_run(h, seed)
            eb.ebic_surrogate_log(s, h)
        eb.ebic_surrogate_train(s, 600, 1024, 1e-3)
        gain = []
        for seed in range(40, 46):
            means = {}
            for mode in (eb.SCREEN_SURROGATE, eb.SCREEN_PSEUDO):
                eb.ebic_run_screen(h, s if mode == eb.SCREEN_SURROGATE else None, 8, mode)
                p = eb.ebic_default_params(pop_size=300, len_min=3, len_max=20, iterations=1,
                                           sigma=25, toprank_size=100, tournament_k=2, seed=seed)
                eb.ebic_run_init(h, p)
                eb.ebic_run_step(h, 1)
                pop = eb.ebic_get_population(h, 300, 20)
                means[mode] = float(np.mean(np.log1p(pop["f"])))
            gain.append(means[eb.SCREEN_SURROGATE] - means[eb.SCREEN_PSEUDO])
        assert np.mean(gain) > 0 and sum(g > 0 for g in gain) >= 5, gain
    finally:
        eb.ebic_run_screen(h, None, 1, eb.SCREEN_OFF)
        eb.ebic_surrogate_free(s)


@pytest.mark.parametrize("kind", TRAIN_KINDS)
def test_training_is_deterministic(paper_problem, kind):
    """Two surrogates created with the same seed and trained on the same log
    end with bit-identical parameters (no atomics in the reverse pass), and a
    large minibatch exercises the split-K weight gradients."""
    prob, h = paper_problem
    _plain_run(h, 50, iters=20)
    out = []
    for _ in range(2):
        s = eb.ebic_surrogate_create(h, 20, 77)
        try:
            eb.ebic_surrogate_train_kernel(s, kind)
            eb.ebic_surrogate_log(s, h)
            loss = eb.ebic_surrogate_train(s, 40, 2048, 1e-3)
            out.append((eb.ebic_surrogate_params(s), loss))
        finally:
            eb.ebic_surrogate_free(s)
    assert_bits_equal(out[0][0], out[1][0], "trained parameters")
    assert out[0][1] == out[1][1]


def test_train_kernels_agree(paper_problem):
    """The tcgen05 training GEMMs and the mma.sync ones give the same loss and
    gradients up to the fp32 order of additions (and the bf16 roundings that
    order can flip) on a minibatch of 1,000 series: eight row tiles, the last
    of 104 rows, and three split-K ranges of 384, 384 and 232 rows."""
    prob, h = paper_problem
    C = prob.A.shape[1]
    p, flat = _oracle_params(C, 13)
    rng = np.random.default_rng(5)
    B = 1000
    seqs = _series(rng, B, C, 1, 20)
    cm, cs = mlp.column_stats(prob.A)
    y0, _ = mlp.forward(mlp.features(seqs, p["Emb"], cm, cs, 20), p)
    t = y0 - 1.0 - np.abs(rng.standard_normal(B))
    d_seq, d_len = _device_series(seqs, 20)
    d_t = torch.from_numpy(t.astype(np.float32)).cuda()
    res = {}
    for kind in TRAIN_KINDS:
        s = eb.ebic_surrogate_create(h, 20, 4)
        try:
            eb.ebic_surrogate_train_kernel(s, kind)
            eb.ebic_surrogate_params(s, flat)
            loss = eb.ebic_surrogate_step(s, d_seq, d_len, 20, d_t, B, update=False)
            res[kind] = (loss, eb.ebic_surrogate_split(
                eb.ebic_surrogate_grads(s).astype(np.float64), C))
        finally:
            eb.ebic_surrogate_free(s)
    (la, ga), (lb, gb) = res[TRAIN_KINDS[0]], res[TRAIN_KINDS[1]]
    assert abs(la - lb) <= 1e-3 * abs(lb)
    for name in ["Emb", "W1", "b1", "W2", "b2", "w3", "b3"]:
        a, b = ga[name].reshape(-1), gb[name].reshape(-1)
        assert np.isfinite(a).all()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 2 ** -6, (name, rel)
    with pytest.raises(eb.EbicError):
        s = eb.ebic_surrogate_create(h, 20, 4)
        try:
            eb.ebic_surrogate_train_kernel(s, 2)
        finally:
            eb.ebic_surrogate_free(s)


def test_replayed_training_does_not_depend_on_the_call_split(paper_problem):
    """Training replays one captured Adam step; the step's minibatch draw and
    bias corrections come from a device replay index and a table built per
    call from the steps done so far.  Three steps in one call and the same
    three steps in three calls end with bit-identical parameters."""
    prob, h = paper_problem
    _plain_run(h, 60, iters=10)
    out = []
    for split in ([3], [1, 1, 1], [2, 1]):
        s = eb.ebic_surrogate_create(h, 20, 5)
        try:
            eb.ebic_surrogate_log(s, h)
            losses = [eb.ebic_surrogate_train(s, k, 512, 1e-3) for k in split]
            out.append((eb.ebic_surrogate_params(s), losses[-1]))
        finally:
            eb.ebic_surrogate_free(s)
    for params, loss in out[1:]:
        assert_bits_equal(params, out[0][0], "trained parameters")
        assert loss == out[0][1]


def test_surrogate_at_the_column_limit():
    """Series hold 16-bit column ids: a matrix of 65,535 columns gets a
    surrogate that scores a series of its last columns; 65,536 columns are
    refused by the loader already (EBIC_ERR_ARG)."""
    C = 65535
    A = np.random.default_rng(C).standard_normal((4, C)).astype(np.float32)
    h = eb.ebic_load_matrix(A)
    try:
        s = eb.ebic_surrogate_create(h, 8, 0)
        try:
            d_seq, d_len = _device_series([np.array([C - 3, C - 2, C - 1])], 8)
            out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
            eb.ebic_surrogate_predict(s, d_seq, d_len, 8, 1, out)
            assert np.isfinite(out.cpu().numpy()).all()
        finally:
            eb.ebic_surrogate_free(s)
    finally:
        eb.ebic_free(h)
    with pytest.raises(eb.EbicError) as e:
        eb.ebic_load_matrix(np.zeros((4, C + 1), np.float32))
    assert e.value.status == 1
