"""Pins of the time-to-solution statistics (Sec. IV, Algorithm 3) in the oracle,
and the library's host implementation of them checked against the oracle bit
for bit (host code: no GPU needed)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("a,b", [(0.5, 0.5), (0.5, 100.5), (3.5, 97.5), (50.5, 50.5), (0.5, 5000.5)])
def test_beta_sampler_matches_the_beta_distribution(orc, a, b):
    """The posterior sampler against the Beta law itself: mean, variance and a
    Kolmogorov-Smirnov test against scipy's Beta CDF."""
    stats = pytest.importorskip("scipy.stats")
    n = 200_000
    x = orc.beta_samples(a, b, n, 11)
    mean = a / (a + b)
    var = a * b / ((a + b) ** 2 * (a + b + 1))
    assert abs(x.mean() - mean) < 5 * np.sqrt(var / n)
    assert abs(x.var() / var - 1) < 0.03
    assert stats.kstest(x, stats.beta(a, b).cdf).pvalue > 1e-4


def test_percentile_is_linear_interpolation(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 100):
        v = rng.standard_normal(n)
        for q in (0, 5, 50, 80, 95, 100, 37.3):
            assert orc.percentile(v, q) == pytest.approx(np.percentile(v, q), rel=1e-14, abs=1e-14)


def test_bootstrap_degenerate_posteriors(orc):
    """Posteriors concentrated at theta (10^9 runs): every bootstrap sample of
    identical instances is tau R99(theta); theta = 1 needs one run; theta > 0.99
    is clamped to one run."""
    theta, tau = 0.02, 1e-3
    r = np.full(5, 10 ** 9)
    y = (r * theta).astype(np.int64)
    s = orc.tts_bootstrap(y, r, tau, 80, 200, 1)
    assert np.allclose(s, tau * np.log(0.01) / np.log(1 - theta), rtol=1e-3)
    assert np.allclose(orc.tts_bootstrap(r, r, tau, 50, 50, 2), tau)
    assert np.allclose(orc.tts_bootstrap((r * 0.995).astype(np.int64), r, tau, 50, 50, 2), tau)


def test_bootstrap_percentile_of_a_known_population(orc):
    """Well-determined instances with theta spread over a range: the bootstrap
    distribution of the q-th percentile of R99 centres on the q-th percentile of
    the population of R99 values (resampling the instances only)."""
    rng = np.random.default_rng(5)
    I = 400
    theta = rng.uniform(0.005, 0.3, I)
    r = np.full(I, 10 ** 8)
    y = np.rint(theta * r).astype(np.int64)
    r99 = np.log(0.01) / np.log(1 - y / r)
    for q in (50, 80):
        s = orc.tts_bootstrap(y, r, 1.0, q, 2000, 9)
        assert abs(np.median(s) / np.percentile(r99, q) - 1) < 0.03
        # the spread matches plain resampling of the population
        boot = [np.percentile(rng.choice(r99, I), q) for _ in range(2000)]
        assert abs(np.std(s) / np.std(boot) - 1) < 0.15


def test_library_bootstrap_equals_oracle(orc):
    """da_tts_bootstrap (library host code) reproduces the oracle bit for bit."""
    import ctypes
    from paper_1806_08815_gb300 import build, binding
    build.build()
    rng = np.random.default_rng(8)
    r = rng.integers(1, 500, 37)
    y = rng.integers(0, r + 1)
    y[:3] = 0
    y[3:5] = r[3:5]
    for q, B, seed in ((50, 300, 1), (80, 120, 2 ** 40 + 5), (95, 64, 3)):
        got = binding.da_tts_bootstrap(y, r, 2.5e-3, q, B, seed)
        ref = orc.tts_bootstrap(y, r, 2.5e-3, q, B, seed)
        assert np.array_equal(got, ref)
    v = rng.standard_normal(1001)
    assert np.array_equal(binding.da_percentiles(v, [0, 5, 50, 80, 85, 100]),
                          [orc.percentile(v, q) for q in (0, 5, 50, 80, 85, 100)])
    with pytest.raises(binding.DAError):
        binding.da_tts_bootstrap([5], [3], 1.0, 50, 10, 0)


def test_best_sweep_count_picks_the_lowest_mean(orc):
    """Longer anneals raise the hit rate but cost more per run: the helper returns
    the sweep count whose bootstrap TTS distribution has the lowest mean."""
    from paper_1806_08815_gb300 import build, tuning
    build.build()
    I = 30
    runs = np.full(I, 100)
    cand = {10: (np.full(I, 1), runs, 1.0), 100: (np.full(I, 40), runs, 10.0), 1000: (np.full(I, 99), runs, 100.0)}
    best, stats = tuning.best_sweep_count(cand, q=50, B=400, seed=1)
    # R99 at theta = 0.01, 0.4, 0.99 (posterior means close): 458, 9.0, 1 runs
    assert best == 100
    assert stats[100]["p5"] <= stats[100]["mean"] <= stats[100]["p95"]
    assert stats[10]["mean"] > stats[100]["mean"] and stats[1000]["mean"] > stats[100]["mean"]
