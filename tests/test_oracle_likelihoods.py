"""Pins of the checker's priors and likelihoods against scipy library routines."""
import numpy as np
from scipy import special, stats

import oracle as O
from paper_2601_23252_gb300 import workloads as W


def test_gauss_matches_scipy_mvn():
    rng = np.random.default_rng(1)
    d = 7
    mu = rng.uniform(size=d)
    pb = O.Problem(("box", np.zeros(d), np.ones(d)), "gauss", mu=mu, sigma=0.3)
    for _ in range(20):
        x = rng.uniform(size=d)
        want = stats.multivariate_normal(mu, 0.09 * np.eye(d)).logpdf(x)
        assert abs(pb.loglik(x) - want) < 1e-10 * max(1, abs(want))


def test_gmm_matches_scipy_mixture():
    wl = W.gmm_d32(seed=3)
    pb = O.Problem(("box", wl.a, wl.b), "gmm", **wl.oracle_kwargs())
    rng = np.random.default_rng(2)
    comps = [stats.multivariate_normal(m, wl.sigma**2 * np.eye(wl.d)) for m in wl.mu]
    for i in range(10):
        x = wl.mu[i % 4] + 0.03 * rng.standard_normal(wl.d)
        want = special.logsumexp([c.logpdf(x) for c in comps]) - np.log(4)
        assert abs(pb.loglik(x) - want) < 1e-9 * max(1, abs(want))


def test_logreg_matches_scipy_log_expit():
    wl = W.logreg_d100(seed=0, n_rows=500, d=10)
    pb = O.Problem(("gauss", wl.a, wl.b), "logreg", **wl.oracle_kwargs())
    rng = np.random.default_rng(3)
    X = wl.X.astype(np.float64)
    for _ in range(10):
        x = rng.standard_normal(wl.d)
        z = X @ x
        want = np.sum(wl.y * special.log_expit(z) + (1 - wl.y) * special.log_expit(-z))
        assert abs(pb.loglik(x) - want) < 1e-9 * abs(want)


def test_gp_matches_scipy_mvn():
    wl = W.gp_d3(seed=1, n=40)
    pb = O.Problem(("box", wl.a, wl.b), "gp", **wl.oracle_kwargs())
    for th in [(0.0, 0.0, np.log(0.1)), (np.log(2.0), np.log(0.5), np.log(0.3)),
               (np.log(0.05), np.log(3.0), np.log(0.01))]:
        ell, amp, sn = np.exp(th)
        K = amp**2 * np.exp(-np.subtract.outer(wl.t, wl.t) ** 2 / (2 * ell**2)) + sn**2 * np.eye(wl.t.size)
        want = stats.multivariate_normal(np.zeros(wl.t.size), K).logpdf(wl.y)
        assert abs(pb.loglik(np.array(th)) - want) < 1e-7 * max(1, abs(want))


def test_gp_breakdown_is_minus_inf():
    # an indefinite kernel (negative noise variance cannot arise; force
    # breakdown with a huge lengthscale and no noise) reads as -inf, not NaN
    wl = W.gp_d3(seed=1, n=60)
    pb = O.Problem(("box", wl.a, wl.b), "gp", **wl.oracle_kwargs())
    v = pb.loglik(np.array([np.log(1e4), np.log(10.0), np.log(1e-12)]))
    assert v == -np.inf or np.isfinite(v)
    assert not np.isnan(v)


def test_priors_match_scipy():
    d = 4
    rng = np.random.default_rng(4)
    a, b = rng.uniform(-1, 0, d), rng.uniform(1, 2, d)
    box = O.Problem(("box", a, b), "flat")
    x = (a + b) / 2
    assert abs(box.log_prior(x) - np.sum(stats.uniform(a, b - a).logpdf(x))) < 1e-12
    assert box.in_support(x) and not box.in_support(b + 1e-9)
    assert box.log_prior(b + 1.0) == -np.inf
    g = O.Problem(("gauss", a, b), "flat")
    assert abs(g.log_prior(x) - np.sum(stats.norm(a, b).logpdf(x))) < 1e-12


def test_rastrigin_mixture_endpoints():
    d = 2
    r = 5.14
    x = np.array([0.3, -1.2])
    pure_gauss = O.Problem(("box", -r * np.ones(d), r * np.ones(d)), "rastrigin", alpha=1.0)
    assert abs(pure_gauss.loglik(x) - (-0.5 * x @ x)) < 1e-12
    pure_rast = O.Problem(("box", -r * np.ones(d), r * np.ones(d)), "rastrigin", alpha=0.0)
    # integer lattice points are the Rastrigin maxima: g = 1
    assert abs(pure_rast.loglik(np.array([1.0, -2.0]))) < 1e-12
