"""Pins of the posterior expectations and Fisher-identity gradients of log Z
(d log Z / d theta = E_post[d/dtheta (log L + log Pi)]): the oracle's
estimator applied to a quadrature grid whose weights are the exact posterior
reproduces the derivative of the closed-form (or quadrature) evidence; and a
few oracle NS runs agree with the closed form within their statistical error."""
import numpy as np
import pytest
from scipy.special import logsumexp, ndtr

import oracle as O


def _phi(z):
    return np.exp(-0.5 * z * z) / np.sqrt(2 * np.pi)


def _grid(lo, hi, n):
    g = lo + (hi - lo) * (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], 1), ((hi - lo) / n) ** 2


def _post_weights(pb, x, log_prior):
    lw = pb.loglik(x) + log_prior
    return lw - logsumexp(lw)


def test_gauss_box_sigma_and_mu_on_exact_posterior_grid():
    mu, s = np.array([0.3, 0.7]), 0.3
    pb = O.Problem(("box", np.zeros(2), np.ones(2)), "gauss", mu=mu, sigma=s)
    x, _ = _grid(0.0, 1.0, 600)
    lw = _post_weights(pb, x, 0.0)
    a, b = -mu / s, (1 - mu) / s
    Zi = ndtr(b) - ndtr(a)
    dsig = np.sum((-_phi(b) * b + _phi(a) * a) / s / Zi)
    dmu = (_phi(a) - _phi(b)) / (s * Zi)
    assert O.posterior_expectation(pb, O.GRAD_LIK_SIGMA, x, lw)[0] == pytest.approx(dsig, rel=2e-4, abs=2e-5)
    assert np.allclose(O.posterior_expectation(pb, O.GRAD_LIK_MU, x, lw), dmu, rtol=2e-4, atol=2e-5)
    # the posterior mean of a truncated normal
    mean = mu + s * (_phi(a) - _phi(b)) / Zi
    assert np.allclose(O.posterior_expectation(pb, O.MOMENT_MEAN, x, lw), mean, rtol=1e-5, atol=1e-6)


def test_mixture_sigma_and_means_on_exact_posterior_grid():
    mu, s = np.array([[0.25, 0.35], [0.7, 0.6]]), 0.15
    pb = O.Problem(("box", np.zeros(2), np.ones(2)), "gmm", mu=mu, sigma=s)
    x, _ = _grid(0.0, 1.0, 700)
    lw = _post_weights(pb, x, 0.0)

    def lnZ(mu_, s_):
        a, b = -mu_ / s_, (1 - mu_) / s_
        return np.log(np.mean(np.prod(ndtr(b) - ndtr(a), axis=1)))

    h = 1e-5
    dsig = (lnZ(mu, s + h) - lnZ(mu, s - h)) / (2 * h)
    dmu = np.zeros_like(mu)
    for c in range(2):
        for i in range(2):
            e = np.zeros_like(mu)
            e[c, i] = h
            dmu[c, i] = (lnZ(mu + e, s) - lnZ(mu - e, s)) / (2 * h)
    assert O.posterior_expectation(pb, O.GRAD_LIK_SIGMA, x, lw)[0] == pytest.approx(dsig, rel=5e-4, abs=5e-5)
    assert np.allclose(O.posterior_expectation(pb, O.GRAD_LIK_MU, x, lw).reshape(2, 2), dmu, rtol=5e-4, atol=5e-5)


def test_prior_log_precision_on_exact_posterior_grid():
    # Gaussian prior N(a, diag b^2), Gaussian likelihood N(x; muL, sL^2 I):
    # Z = N(muL; a, sL^2 + b^2 e^{-lambda}), d lnZ/dlambda = 1/2 sum b^2 (1/v - (muL - a)^2 / v^2)
    a, b, muL, sL = np.array([0.1, -0.2]), np.array([1.0, 0.7]), np.array([0.8, 0.4]), 0.3
    pb = O.Problem(("gauss", a, b), "gauss", mu=muL, sigma=sL)
    x, _ = _grid(-5.0, 5.0, 800)
    logprior = np.sum(-0.5 * ((x - a) / b) ** 2 - np.log(b) - 0.5 * np.log(2 * np.pi), axis=1)
    lw = _post_weights(pb, x, logprior)
    v = sL ** 2 + b ** 2
    expect = 0.5 * np.sum(b ** 2 * (1 / v - (muL - a) ** 2 / v ** 2))
    got = O.posterior_expectation(pb, O.GRAD_PRIOR_LOG_PREC, x, lw)[0]
    assert got == pytest.approx(expect, rel=1e-4, abs=1e-5)


def _gp_loglik(t, y, th, s=1.0):
    ell, amp, sn = np.exp(th)
    K = amp ** 2 * np.exp(-(t[:, None] - t[None, :]) ** 2 / (2 * ell ** 2)) + (s * sn) ** 2 * np.eye(t.size)
    L = np.linalg.cholesky(K)
    al = np.linalg.solve(L, y)
    return -0.5 * al @ al - np.log(np.diag(L)).sum() - 0.5 * t.size * np.log(2 * np.pi)


def test_gp_noise_scale_on_posterior_grid():
    g = np.random.default_rng(7)
    t = g.uniform(0, 10, 12)
    y = np.sin(t) + 0.3 * g.standard_normal(12)
    lo, hi = np.log([0.3, 0.3, 0.05]), np.log([3.0, 3.0, 1.0])
    pb = O.Problem(("box", lo, hi), "gp", t=t, y=y)
    n = 14
    ax = [lo[q] + (hi[q] - lo[q]) * (np.arange(n) + 0.5) / n for q in range(3)]
    th = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    ll = pb.loglik(th)
    lw = ll - logsumexp(ll)
    # d/ds lnZ at s = 1 by central differences of the same quadrature
    h = 1e-4
    lp = np.array([_gp_loglik(t, y, q, 1 + h) for q in th])
    lm = np.array([_gp_loglik(t, y, q, 1 - h) for q in th])
    fd = (logsumexp(lp) - logsumexp(lm)) / (2 * h)
    got = O.posterior_expectation(pb, O.GRAD_GP_NOISE_SCALE, th, lw)[0]
    assert got == pytest.approx(fd, rel=1e-5, abs=1e-6)


def test_gauss_box_sigma_from_ns_runs():
    """Six oracle NS runs: the Fisher estimate of d lnZ/dsigma over the
    weighted dead points agrees with the closed form within its spread."""
    mu, s = np.array([0.3, 0.7]), 0.3
    pb = O.Problem(("box", np.zeros(2), np.ones(2)), "gauss", mu=mu, sigma=s)
    a, b = -mu / s, (1 - mu) / s
    truth = np.sum((-_phi(b) * b + _phi(a) * a) / s / (ndtr(b) - ndtr(a)))
    est = []
    for seed in range(6):
        op = O.make_opts(200, 100, 10, seed=seed)
        r = O.run(pb, op)
        n = r["n_dead"]
        lz, err, lw = O.finalise(r["logL"][:n], r["nlive"][:n], 100, seed, 0)[:3]
        est.append(O.posterior_expectation(pb, O.GRAD_LIK_SIGMA, r["x"][:n], lw)[0])
    est = np.array(est)
    se = est.std(ddof=1) / np.sqrt(est.size)
    assert abs(est.mean() - truth) <= 4 * se + 0.05, (est, truth)
