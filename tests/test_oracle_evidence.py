"""Pins of the checker's evidence bookkeeping and whole runs: volume-shrinkage
moments, quadrature identities, closed-form and quadrature evidences, the
paper's printed analytic evidence, and the run invariants."""
import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from closed_forms import box_gauss_logZ, box_gmm_logZ, gauss_gauss_logZ, rastrigin_logZ
from conftest import paper_value
from paper_2601_23252_gb300 import workloads as W


def _run(wl, seed=None, **kw):
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed if seed is None else seed,
                     run_id=wl.run_id, w=wl.w, tol=wl.tol, **kw)
    r = O.run(pb, op)
    lz, err, lw = O.finalise(r["logL"], r["nlive"], 100, op.seed, op.run_id)
    r.update(logZ=lz, err=err, log_w=lw)
    return r


# --------------- volume bookkeeping (App. D) -------------------------------

def test_unrolled_deterministic_log_volume():
    m, k = 1000, 500
    logZ, logX = -np.inf, 0.0
    for j in range(k):
        logZ, logX = O.evidence_death(0.0, m - j, logZ, logX)
    want = -np.sum(1.0 / np.arange(m - k + 1, m + 1))
    assert abs(logX - want) < 1e-13
    # with L = 1 the quadrature sums the removed volume exactly: Z = 1 - X
    assert abs(np.exp(logZ) - (1 - np.exp(logX))) < 1e-13


@pytest.mark.parametrize("m,k", [(500, 250), (1000, 100), (50, 49)])
def test_unrolled_batch_matches_beta_contraction(m, k):
    """Unrolling k deaths with n = m..m-k+1 gives the joint Beta(m-k+1, k)
    contraction (App. D.1): E[log t] = psi(m-k+1) - psi(m+1) and
    Var[log t] = psi1(m-k+1) - psi1(m+1)."""
    nlive = np.arange(m, m - k, -1)
    R = 4000
    tot = np.array([O.volume_trajectory(nlive, r, 21, 0)[-1] for r in range(R)])
    mean = special.digamma(m - k + 1) - special.digamma(m + 1)
    var = special.polygamma(1, m - k + 1) - special.polygamma(1, m + 1)
    assert abs(tot.mean() - mean) < 4 * np.sqrt(var / R)
    assert abs(tot.var(ddof=1) / var - 1) < 4 * np.sqrt(2 / (R - 1))


def test_single_death_is_beta_n_1():
    n = 7
    t = np.exp(np.array([O.volume_trajectory([n], r, 4, 1)[0] for r in range(5000)]))
    assert stats.kstest(t, stats.beta(n, 1).cdf).pvalue > 1e-3


def test_trapezoid_with_unit_likelihood_telescopes():
    """With L_i = 1 the trapezoid sum telescopes: Z^(r) = (1 + X_1 - X_N)/2."""
    nlive = np.array([5, 4, 3, 5, 4, 3, 2, 1])
    logL = np.zeros(nlive.size)
    _, _, _, lz = O.finalise(logL, nlive, 6, 8, 2, want_r=True)
    for r in range(6):
        lx = O.volume_trajectory(nlive, r, 8, 2)
        want = np.log((1 + np.exp(lx[0]) - np.exp(lx[-1])) / 2)
        assert abs(lz[r] - want) < 1e-13


def test_weights_normalised_and_geometric_mean():
    rng = np.random.default_rng(0)
    nlive = np.concatenate([np.arange(20, 10, -1)] * 3 + [np.arange(20, 0, -1)])
    logL = np.sort(rng.standard_normal(nlive.size)) * 3
    R = 9
    _, _, lw, lz = O.finalise(logL, nlive, R, 3, 0, want_r=True)
    assert abs(special.logsumexp(lw)) < 1e-12
    # brute force: per trajectory trapezoid weights, log-mean over r
    acc = np.zeros(nlive.size)
    for r in range(R):
        lx = np.concatenate([[0.0], O.volume_trajectory(nlive, r, 3, 0), [-np.inf]])
        X = np.exp(lx)
        dX = (X[:-2] - X[2:]) / 2
        acc += logL + np.log(dX)
        assert abs(special.logsumexp(logL + np.log(dX)) - lz[r]) < 1e-12
    want = acc / R
    want -= special.logsumexp(want)
    assert np.allclose(lw, want, atol=1e-12)


# --------------- whole runs against closed forms ---------------------------

def test_gauss_d2_closed_form_over_seeds():
    wl = W.gauss_d2()
    truth = box_gauss_logZ(wl.mu[0], wl.sigma, wl.a, wl.b)
    assert abs(truth - (-1.1466e-6)) < 1e-9
    res = [_run(wl, seed=s) for s in range(10)]
    lz = np.array([r["logZ"] for r in res])
    for r in res:
        assert abs(r["logZ"] - truth) < 3.5 * r["err"]
    assert abs(lz.mean() - truth) < 3 * lz.std(ddof=1) / np.sqrt(lz.size) + 0.01


def test_gauss20_paper_analytic_value():
    """App. B.2 / Table tab:overhead: 20-d Gaussian, prior N(0, I), likelihood
    N(x; 1, 0.01 I); the printed analytic evidence is -28.38."""
    val, digits = paper_value("gauss20_lnZ")
    wl = W.gauss20_paper(n_live=400, k=200)
    truth = gauss_gauss_logZ(wl.mu[0], wl.sigma, wl.a, wl.b)
    assert abs(truth - val) < 0.5 * 10**-digits
    r = _run(wl, seed=1)
    assert abs(r["logZ"] - truth) < 3.5 * r["err"]


def test_gmm_d2_closed_form():
    rng = np.random.default_rng(5)
    d = 2
    mu = rng.uniform(0.2, 0.8, size=(4, d))
    wl = W.Workload("gmm2", d, "box", np.zeros(d), np.ones(d), "gmm", 400, 200, 10,
                    sigma=0.03, mu=mu)
    truth = box_gmm_logZ(mu, 0.03, wl.a, wl.b)
    lz = np.array([_run(wl, seed=s)["logZ"] for s in range(6)])
    errs = np.array([_run(wl, seed=s)["err"] for s in range(6)])
    assert np.all(np.abs(lz - truth) < 3.5 * errs)


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
def test_rastrigin_mixture_quadrature(d, alpha):
    """App. F.3 test likelihood, uniform prior on [-5.14, 5.14]^d; evidence by
    one-dimensional quadrature, and for d = 2 by brute-force 2-D Gauss-Legendre."""
    r = 5.14
    truth = rastrigin_logZ(alpha, d)
    if d == 2:
        # composite: 40 panels x 20-point rule per axis
        xq, wq = np.polynomial.legendre.leggauss(20)
        edges = np.linspace(-r, r, 41)
        pts = np.concatenate([(e0 + e1) / 2 + (e1 - e0) / 2 * xq for e0, e1 in zip(edges[:-1], edges[1:])])
        wts = np.concatenate([(e1 - e0) / 2 * wq for e0, e1 in zip(edges[:-1], edges[1:])])
        X, Y = np.meshgrid(pts, pts, indexing="ij")
        f = np.exp(-0.5 * (X**2 + Y**2))
        g = np.exp(-20 + 10 * (np.cos(2 * np.pi * X) + np.cos(2 * np.pi * Y)))
        Z = np.sum(np.outer(wts, wts) * (alpha * f + (1 - alpha) * g)) / (2 * r) ** 2
        assert abs(np.log(Z) - truth) < 1e-8
    wl = W.Workload("rast", d, "box", -r * np.ones(d), r * np.ones(d), "flat", 400, 200, 5 * d)
    pb = O.Problem(("box", wl.a, wl.b), "rastrigin", alpha=alpha)
    vals = []
    for s in range(3):
        op = O.make_opts(400, 200, 5 * d, seed=s, tol=1e-3)
        res = O.run(pb, op)
        lz, err, _ = O.finalise(res["logL"], res["nlive"], 100, s, 0)
        assert abs(lz - truth) < 3.5 * err + 0.02
        vals.append(lz)
    assert abs(np.mean(vals) - truth) < 0.15


def test_run_invariants_and_posterior_moments():
    wl = W.gauss_d2()
    r = _run(wl, seed=3)
    m, k = wl.n_live, wl.k
    logL, birth, nlive = r["logL"], r["birth"], r["nlive"]
    # dead logL non-decreasing over the whole run
    assert np.all(np.diff(logL) >= 0)
    # every point born at a threshold lies strictly above it
    born = birth > -np.inf
    assert np.all(logL[born] > birth[born])
    # live count schedule: iterations of m..m-k+1, then m..1
    it = r["iters"]
    want = np.concatenate([np.arange(m, m - k, -1)] * it + [np.arange(m, 0, -1)])
    assert np.array_equal(nlive, want) and r["n_dead"] == it * k + m
    # deterministic final log X = -sum 1/n over all deaths
    assert abs(r["logX"] + np.sum(1.0 / nlive)) < 1e-9
    # posterior moments of the truncated normal N(0.5, 0.1^2) on [0, 1]
    w = np.exp(r["log_w"])
    assert abs(w.sum() - 1) < 1e-12
    tn = stats.truncnorm(-5, 5, loc=0.5, scale=0.1)
    ess = 1 / np.sum(w**2)
    for i in range(2):
        mean = np.sum(w * r["x"][:, i])
        var = np.sum(w * (r["x"][:, i] - mean) ** 2)
        assert abs(mean - tn.mean()) < 5 * tn.std() / np.sqrt(ess)
        assert abs(var / tn.var() - 1) < 5 * np.sqrt(2 / ess)


@pytest.mark.parametrize("live", [[0.0, 0.0, 0.0, 0.0], [0.0, -1.0, -2.0, -3.0], [1.5, -0.5, 0.2]])
def test_termination_is_the_live_fraction_threshold(live):
    """Reading C11: stop when Z_live / (Z + Z_live) < tol with Z_live = X
    times the mean live likelihood; just below the threshold stops, just
    above does not."""
    live = np.array(live)
    tol, logX = 1e-3, -2.0
    z_live = np.exp(logX) * np.mean(np.exp(live))
    for f, want in ((0.999 * tol, True), (1.001 * tol, False)):
        logZ = np.log(z_live * (1.0 / f - 1.0))
        assert O.should_stop(live, logZ, logX, tol) == want
