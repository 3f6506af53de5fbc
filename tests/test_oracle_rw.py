"""Pins of the constrained random-walk replacement kernel (the paper's RW
baseline): stationarity of the uniform law on a constrained set, the
Metropolis prior ratio under a Gaussian prior, a whole-run evidence against
the closed form, and the cost comparison with HRSS on an ill-conditioned
Gaussian (App. "Slice sampling vs random walk": RW needs more evaluations per
moved point, with a far larger spread)."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from closed_forms import box_gauss_logZ


def test_rw_leaves_uniform_invariant_in_disc():
    # constrained set: the unit-box part of {|x - 0.5| < 0.35}, flat prior
    pb = O.Problem(("box", np.zeros(2), np.ones(2)), "gauss", mu=np.full(2, 0.5), sigma=0.1)
    lstar = pb.loglik(np.array([0.5 + 0.35, 0.5]))
    L = 0.15 * np.eye(2)
    rng = np.random.default_rng(5)
    rs = []
    for c in range(1500):
        while True:
            x = rng.uniform(size=2)
            if pb.loglik(x) > lstar:
                break
        lx = pb.loglik(x)
        for s in range(8):
            x, lx, cnt = O.rw_step(pb, L, 1.2, lstar, 3, 0, 0, c, s, x, lx)
            assert lx > lstar
        rs.append(np.sum((x - 0.5) ** 2) / 0.35 ** 2)
    # uniform in a disc: r^2 / R^2 ~ U(0, 1)
    assert stats.kstest(rs, "uniform").pvalue > 1e-3


def test_rw_metropolis_prior_ratio():
    """Under a Gaussian prior and no constraint the kernel samples the prior."""
    pb = O.Problem(("gauss", np.zeros(1), np.ones(1)), "flat")
    xs = []
    x, lx = np.zeros(1), 0.0
    for s in range(6000):
        x, lx, _ = O.rw_step(pb, np.eye(1), 2.4, -np.inf, 9, 0, 0, 0, s, x, lx)
        xs.append(x[0])
    xs = np.array(xs[500::5])
    assert stats.kstest(xs, "norm").pvalue > 1e-3


def test_rw_run_evidence():
    mu, s = np.full(2, 0.5), 0.1
    pb = O.Problem(("box", np.zeros(2), np.ones(2)), "gauss", mu=mu, sigma=s)
    truth = box_gauss_logZ(mu, s, np.zeros(2), np.ones(2))
    dev = []
    for seed in range(4):
        op = O.make_opts(300, 150, 40, seed=seed, kernel=O.KERNEL_RW)
        r = O.run(pb, op)
        n = r["n_dead"]
        lz, err, _ = O.finalise(r["logL"][:n], r["nlive"][:n], 100, seed, 0)
        dev.append((lz - truth) / err)
    assert np.all(np.abs(dev) < 4.0), dev


def test_rw_cost_spread_exceeds_hrss():
    """Constrained set: a Gaussian contour (ball of radius 2 in d = 10),
    points started uniformly in it, both kernels with the live-set-matched
    metric.  HRSS evaluations per step are concentrated; the random walk's
    evaluations until it moves have a heavy, geometric tail."""
    d = 10
    pb = O.Problem(("box", np.full(d, -10.0), np.full(d, 10.0)), "gauss", mu=np.zeros(d), sigma=1.0)
    R = 2.0
    lstar = pb.loglik(np.r_[R, np.zeros(d - 1)])
    L = R / np.sqrt(d + 2) * np.eye(d)            # covariance of the uniform ball
    rng = np.random.default_rng(1)
    rw, hr = [], []
    for c in range(300):
        z = rng.standard_normal(d)
        x = z / np.linalg.norm(z) * rng.uniform() ** (1 / d) * R
        lx = pb.loglik(x)
        tries = 0
        for s in range(500):
            _, _, cnt = O.rw_step(pb, L, 2.38 / np.sqrt(d), lstar, 4, 0, 0, c, s, x, lx)
            tries += 1
            if cnt["accepts"]:
                break
        rw.append(tries)
        _, _, cnt = O.hrss_step(pb, L, 1.0, 0, lstar, 4, 0, 0, c, 0, x, lx)
        hr.append(cnt["evals"])
    rw, hr = np.array(rw), np.array(hr)
    assert rw.std() > 2.0 * hr.std()
    assert np.percentile(rw, 95) > np.percentile(hr, 95)


@pytest.mark.parametrize("scale", [0.3, 2.38 / np.sqrt(3)])
def test_rw_proposal_is_scaled_metric_step(scale):
    """Sec. 3.1 random walk: y = x + s L z with z ~ N(0, I); on an
    unconstrained flat problem every proposal is taken, so (y - x) / s has
    covariance L L^T (here diag(4, 1, 0.25)) and |L^-1 (y - x)|^2 / s^2 is
    chi-square with d degrees of freedom."""
    d = 3
    pb = O.Problem(("box", np.full(d, -1e6), np.full(d, 1e6)), "flat")
    L = np.diag([2.0, 1.0, 0.5])
    Linv = np.linalg.inv(L)
    n = 4000
    q = np.empty(n)
    dev = np.empty((n, d))
    for c in range(n):
        x0 = np.zeros(d)
        y, _, cnt = O.rw_step(pb, L, scale, -np.inf, 21, 0, 0, c, 0, x0, 0.0)
        assert cnt["accepts"] == 1
        dev[c] = (y - x0) / scale
        q[c] = np.sum((Linv @ dev[c]) ** 2)
    assert stats.kstest(q, "chi2", args=(d,)).pvalue > 1e-3
    assert np.allclose(np.var(dev, axis=0), np.diag(L) ** 2, rtol=0.1)


def test_rw_default_scale_is_2_38_over_sqrt_d():
    """With no scale given, the random walk proposes with s = 2.38 / sqrt(d)
    (the optimal-scaling rule the RW baseline is run with): on an
    unconstrained flat problem one step moves every chain by s L z, so the
    mean of |L^-1 (y - x)|^2 over the chains is s^2 d."""
    d, m, k = 4, 3000, 1500
    pb = O.Problem(("box", np.full(d, -1e6), np.full(d, 1e6)), "flat")
    rng = np.random.default_rng(3)
    x = rng.normal(size=(m, d)) * np.array([1.0, 2.0, 0.5, 3.0])
    logL = np.zeros(m)
    logL[:k] = -1.0  # the first k slots die; every survivor sits at 0 > logL*
    op = O.make_opts(m, k, 1, seed=8, kernel=O.KERNEL_RW)
    (_, _, _, _, _), tr = O.step(pb, op, 0, x, logL, np.full(m, -np.inf), -np.inf, 0.0)
    assert np.all(tr["accepts"] == 1)
    dlt = tr["new_x"] - x[tr["parent"]]
    q = np.sum(np.linalg.solve(tr["L"], dlt.T) ** 2, axis=0)
    s2 = q.mean() / d
    assert abs(np.sqrt(s2) - 2.38 / np.sqrt(d)) < 0.05 * 2.38 / np.sqrt(d)
