"""Pins of the checker's selection, metric, resampling and HRSS step against
brute force, library routines and the paper's slice-sampling theorems."""
import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from conftest import paper_value


# ---------------- selection (Sec. 3.1 (i); Algorithm 1) -------------------

def test_select_matches_lexsort_with_ties():
    rng = np.random.default_rng(0)
    for trial in range(20):
        m = int(rng.integers(3, 60))
        k = int(rng.integers(1, m))
        logL = np.round(rng.standard_normal(m), 1)  # many ties
        logL[rng.integers(0, m)] = -np.inf
        dead, surv, ls = O.select(logL, k)
        order = np.lexsort((np.arange(m), logL))
        assert list(dead) == list(order[:k])
        assert list(surv) == sorted(order[k:])
        assert ls == logL[order[k - 1]]


# ---------------- metric (Sec. 3.2 "Direction metric") ---------------------

def test_covariance_matches_numpy():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 6)) @ rng.standard_normal((6, 6)) + 3.0
    assert np.allclose(O.covariance(X), np.cov(X.T, ddof=1), rtol=1e-12, atol=1e-12)


def test_metric_is_cholesky_of_regularised_covariance():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((80, 5)) * np.array([1, 2, 0.1, 5, 0.01])
    L, st = O.metric(X, eps=1e-6)
    S = np.cov(X.T, ddof=1)
    S = S + 1e-6 * np.trace(S) / 5 * np.eye(5)
    assert st == 0
    assert np.allclose(L, np.linalg.cholesky(S), rtol=1e-10, atol=1e-14)
    assert np.allclose(np.triu(L, 1), 0)


def test_metric_degenerate_live_set_is_identity():
    X = np.tile(np.array([0.25, 0.5, 0.75]), (20, 1))  # exact mean: zero covariance
    L, st = O.metric(X)
    assert st == 1 and np.array_equal(L, np.eye(3))


# ---------------- resampling (Sec. 3.1 (ii)) -------------------------------

def test_parents_uniform_over_survivors():
    m, k = 400, 200
    surv = np.arange(0, 2 * (m - k), 2, dtype=np.int32)  # arbitrary slot ids
    counts = np.zeros(m - k)
    for it in range(60):
        par = O.parents(9, 0, it, m, k, surv)
        assert np.all(np.isin(par, surv))
        counts += np.bincount(par // 2, minlength=m - k)
    assert stats.chisquare(counts).pvalue > 1e-3


# ---------------- HRSS step theory (App. E) --------------------------------

def _interval_problem(ell):
    return O.Problem(("box", np.zeros(1), np.full(1, float(ell))), "flat")


@pytest.mark.parametrize("w", [2.0, 5.0, 13.5, 30.0])
def test_hrss_cost_theorem_on_interval(w):
    """Theorem 'Computational cost': on a slice [0, ell],
    E[N_out | ell] = ell / w and E[N_shrink | ell] = 1 + 2 phi(w / ell)."""
    ell, _ = paper_value("hrss_interval_ell")
    pb = _interval_problem(ell)
    rng = np.random.default_rng(int(w * 10))
    n = 6000
    outs, shr = np.empty(n), np.empty(n)
    for i in range(n):
        x0 = rng.uniform(0, ell)
        _, _, c = O.hrss_step(pb, np.eye(1), w, 0, -np.inf, 3, 0, 0, i, 0, [x0], 0.0)
        assert c["accepts"] == 1 and c["cap_out"] == 0
        outs[i], shr[i] = c["expansions"], c["shrinks"]
    e_out, e_shr = ell / w, 1 + 2 * O.phi(w / ell)
    assert abs(outs.mean() - e_out) < 4 * outs.std() / np.sqrt(n) + 1e-9
    assert abs(shr.mean() - e_shr) < 4 * shr.std() / np.sqrt(n)


def test_hrss_accepted_point_uniform_on_chord():
    ell = 10.0
    pb = _interval_problem(ell)
    xs = [O.hrss_step(pb, np.eye(1), 4.0, 0, -np.inf, 5, 0, 0, i, 0, [2.5], 0.0)[0][0]
          for i in range(4000)]
    assert stats.kstest(np.array(xs) / ell, "uniform").pvalue > 1e-3


def test_hrss_leaves_uniform_invariant_in_square():
    """Stationarity: started from the uniform law on the constrained set, the
    HRSS kernel keeps it (App. B.4: the kernel leaves its target invariant)."""
    pb = O.Problem(("box", np.zeros(2), np.ones(2)), "flat")
    L = np.array([[0.3, 0.0], [0.1, 0.25]])
    rng = np.random.default_rng(11)
    pts = []
    for c in range(1500):
        x, lx = rng.uniform(size=2), 0.0
        for s in range(6):
            x, lx, _ = O.hrss_step(pb, L, 1.0, 0, -np.inf, 1, 0, 0, c, s, x, lx)
        pts.append(x)
    pts = np.array(pts)
    for i in range(2):
        assert stats.kstest(pts[:, i], "uniform").pvalue > 1e-3


def test_hrss_evals_decompose():
    """Every logical evaluation is an initial bracket end, an expansion or a
    shrinkage proposal: evals = expansions + (2 - capped sides) + shrinks."""
    pb = O.Problem(("box", np.zeros(3), np.ones(3)), "gauss", mu=np.full(3, 0.5), sigma=0.1)
    x = np.full(3, 0.5)
    lx = pb.loglik(x)
    for s in range(50):
        x, lx, c = O.hrss_step(pb, 0.1 * np.eye(3), 0.7, 0, lx - 2.0, 2, 0, 0, 0, s, x, lx)
        assert c["evals"] == c["expansions"] + 2 - c["cap_out"] + c["shrinks"]


def test_step_out_cap_and_shrink_cap():
    # tiny width on a long flat slice: stepping-out stops at 10 per side
    pb = O.Problem(("box", np.zeros(1), np.full(1, 1000.0)), "flat")
    _, _, c = O.hrss_step(pb, np.eye(1), 1.0, 0, -np.inf, 0, 0, 0, 0, 0, [500.0], 0.0)
    assert c["expansions"] == 20 and c["cap_out"] == 2 and c["accepts"] == 1
    # plateau at the threshold: logL = 0 is never > logL* = 0, so every
    # proposal fails and the step ends as a null move after 100 proposals
    x0 = np.array([500.0])
    x, lx, c = O.hrss_step(pb, np.eye(1), 1.0, 0, 0.0, 0, 0, 0, 0, 0, x0, 0.0)
    assert c["nulls"] == 1 and c["shrinks"] == 100 and c["evals"] == 102
    assert x[0] == 500.0


def test_u_star_matches_paper_and_lambert_w():
    val, digits = paper_value("u_star")
    u = O.u_star()
    assert abs(u - val) < 0.5 * 10**-digits
    lw = -1 - special.lambertw(-np.exp(-1.5), k=-1).real
    assert abs(u - lw) < 1e-12
    # and it minimises the fixed-slice cost 1/u + 1 + 2 phi(u)
    grid = np.linspace(0.5, 3.0, 2501)
    cost = [1 / g + 1 + 2 * O.phi(g) for g in grid]
    assert abs(grid[int(np.argmin(cost))] - u) < 2e-3


def test_kappa_inf_matches_paper():
    val, digits = paper_value("kappa_inf")
    assert abs(O.kappa_inf() - val) < 0.5 * 10**-digits


def test_mean_chord_matches_monte_carlo_and_asymptotics():
    rng = np.random.default_rng(7)
    for d in (2, 5):
        R = np.sqrt(d + 2.0)
        n = 200000
        g = rng.standard_normal((n, d))
        x = g / np.linalg.norm(g, axis=1, keepdims=True) * R * rng.uniform(size=(n, 1)) ** (1 / d)
        v = rng.standard_normal((n, d))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        b = np.sum(x * v, axis=1)
        chord = 2 * np.sqrt(b * b - (np.sum(x * x, axis=1) - R * R))
        assert abs(O.mean_chord_ball(d, R) - chord.mean()) < 4 * chord.std() / np.sqrt(n)
    # Lemma "mean chord length in ellipsoids": E[l] -> 4 R sqrt(2/(pi d))
    d = 400
    assert abs(O.mean_chord_ball(d, 1.0) / (4 * np.sqrt(2 / (np.pi * d))) - 1) < 5e-3


@pytest.mark.parametrize("dir_norm,scale", [(0, 2.5), (1, 2.5), (0, 0.8)])
def test_direction_normalisation_sets_the_slice_scale(dir_norm, scale):
    """Reading C5: by default v = L z / |z|, so the bracket width w acts in
    whitened units and on a slice of length ell the cost theorem holds with
    ell / s (L = [[s]]); the literal v = d~ / |d~| (dir_norm 1) keeps ell."""
    ell, w = 10.0, 2.0
    pb = _interval_problem(ell)
    rng = np.random.default_rng(17 + dir_norm)
    n = 4000
    outs = np.empty(n)
    for i in range(n):
        x0 = rng.uniform(0, ell)
        _, _, c = O.hrss_step(pb, np.array([[scale]]), w, dir_norm, -np.inf, 9, 0, 0, i, 0, [x0], 0.0)
        outs[i] = c["expansions"]
    ell_eff = ell / scale if dir_norm == 0 else ell
    assert abs(outs.mean() - ell_eff / w) < 4 * outs.std() / np.sqrt(n) + 1e-9
