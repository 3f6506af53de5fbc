"""Pin of the checker's GP path: the NS evidence of the GP hyperparameter
posterior (RBF + white kernel, log-uniform priors) against brute-force 3-D
Gauss-Legendre quadrature of the same marginal likelihood."""
import numpy as np
import pytest

import oracle as O
from closed_forms import gp_quadrature_logZ
from paper_2601_23252_gb300 import workloads as W


@pytest.fixture(scope="module")
def gp_small():
    wl = W.gp_d3(seed=2, n=24).with_(n_live=200, k=100)
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    truth = gp_quadrature_logZ(pb.loglik, wl.a, wl.b, panels=10, order=6)
    return wl, pb, truth


def test_quadrature_is_converged(gp_small):
    wl, pb, truth = gp_small
    coarse = gp_quadrature_logZ(pb.loglik, wl.a, wl.b, panels=8, order=5)
    assert abs(coarse - truth) < 0.02


def test_gp_evidence_matches_quadrature(gp_small):
    wl, pb, truth = gp_small
    for seed in (0, 1):
        op = O.make_opts(wl.n_live, wl.k, wl.p, seed=seed, tol=1e-3)
        r = O.run(pb, op)
        lz, err, _ = O.finalise(r["logL"], r["nlive"], 100, seed, 0)
        assert abs(lz - truth) < 3.5 * err + 0.02, (lz, err, truth)


def _golden_rows(name):
    from conftest import golden_path
    return [l.split() for l in open(golden_path(name)) if not l.startswith("#") and l.strip()]


def test_full_size_checker_runs_match_quadrature():
    """The checker's 8 full-size GP runs (n = 256 data of gp_d3 seed 0, m = 500,
    k = 250, p = 15; tests/golden/oracle_gp_d3_logz.txt) against brute-force
    quadrature of the same FP64 marginal likelihood in the posterior's
    principal axes (tests/golden/gp_d3_quadrature.txt): every run within 3.5
    of its own reported error, the mean within three standard errors."""
    truth = float([r for r in _golden_rows("gp_d3_quadrature.txt") if r[0] == "gp_d3_seed0_logZ"][0][1])
    rows = np.array([[float(x) for x in r] for r in _golden_rows("oracle_gp_d3_logz.txt")])
    lz, err = rows[:, 1], rows[:, 2]
    assert len(lz) == 8
    se = lz.std(ddof=1) / np.sqrt(len(lz))
    assert np.all(np.abs(lz - truth) < 3.5 * err + 0.02)
    assert abs(lz.mean() - truth) < 3 * se + 0.05
