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
