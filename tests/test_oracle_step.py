"""One outer iteration of the checker (Sec. 3.1 (i)-(iv); Algorithm 1):
selection, replacement and per-chain counter invariants."""
import numpy as np

import oracle as O
from paper_2601_23252_gb300 import workloads as W


def _state(wl, it_warm=2):
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed, run_id=wl.run_id, w=wl.w, tol=wl.tol)
    x, logL, birth = O.init_live(pb, op)
    st = (x, logL, birth, -np.inf, 0.0)
    for it in range(it_warm):
        st, _ = O.step(pb, op, it, *st)
    return pb, op, st


def test_step_selection_replacement_and_counters():
    wl = W.gmm_d32(seed=1, n_live=200, k=100).with_(p=8)
    pb, op, st = _state(wl)
    x, logL, birth, logZ, logX = st
    (x2, logL2, birth2, logZ2, logX2), tr = O.step(pb, op, 2, *st)
    k, m = wl.k, wl.n_live
    order = np.lexsort((np.arange(m), logL))
    assert np.array_equal(tr["dead_idx"], order[:k])
    assert tr["logLstar"] == logL[order[k - 1]]
    surv = np.sort(order[k:])
    assert np.all(np.isin(tr["parent"], surv))
    acc = tr["nulls"] < wl.p
    # every chain that moved sits strictly above the threshold
    assert np.all(tr["new_logL"][acc] > tr["logLstar"])
    # the dead slots now hold the new points, born at logL*
    assert np.array_equal(x2[tr["dead_idx"]], tr["new_x"])
    assert np.all(birth2[tr["dead_idx"]] == tr["logLstar"])
    keep = np.setdiff1d(np.arange(m), tr["dead_idx"])
    assert np.array_equal(x2[keep], x[keep]) and np.array_equal(logL2[keep], logL[keep])
    # counter identities per chain: p steps, each accepted or null
    assert np.all(tr["accepts"] + tr["nulls"] == wl.p)
    assert np.all(tr["evals"] == tr["expansions"] + 2 * wl.p - tr["cap_out"] + tr["shrinks"])
    # recorded likelihoods are the likelihoods of the recorded points
    for j in range(0, k, 17):
        assert abs(pb.loglik(tr["new_x"][j]) - tr["new_logL"][j]) < 1e-12
    # evidence: k unrolled deaths
    assert abs(logX2 - (logX - np.sum(1.0 / np.arange(m - k + 1, m + 1)))) < 1e-12
    assert logZ2 > logZ


def test_step_is_deterministic_given_counters():
    wl = W.gauss_d2(seed=4)
    pb, op, st = _state(wl, it_warm=1)
    a = O.step(pb, op, 1, *st)
    b = O.step(pb, op, 1, *st)
    for key in ("dead_idx", "parent", "evals", "new_x", "new_logL"):
        assert np.array_equal(a[1][key], b[1][key])


def test_step_metric_is_the_live_set_at_the_start():
    """Reading C4: the direction metric of an iteration is the Cholesky factor
    of the regularised covariance of all m live points before deletion."""
    wl = W.gmm_d32(seed=2, n_live=120, k=60).with_(p=3)
    pb, op, st = _state(wl, 1)
    x = st[0]
    _, tr = O.step(pb, op, 1, *st)
    L_start, _ = O.metric(x)
    assert np.array_equal(tr["L"], L_start)
    survivors = np.setdiff1d(np.arange(wl.n_live), tr["dead_idx"])
    L_surv, _ = O.metric(x[survivors])
    assert not np.allclose(tr["L"], L_surv)
