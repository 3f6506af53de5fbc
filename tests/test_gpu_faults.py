"""Failure handling on the GPU without faulting it: NaN and +inf likelihood
values, a likelihood plateau (shrinkage-cap null moves), a degenerate live
set (identity metric), a full dead-point store."""
import numpy as np
import pytest

from closed_forms import box_gauss_logZ
from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_nan_likelihood_reads_as_minus_inf(gpu_lib):
    wl = W.gauss_d2(seed=2).with_(lik="fault", extra={"fault_mode": 1, "fault_param": 0.3})
    with native.Sampler(wl) as s:
        res = s.run()[0]
        d = s.dead(0)
    assert res["status"] == 0 and res["nan_evals"] > 0
    finite = np.isfinite(d["logL"])
    assert np.all(d["x"][finite, 0] >= 0.3)
    # the evidence of the likelihood restricted to x_0 >= 0.3
    truth = box_gauss_logZ(wl.mu[0], wl.sigma, np.array([0.3, 0.0]), np.ones(2)) + np.log(0.7)
    assert abs(res["logZ"] - truth) < 4 * res["logZ_err"]


def test_plus_inf_likelihood_ends_with_an_error_status(gpu_lib):
    wl = W.gauss_d2(seed=2).with_(lik="fault", extra={"fault_mode": 2, "fault_param": 0.3,
                                                      "options": {"max_iter": 60}})
    with native.Sampler(wl) as s:
        with pytest.raises(native.NSSError) as e:
            res = s.run()
            if res[0]["status"] != 0:
                raise native.NSSError(res[0]["status"], "run status")
    assert e.value.status in (-5, -6)


def test_plateau_gives_null_moves_and_terminates(gpu_lib):
    wl = W.gauss_d2(seed=4).with_(lik="flat", mu=None)
    with native.Sampler(wl) as s:
        res = s.run()[0]
        d = s.dead(0)
    assert res["status"] == 0
    assert res["nulls"] == res["iters"] * wl.k * wl.p
    # with L = 1 the Delta-X quadrature sums the removed volume: Z = 1 - X_N,
    # log X_N = -sum 1/n over every death including the final live set
    logXN = -np.sum(1.0 / d["nlive"])
    # FP64 accumulation of FP32 exponentials: relative 1e-7 of Z
    assert abs(res["logZ_det"] - np.log1p(-np.exp(logXN))) < 1e-7
    assert abs(res["logZ"]) < 0.01


def test_degenerate_live_set_uses_identity_metric(gpu_lib):
    wl = W.gauss_d2(seed=6)
    x = np.tile(np.array([0.25, 0.75], np.float32), (wl.n_live, 1))
    logL = np.full(wl.n_live, -3.0, np.float32)
    with native.Sampler(wl) as s:
        s.import_state(0, x, logL)
        done, info = s.step()
        t = s.trace(0)
    assert info[0]["metric_status"] == 1
    assert np.array_equal(t["L"], np.eye(2, dtype=np.float32))


def test_full_dead_store_reports_capacity(gpu_lib):
    # room for two batches of k = 250 deaths but not three
    wl = W.gauss_d2(seed=7).with_(extra={"options": {"dead_capacity": 600}})
    with native.Sampler(wl) as s:
        s.step()
        s.step()
        with pytest.raises(native.NSSError) as e:
            s.step()
        assert s.n_dead() == 500
    assert e.value.status == -4


def test_bounded_device_wait_gives_up_and_the_context_stays_usable(gpu_lib):
    """A wait on an mbarrier that nothing completes (the tensor-core kernels'
    wait primitive, poll-limited) gives up and reports it; the device then
    runs a normal sampler as before."""
    assert native.wait_selftest(2000) == 2
    with pytest.raises(native.NSSError):
        native.wait_selftest(0)
    with native.Sampler(W.gauss_d2(seed=3)) as s:
        res = s.run()[0]
    assert np.isfinite(res["logZ"]) and res["n_dead"] > 0
