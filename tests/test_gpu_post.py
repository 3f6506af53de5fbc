"""Device posterior expectations and Fisher-identity gradients of log Z:
(i) the kernel equals the checker's estimator applied to the GPU's own dead
points and weights; (ii) the gradient agrees with the closed form over seeds;
(iii) the torch.autograd.Function; (iv) the prior log-precision gradient of a
logistic regression against finite differences of log Z."""
import numpy as np
import pytest
import torch
from scipy.special import ndtr

import oracle as O
from paper_2601_23252_gb300 import autograd as NA
from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _phi(z):
    return np.exp(-0.5 * z * z) / np.sqrt(2 * np.pi)


def _gauss_box(seed, mu=(0.3, 0.7), sigma=0.3):
    mu = np.asarray(mu, float)
    d = mu.size
    return W.Workload("gauss_box", d, "box", np.zeros(d), np.ones(d), "gauss", 300, 150, 5 * d,
                      sigma=sigma, mu=mu[None, :], seed=seed)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _checker_on_gpu_points(wl, s, kind, run=0):
    """The checker's estimator on the dead points and weights the GPU produced,
    with the problem's constants as the device holds them (FP32)."""
    dd = s.dead(run)
    kw = wl.oracle_kwargs()
    if "mu" in kw:
        kw["mu"] = _f32(kw["mu"])
    if wl.lik == "gp":
        kw["t"], kw["y"] = _f32(kw["t"]), _f32(kw["y"])
    pb = O.Problem((wl.prior, _f32(wl.a), _f32(wl.b)), wl.lik, **kw)
    return O.posterior_expectation(pb, kind, dd["x"].astype(np.float64), dd["log_w"])


@pytest.mark.parametrize("case", ["gauss_box", "gmm", "gauss_prior"])
def test_kernel_equals_checker_formula(gpu_lib, case):
    if case == "gauss_box":
        wl = _gauss_box(3)
        kinds = [native.GRAD_LIK_SIGMA, native.GRAD_LIK_MU, native.MOMENT_MEAN]
    elif case == "gmm":
        wl = W.gmm_d32(seed=2, n_live=300, k=150).with_(p=32)
        kinds = [native.GRAD_LIK_SIGMA, native.GRAD_LIK_MU, native.MOMENT_MEAN]
    else:
        wl = W.gauss20_paper(seed=4, n_live=256, k=128).with_(p=20)
        kinds = [native.GRAD_PRIOR_LOG_PREC, native.GRAD_LIK_SIGMA, native.MOMENT_MEAN]
    with native.Sampler(wl) as s:
        s.run()
        for kind in kinds:
            g = s.posterior(kind)
            ref = _checker_on_gpu_points(wl, s, kind)
            scale = max(1.0, np.abs(ref).max())
            print(f"\n{case} kind {kind}: gpu {g[:3]} checker {ref[:3]}")
            assert np.allclose(g, ref, rtol=1e-9, atol=1e-9 * scale)


def test_gp_noise_scale_kernel_equals_checker_formula(gpu_lib):
    wl = W.gp_d3(seed=1, n=48).with_(n_live=200, k=100)
    with native.Sampler(wl) as s:
        s.run()
        g = s.posterior(native.GRAD_GP_NOISE_SCALE)[0]
        ref = _checker_on_gpu_points(wl, s, native.GRAD_GP_NOISE_SCALE)[0]
    print(f"\ngp noise scale: gpu {g:.6f} checker {ref:.6f}")
    # FP32 Cholesky and triangular inverse per point against FP64
    assert g == pytest.approx(ref, rel=2e-3, abs=2e-3)


def test_sigma_and_mu_gradients_against_closed_form(gpu_lib):
    mu, s = np.array([0.3, 0.7]), 0.3
    a, b = -mu / s, (1 - mu) / s
    Zi = ndtr(b) - ndtr(a)
    t_sig = np.sum((-_phi(b) * b + _phi(a) * a) / s / Zi)
    t_mu = (_phi(a) - _phi(b)) / (s * Zi)
    wls = [_gauss_box(sd).with_(run_id=sd) for sd in range(16)]
    with native.Sampler(wls) as smp:
        smp.run()
        gs = np.array([smp.posterior(native.GRAD_LIK_SIGMA, r)[0] for r in range(16)])
        gm = np.array([smp.posterior(native.GRAD_LIK_MU, r) for r in range(16)])
    se_s = gs.std(ddof=1) / 4.0
    se_m = gm.std(0, ddof=1) / 4.0
    print(f"\nd lnZ/dsigma {gs.mean():.4f} +- {se_s:.4f} (closed form {t_sig:.4f}); "
          f"d lnZ/dmu {gm.mean(0)} +- {se_m} (closed form {t_mu})")
    assert abs(gs.mean() - t_sig) <= 4 * se_s + 0.02
    assert np.all(np.abs(gm.mean(0) - t_mu) <= 4 * se_m + 0.02)


def test_autograd_function(gpu_lib):
    base = _gauss_box(5)
    theta = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    z = NA.logz(theta, lambda v: base.with_(sigma=float(v)), native.GRAD_LIK_SIGMA)
    z.backward()
    with native.Sampler(base) as s:
        r = s.run()[0]
        g = s.posterior(native.GRAD_LIK_SIGMA)[0]
    assert z.item() == r["logZ"]
    assert theta.grad.item() == g
    # vector parameter: the mean
    m = torch.tensor([0.3, 0.7], dtype=torch.float64, requires_grad=True)
    z2 = NA.logz(m, lambda v: base.with_(mu=np.asarray(v)[None, :]), native.GRAD_LIK_MU)
    (2.0 * z2).backward()
    with native.Sampler(base) as s:
        s.run()
        gm = s.posterior(native.GRAD_LIK_MU)
    assert np.array_equal(m.grad.numpy(), 2.0 * gm)


def test_logistic_prior_log_precision_against_finite_differences(gpu_lib):
    """d lnZ/d lambda (prior sd b e^{-lambda/2}) at lambda = 0 from the Fisher
    kernel against the five-point difference of lnZ at +-h, +-2h, the same
    seeds at every lambda, at the shape of the paper's GermanCredit logistic
    regression (d = 25, N = 1000 rows).  lnZ(lambda) carries the term
    -e^lambda E|w|^2 / 2 (about -12 nat here), whose odd derivatives are all
    about -12: a central difference at h = 0.5 would be biased by h^2/6 of
    that (-0.5 nat); the five-point rule leaves h^4/30 of it (0.03)."""
    h = 0.5
    seeds = range(32)
    base = [W.logreg_d100(seed=sd, n_rows=1000, d=25, n_live=200, k=100).with_(run_id=sd) for sd in seeds]
    d = base[0].d

    def at(lam):
        return [w.with_(b=np.full(d, np.exp(-lam / 2))) for w in base]

    with native.Sampler(at(0.0)) as s:
        res = s.run()
        g = np.array([s.posterior(native.GRAD_PRIOR_LOG_PREC, r)[0] for r in range(len(base))])
    z = {}
    for q in (-2, -1, 1, 2):
        with native.Sampler(at(q * h)) as s:
            z[q] = np.array([r["logZ"] for r in s.run()])
    fd = (8.0 * (z[1] - z[-1]) - (z[2] - z[-2])) / (12.0 * h)
    diff = g - fd
    se = diff.std(ddof=1) / np.sqrt(diff.size)
    print(f"\nFisher {g.mean():.4f}, five-point differences {fd.mean():.4f}, paired se {se:.4f}, "
          f"logZ err {np.mean([r['logZ_err'] for r in res]):.3f}")
    assert abs(diff.mean()) <= 4 * se + 0.05


def test_reweighting_to_other_temperatures(gpu_lib):
    """Z(beta) = sum_i L_i^beta dX_i from the same dead points: beta = 1
    reproduces the run; beta = 0.5 against the closed form of the tempered
    box Gaussian; the Kish ESS at beta = 1 from the run's own weights."""
    mu, s = np.array([0.3, 0.7]), 0.3
    wls = [_gauss_box(sd).with_(run_id=sd) for sd in range(8)]
    beta = 0.5
    d = 2
    a, b = -mu * np.sqrt(beta) / s, (1 - mu) * np.sqrt(beta) / s
    t_half = (-0.5 * d * beta * np.log(2 * np.pi * s * s) + 0.5 * d * np.log(2 * np.pi * s * s / beta)
              + np.sum(np.log(ndtr(b) - ndtr(a))))
    dev = []
    with native.Sampler(wls) as smp:
        res = smp.run()
        for r in range(len(wls)):
            one = smp.reweight(1.0, r)
            assert one["logZ"] == pytest.approx(res[r]["logZ"], abs=1e-6)
            assert one["logZ_err"] == pytest.approx(res[r]["logZ_err"], abs=1e-6)
            lw = smp.dead(r)["log_w"]
            assert one["ess"] == pytest.approx(1.0 / np.sum(np.exp(2 * lw)), rel=1e-6)
            h = smp.reweight(beta, r)
            dev.append((h["logZ"] - t_half) / h["logZ_err"])
    dev = np.array(dev)
    print(f"\nbeta = 0.5: closed form {t_half:.4f}, dev/err {np.round(dev, 2)}")
    assert np.all(np.abs(dev) < 4.0)


def test_reweighting_with_many_trajectories_and_beta_range(gpu_lib):
    """nss_reweight runs the context's own volume simulation: a run with 300
    simulated trajectories (more than the fixed-scratch entry point takes)
    reweights at beta = 1 to its own logZ and error, its stored weights stay
    untouched, and beta outside (0, inf) is rejected."""
    wl = _gauss_box(3).with_(extra={"options": {"n_sim": 300}})
    with native.Sampler(wl) as smp:
        res = smp.run()[0]
        lw0 = smp.dead(0)["log_w"].copy()
        one = smp.reweight(1.0, 0)
        assert one["logZ"] == pytest.approx(res["logZ"], abs=1e-6)
        assert one["logZ_err"] == pytest.approx(res["logZ_err"], abs=1e-6)
        hot = smp.reweight(2.0, 0)
        assert np.isfinite(hot["logZ"]) and 1.0 < hot["ess"] <= res["n_dead"]
        assert np.array_equal(smp.dead(0)["log_w"], lw0)
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(native.NSSError) as e:
                smp.reweight(bad, 0)
            assert e.value.status == -1
