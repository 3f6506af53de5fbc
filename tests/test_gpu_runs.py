"""Whole runs on the GPU: evidences over 20 seeds against closed forms, the
post-hoc volume simulation against the checker on the GPU's own dead list,
run invariants and posterior moments."""
import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from closed_forms import box_gauss_logZ, box_gmm_logZ, rastrigin_logZ
from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W
from conftest import golden_path

pytestmark = pytest.mark.gpu


def _check_seeds(lz, err, truth, label):
    lz, err, truth = map(np.asarray, (lz, err, truth))
    dev = lz - truth
    print(f"\n{label}: mean dev {dev.mean():+.4f}, std {dev.std(ddof=1):.4f}, mean err {err.mean():.4f}, "
          f"max |dev|/err {np.max(np.abs(dev) / err):.2f}")
    # each run within 3 of its own reported error (with 20 runs, allow one at 3.5)
    assert np.sum(np.abs(dev) > 3.0 * err) <= 1
    assert np.all(np.abs(dev) < 3.5 * err)
    # the 20-seed mean within 3 standard errors of the truth
    assert abs(dev.mean()) < 3.0 * dev.std(ddof=1) / np.sqrt(dev.size) + 1e-3


def test_gauss_d2_twenty_seeds_closed_form(gpu_lib):
    wls = [W.gauss_d2(seed=s) for s in range(20)]
    truth = box_gauss_logZ(wls[0].mu[0], wls[0].sigma, wls[0].a, wls[0].b)
    with native.Sampler(wls) as s:
        res = s.run()
    _check_seeds([r["logZ"] for r in res], [r["logZ_err"] for r in res], [truth] * 20, "gauss_d2")
    for r in res:
        # a null move needs a chain whose own point sits within FP32 rounding of
        # logL*; it may happen, but only at the rate of such near-ties
        assert r["status"] == 0 and r["nan_evals"] == 0
        assert r["nulls"] <= 1e-4 * r["iters"] * 250 * 10
        assert r["n_dead"] == r["iters"] * 250 + 500


def _golden_gmm():
    rows = [l.split() for l in open(golden_path("oracle_gmm_d32_logz.txt")) if not l.startswith("#")]
    return {int(r[0]): (float(r[1]), float(r[2])) for r in rows}


def test_gmm_d32_twenty_seeds_against_checker(gpu_lib):
    """20 seeds of the 32-d mixture against the FP64 checker's 20 runs of the
    same seeds (tests/golden/oracle_gmm_d32_logz.txt) and the closed form.
    Both sides overestimate the closed form by ~1.2 nat at p = 3d: the
    live-set whitening mixes slowly inside four modes ~70 sigma apart; the
    GPU must reproduce the checker, bias included."""
    gold = _golden_gmm()
    wls = [W.gmm_d32(seed=s) for s in range(20)]
    truth = np.array([box_gmm_logZ(w.mu, w.sigma, w.a, w.b) for w in wls])
    with native.Sampler(wls) as s:
        res = s.run()
    lz = np.array([r["logZ"] for r in res]); err = np.array([r["logZ_err"] for r in res])
    lo = np.array([gold[i][0] for i in range(20)]); eo = np.array([gold[i][1] for i in range(20)])
    diff = lz - lo
    print(f"\ngmm_d32: gpu mean dev from closed form {np.mean(lz - truth):+.4f}, checker {np.mean(lo - truth):+.4f}; "
          f"paired gpu-checker mean {diff.mean():+.4f} sd {diff.std(ddof=1):.4f}, max |d|/err {np.max(np.abs(diff) / err):.2f}")
    # The reported error (volume trajectories, App. D.2) under-covers this
    # workload's run-to-run scatter: the checker's own 20 runs scatter about
    # the closed form by kappa ~ 1.24 times their mean reported error (finite
    # HRSS chains leave successive dead points correlated).  Each GPU run
    # within 3 kappa combined errors of the checker's run of the same seed
    # (the two decorrelate after their first near-tie), one of 20 allowed up
    # to 4 kappa.
    kappa = (lo - truth).std(ddof=1) / eo.mean()
    band = kappa * np.sqrt(err**2 + eo**2)
    print(f"kappa {kappa:.3f}; max |d| / (kappa combined err) {np.max(np.abs(diff) / band):.2f}")
    assert np.sum(np.abs(diff) > 3.0 * band) <= 1
    assert np.all(np.abs(diff) < 4.0 * band)
    # 20-seed means agree within three standard errors of the paired difference
    assert abs(diff.mean()) < 3.0 * diff.std(ddof=1) / np.sqrt(20) + 1e-3
    # same mean bias relative to the closed form on both sides
    assert abs(np.mean(lz - truth) - np.mean(lo - truth)) < 3.0 * diff.std(ddof=1) / np.sqrt(20) + 1e-3
    ev = np.array([r["evals"] for r in res], float)
    steps = np.array([r["iters"] * 500 * 96 for r in res], float)
    print(f"evals per HRSS step {np.mean(ev / steps):.2f}, iterations {np.mean([r['iters'] for r in res]):.1f}")


def _traj_se(dd, w, gi, n_traj=16):
    """Dispersion of the Fisher-identity estimate sum_i w_i g_i over simulated
    volume trajectories (App. D.2: trapezoid dX from the checker's
    trajectories of the run's own live counts)."""
    ll = dd["logL"].astype(np.float64)
    per = []
    for t in range(n_traj):
        lx = O.volume_trajectory(dd["nlive"], t, w.seed, w.run_id)
        X = np.concatenate([[1.0], np.exp(lx), [0.0]])
        dX = 0.5 * (X[:-2] - X[2:])
        lw = ll + np.log(np.maximum(dX, 1e-300))
        wt = np.exp(lw - special.logsumexp(lw))
        per.append(np.sum(wt * gi))
    return float(np.std(per, ddof=1))


def test_batch64_closed_form(gpu_lib):
    """The 64 runs of the batched workload against their closed-form evidences
    and closed-form d lnZ/dsigma (Fisher identity on the device).  The
    gradient's error bar: the volume-trajectory dispersion of each run (App.
    D.2), scaled by one factor kappa calibrated on independent repeats (the
    same 64 problems under three more seeds): the trajectories model the
    volume noise, while successive dead points of a finite HRSS chain stay
    correlated, so the true run-to-run scatter is somewhat larger."""
    base = W.batch64(seed=0)
    reps = [w.with_(seed=100 + q) for q in range(3) for w in base]
    wls = base + reps
    nb = len(base)
    with native.Sampler(wls) as s:
        res = s.run()
        grads = np.array([s.posterior(native.GRAD_LIK_SIGMA, r)[0] for r in range(len(wls))])
        ses = []
        for r, w in enumerate(base):
            dd = s.dead(r)
            q = np.sum((dd["x"].astype(np.float64) - np.float32(w.mu[0][0])) ** 2, axis=1)
            ses.append(_traj_se(dd, w, q / w.sigma ** 3 - w.d / w.sigma))
    ses = np.array(ses)
    # closed form: lnZ(sigma) = sum_i ln[Phi((b - mu)/sigma) - Phi((a - mu)/sigma)]
    h = 1e-6
    tg = np.array([(box_gauss_logZ(w.mu[0], w.sigma + h, w.a, w.b) - box_gauss_logZ(w.mu[0], w.sigma - h, w.a, w.b))
                   / (2 * h) for w in base])
    g4 = grads.reshape(4, nb)                      # [seed][problem]
    s_emp2 = g4.var(axis=0, ddof=1)                # run-to-run scatter, 3 dof per problem
    kappa = float(np.sqrt(np.mean(s_emp2 / ses ** 2)))
    zg = (g4[0] - tg) / (kappa * ses)
    zm = (g4.mean(axis=0) - tg) / (kappa * ses / 2.0)
    print(f"\nbatch64 d lnZ/dsigma: kappa {kappa:.3f}; seed 0: max |dev|/se {np.max(np.abs(zg)):.2f}, "
          f"beyond 3 se {int(np.sum(np.abs(zg) > 3))}, mean {np.mean(zg):+.3f}; "
          f"4-seed means: max |dev|/se {np.max(np.abs(zm)):.2f}, mean {np.mean(zm):+.3f}")
    # the trajectories carry most of the scatter
    assert 0.7 < kappa < 2.0
    assert np.sum(np.abs(zg) > 3.0) <= 3
    assert np.all(np.abs(zg) < 5.0)
    assert abs(np.mean(zg)) < 3.0 / np.sqrt(nb) + 0.2
    assert np.sum(np.abs(zm) > 3.0) <= 3
    assert np.all(np.abs(zm) < 5.0)
    truth = np.array([box_gauss_logZ(w.mu[0], w.sigma, w.a, w.b) for w in base])
    lz = np.array([r["logZ"] for r in res[:nb]]); err = np.array([r["logZ_err"] for r in res[:nb]])
    dev = lz - truth
    print(f"batch64: max |dev|/err {np.max(np.abs(dev) / err):.2f}, mean dev/err {np.mean(dev / err):+.3f}, "
          f"mean dev {dev.mean():+.4f} nat")
    assert np.sum(np.abs(dev) > 3.0 * err) <= 2
    assert np.all(np.abs(dev) < 4.0 * err)
    assert abs(np.mean(dev / err)) < 3.0 / np.sqrt(nb) + 0.1


def test_volume_simulation_matches_checker_on_gpu_dead_list(gpu_lib):
    wl = W.gauss_d2(seed=5)
    with native.Sampler(wl) as s:
        res = s.run()[0]
        d = s.dead(0)
    lz, err, lw, lzr = O.finalise(d["logL"].astype(np.float64), d["nlive"], 100, wl.seed, wl.run_id,
                                  want_r=True)
    print(f"\nvolsim: gpu {res['logZ']:.9f} +- {res['logZ_err']:.9f}  checker {lz:.9f} +- {err:.9f}; "
          f"max |dlog_w| {np.max(np.abs(d['log_w'] - lw)):.2e}")
    assert abs(res["logZ"] - lz) < 2e-6
    assert abs(res["logZ_err"] - err) < 2e-6
    assert np.max(np.abs(d["log_w"] - lw)) < 2e-5
    # weights normalised to FP32-exponential accuracy (terms e^(lw - max) in FP32, sum in FP64)
    assert abs(special.logsumexp(d["log_w"])) < 1e-7
    # deterministic Delta-X evidence over the same dead list, in death order
    z, x = -np.inf, 0.0
    for l, n in zip(d["logL"].astype(np.float64), d["nlive"]):
        z, x = O.evidence_death(l, int(n), z, x)
    assert abs(res["logZ_det"] - z) < 1e-6


def test_run_invariants_and_posterior_moments(gpu_lib):
    wl = W.gauss_d2(seed=9)
    with native.Sampler(wl) as s:
        res = s.run()[0]
        d = s.dead(0)
    m, k = wl.n_live, wl.k
    assert np.all(np.diff(d["logL"]) >= 0)
    born = d["birth"] > -np.inf
    assert np.all(d["logL"][born] > d["birth"][born])
    want = np.concatenate([np.arange(m, m - k, -1)] * res["iters"] + [np.arange(m, 0, -1)])
    assert np.array_equal(d["nlive"], want)
    w = np.exp(d["log_w"])
    tn = stats.truncnorm(-5, 5, loc=0.5, scale=0.1)
    ess = 1 / np.sum(w**2)
    for i in range(2):
        mean = np.sum(w * d["x"][:, i])
        var = np.sum(w * (d["x"][:, i] - mean) ** 2)
        assert abs(mean - tn.mean()) < 5 * tn.std() / np.sqrt(ess)
        assert abs(var / tn.var() - 1) < 5 * np.sqrt(2 / ess)


def test_step_by_step_equals_run(gpu_lib):
    wl = W.gauss_d2(seed=21)
    with native.Sampler(wl) as a:
        ra = a.run()[0]
        da = a.dead(0)
    with native.Sampler(wl) as b:
        done = False
        while not done:
            done, info = b.step()
        rb = b.finalise()[0]
        db = b.dead(0)
    assert ra["iters"] == rb["iters"] and ra["logZ"] == rb["logZ"]
    assert np.array_equal(da["x"], db["x"]) and np.array_equal(da["log_w"], db["log_w"])


def test_export_import_resume_is_bit_identical(gpu_lib):
    wl = W.gmm_d32(seed=3, n_live=200, k=100).with_(p=10)
    with native.Sampler(wl) as a:
        for _ in range(4):
            a.step()
        st = a.export_state()
        a.step(); a.step()
        ref = a.export_state()
    with native.Sampler(wl) as b:
        b.import_state(0, st["x"], st["logL"], st["birth"], iter=st["iter"], logZ=st["logZ"],
                       logX=st["logX"], n_dead=0)
        b.step(); b.step()
        got = b.export_state()
    assert np.array_equal(ref["x"], got["x"]) and np.array_equal(ref["logL"], got["logL"])
    assert ref["logZ"] == got["logZ"] and ref["logX"] == got["logX"]


def test_random_walk_runs_against_closed_form(gpu_lib):
    """The constrained random-walk kernel (kernel = 1) on gauss_d2 with p = 40:
    evidence within its error of the closed form over 8 seeds; every step
    costs exactly one evaluation."""
    wls = [W.gauss_d2(seed=s).with_(run_id=s, p=40, extra={"options": {"kernel": 1}}) for s in range(8)]
    truth = box_gauss_logZ(wls[0].mu[0], wls[0].sigma, wls[0].a, wls[0].b)
    with native.Sampler(wls) as smp:
        res = smp.run()
    dev = np.array([(r["logZ"] - truth) / r["logZ_err"] for r in res])
    print(f"\nrandom walk gauss_d2: dev/err {np.round(dev, 2)}, evals per dead point "
          f"{np.mean([r['evals'] / r['n_dead'] for r in res]):.1f}")
    assert np.all(np.abs(dev) < 4.0)
    assert abs(dev.mean()) < 3.0 / np.sqrt(len(wls)) + 0.3
    for r in res:
        assert r["spec_evals"] == 0


# (d, alpha, steps per chain in units of d).  The paper's comparison runs
# d in {2, 4, 10, 30, 100, 300} over alpha in [0, 1] with 1000 live points
# (App. F.3).  With p = 3d the d = 100 runs overestimate log Z by ~0.75 nat
# and the d = 30, alpha = 0 runs underestimate it by ~0.3 nat; both vanish
# by p = 10d (inner-kernel mixing, not bookkeeping), so those cases run
# there.  The pure Rastrigin lattice at d = 100 (alpha = 0) does not mix at
# p = 10d and is left out.
RASTRIGIN_CASES = [(2, 0.0, 3), (2, 0.5, 3), (2, 1.0, 3), (4, 0.0, 3), (4, 0.5, 3), (4, 1.0, 3),
                   (10, 0.0, 3), (10, 0.1, 3), (10, 0.5, 3), (10, 1.0, 3), (30, 0.0, 10), (30, 0.5, 3),
                   (30, 0.9, 3), (100, 0.1, 10), (100, 0.5, 10), (100, 1.0, 10)]


@pytest.mark.parametrize("d,alpha,pd", RASTRIGIN_CASES)
def test_rastrigin_mixture_against_quadrature(gpu_lib, d, alpha, pd):
    """App. F.3 test likelihood (alpha f + (1 - alpha) g, f Gaussian, g
    Rastrigin with A = 10, uniform prior on [-5.14, 5.14]^d, 1000 live
    points): evidence against the semi-analytic value (one-dimensional
    quadratures raised to the power d)."""
    n = 8 if d >= 30 else 4
    wls = [W.rastrigin_mix(d, alpha=alpha, seed=s, run_id=s, n_live=1000, k=500).with_(p=pd * d)
           for s in range(n)]
    truth = rastrigin_logZ(alpha, d)
    with native.Sampler(wls) as smp:
        res = smp.run()
    dev = np.array([(r["logZ"] - truth) / r["logZ_err"] for r in res])
    print(f"\nrastrigin d={d} alpha={alpha} p={pd * d}: truth {truth:.4f}, "
          f"logZ {np.mean([r['logZ'] for r in res]):.4f}, dev/err {np.round(dev, 2)}")
    assert np.all(np.abs(dev) < 4.0)
    assert abs(dev.mean()) < 3.0 / np.sqrt(len(wls)) + 0.4
