"""GP hyperparameter likelihood on the GPU (RBF + white kernel): the sweep's
tensor-core factorisation (kernel matrix in tensor memory, 3xTF32 trailing
updates, FP64 log-determinant) and the SIMT initial likelihoods against the
FP64 checker, one-step parity at n = 64 and at the full n = 256, and
evidences against brute-force 3-D quadrature."""
import numpy as np
import pytest

import oracle as O
from conftest import golden_path
from closed_forms import gp_quadrature_logZ
from parity import (MAX_MISMATCH_FRACTION, MAX_TIE_FRACTION, compare_step, near_tie_mask, oracle_opts,
                    oracle_problem)
from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

COUNTERS = ("evals", "accepts", "nulls", "expansions", "shrinks", "cap_out")

# Error of the factorised logL relative to max(1, |logL|).  The trailing
# updates run in 3xTF32 (hi hi + hi lo + lo hi of two TF32 parts), a unit
# roundoff near 2^-21 rather than FP32's 2^-24, and a Cholesky solve's forward
# error on y^T K^-1 y and ln det K grows as cond(K) times the unit roundoff
# (normwise perturbation bound of the factorisation).  Twice 2^-21 per unit of
# cond(K), plus FP32 rounding of the O(n) terms of the sum.
U_EFF = 2.0 ** -21


def gp_tol(cond):
    return 1e-4 + 2.0 * U_EFF * cond


def kernel_cond(wl, th):
    ell, amp, sn = np.exp(th)
    K = amp**2 * np.exp(-np.subtract.outer(wl.t, wl.t) ** 2 / (2 * ell**2)) + sn**2 * np.eye(wl.t.size)
    return np.linalg.cond(K)


def test_initial_logL_matches_checker_full_size(gpu_lib):
    """FP32 Cholesky: the logL error grows with cond(K) (about eps32 * cond);
    below cond 1e5 it stays under 1e-3 relative."""
    wl = W.gp_d3(seed=1)  # n = 256
    with native.Sampler(wl) as s:
        st = s.export_state()
    pb = oracle_problem(wl)
    ref = pb.loglik(st["x"].astype(np.float64))
    cond = np.array([kernel_cond(wl, th.astype(np.float64)) for th in st["x"]])
    good = cond < 1e5
    err = np.abs(st["logL"] - ref) / np.maximum(1.0, np.abs(ref))
    fin = np.isfinite(st["logL"])
    print(f"\nGP initial logL: {good.sum()} points with cond(K) < 1e5, max rel err {err[good].max():.2e}; "
          f"all finite points max rel err {err[fin].max():.2e}; FP32 breakdowns {np.sum(~fin)} of {wl.n_live} "
          f"(min cond among them {cond[~fin].min() if (~fin).any() else 0:.1e})")
    assert err[good].max() < 1e-3
    # FP32 breakdowns only for badly conditioned kernels
    bad = ~fin
    assert (not bad.any()) or cond[bad].min() > 1e6


@pytest.mark.parametrize("n", [24, 100, 256])
def test_tensor_core_loglik_matches_checker(gpu_lib, n):
    """The sweep's tensor-core factorisation against the FP64 checker over
    the prior box (n = 24 and 100 pad to 32 and 128 rows with an identity
    block): the error of the 3xTF32 factorisation grows with cond(K); an
    FP32 breakdown (logL = -inf) only for badly conditioned kernels."""
    wl = W.gp_d3(seed=3, n=n)
    rng = np.random.default_rng(n)
    th = rng.uniform(wl.a, wl.b, size=(400, 3))
    # and a cloud around the data's own scale (l ~ 1, a ~ 1, s ~ 0.1)
    th = np.vstack([th, np.log([1.0, 1.0, 0.1]) + 0.3 * rng.standard_normal((200, 3))])
    got = native.gp_loglik(wl.t, wl.y, th).astype(np.float64)
    pb = oracle_problem(wl)
    # the kernel sees FP32 parameters and data
    th32 = th.astype(np.float32).astype(np.float64)
    ref = pb.loglik(th32)
    cond = np.array([kernel_cond(wl, x) for x in th32])
    fin = np.isfinite(got)
    rel = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    tol = gp_tol(cond)
    worst = np.max(rel[fin] / tol[fin])
    print(f"\nGP tensor-core logL n={n}: {fin.sum()} finite of {len(th)}, max rel err {rel[fin].max():.2e} "
          f"(cond < 1e4: {rel[fin & (cond < 1e4)].max():.2e}), worst err/tol {worst:.3f}, "
          f"breakdowns min cond {cond[~fin].min() if (~fin).any() else 0:.1e}")
    assert np.all(rel[fin] <= tol[fin])
    assert (fin | (cond > 1e6)).all()


def test_one_step_parity_gp_full_size(gpu_lib):
    """One iteration at the full n = 256 data set (m and k reduced so the
    FP64 checker finishes in seconds)."""
    wl = W.gp_d3(seed=4).with_(n_live=100, k=40)
    rep = compare_step(wl, 2)
    g, t = rep["gpu"], rep["orc"]
    assert np.array_equal(g["dead_idx"], t["dead_idx"])
    assert np.array_equal(g["parent"], t["parent"])
    tie = near_tie_mask(rep, "gp_d3")
    same = np.ones(wl.k, bool)
    for c in COUNTERS:
        same &= g[c] == t[c]
    ok = same
    cond = np.array([kernel_cond(wl, th.astype(np.float64)) for th in t["new_x"]])
    rel = np.abs(g["new_logL"] - t["new_logL"]) / np.maximum(1, np.abs(t["new_logL"]))
    xerr = np.abs(g["new_x"][ok] - t["new_x"][ok]).max()
    print(f"\nGP n=256 one step: ties {tie.mean():.3f} mismatch {np.mean(~same):.3f} x err {xerr:.2e} "
          f"logL rel err {rel[ok].max():.2e}")
    assert np.all(same | tie)
    assert tie.mean() <= MAX_TIE_FRACTION and np.mean(~same) <= MAX_MISMATCH_FRACTION
    assert xerr < 1e-4
    assert np.all(rel[ok] <= gp_tol(cond[ok]))


@pytest.mark.parametrize("seed,warm", [(1, 3), (2, 8)])
def test_one_step_parity_gp(gpu_lib, seed, warm):
    wl = W.gp_d3(seed=seed, n=64).with_(n_live=200, k=100)
    rep = compare_step(wl, warm)
    g, t = rep["gpu"], rep["orc"]
    assert np.array_equal(g["dead_idx"], t["dead_idx"])
    assert np.array_equal(g["parent"], t["parent"])
    tie = near_tie_mask(rep, "gp_d3")
    same = np.ones(wl.k, bool)
    for c in COUNTERS:
        same &= g[c] == t[c]
    ok = same
    xerr = np.abs(g["new_x"][ok] - t["new_x"][ok]).max()
    lerr = (np.abs(g["new_logL"][ok] - t["new_logL"][ok]) / np.maximum(1, np.abs(t["new_logL"][ok]))).max()
    print(f"\nGP seed={seed} warm={warm}: ties {tie.mean():.3f} mismatch {np.mean(~same):.3f} "
          f"x err {xerr:.2e} logL rel err {lerr:.2e}")
    assert np.all(same | tie)
    assert tie.mean() <= MAX_TIE_FRACTION and np.mean(~same) <= MAX_MISMATCH_FRACTION
    assert xerr < 1e-4
    # logL of well-conditioned end points within 1e-3; FP32 Cholesky limit otherwise
    cond = np.array([kernel_cond(wl, th.astype(np.float64)) for th in t["new_x"]])
    rel = np.abs(g["new_logL"] - t["new_logL"]) / np.maximum(1, np.abs(t["new_logL"]))
    assert np.all(rel[ok] <= gp_tol(cond[ok])), np.max(rel[ok] / gp_tol(cond[ok]))


def test_gp_evidence_matches_quadrature(gpu_lib):
    wl = W.gp_d3(seed=2, n=24).with_(n_live=200, k=100)
    pb = oracle_problem(wl)
    truth = gp_quadrature_logZ(pb.loglik, wl.a, wl.b, panels=10, order=6)
    wls = [wl.with_(seed=s) for s in range(8)]
    with native.Sampler(wls) as smp:
        res = smp.run()
    lz = np.array([r["logZ"] for r in res]); err = np.array([r["logZ_err"] for r in res])
    print(f"\nGP evidence: quadrature {truth:.4f}, gpu mean {lz.mean():.4f} (err {err.mean():.3f})")
    assert np.all(np.abs(lz - truth) < 3.5 * err + 0.02)
    assert abs(lz.mean() - truth) < 3 * lz.std(ddof=1) / np.sqrt(len(lz)) + 0.05


def test_gp_full_size_run_completes(gpu_lib):
    wl = W.gp_d3(seed=0)
    with native.Sampler(wl) as s:
        res = s.run()[0]
    print(f"\nGP full size (n=256, m=500, k=250, p=15): logZ {res['logZ']:.3f} +- {res['logZ_err']:.3f}, "
          f"{res['iters']} iterations, {res['evals']} evals, {res['nan_evals']} FP32 breakdowns")
    assert res["status"] == 0 and np.isfinite(res["logZ"])


def _golden_value(name, key):
    for line in open(golden_path(name)):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        if parts[0] == key:
            return float(parts[1])
    raise KeyError(key)


def test_gp_full_size_evidence_matches_quadrature(gpu_lib):
    """The full-size GP workload (n = 256 data of gp_d3 seed 0; m = 500,
    k = 250, p = 15) over 8 sampling seeds against brute-force quadrature of
    the checker's FP64 marginal likelihood (tests/golden/gp_d3_quadrature.txt:
    Gauss-Legendre in the posterior's principal axes, converged to 1e-4):
    every run within 3.5 of its own reported error, the mean within three
    standard errors of the seeds; and paired with the FP64 checker's runs of
    the same seeds (tests/golden/oracle_gp_d3_logz.txt): each pair within 3
    combined errors, the mean difference within 3 standard errors."""
    truth = _golden_value("gp_d3_quadrature.txt", "gp_d3_seed0_logZ")
    wl = W.gp_d3(seed=0)
    with native.Sampler([wl.with_(seed=s) for s in range(8)]) as smp:
        res = smp.run()
    lz = np.array([r["logZ"] for r in res])
    err = np.array([r["logZ_err"] for r in res])
    se = lz.std(ddof=1) / np.sqrt(len(lz))
    print(f"\nGP n=256 evidence: quadrature {truth:.4f}, gpu mean {lz.mean():.4f} +- {se:.4f} "
          f"(per-run err {err.mean():.3f}), worst |dlogZ|/err {np.max(np.abs(lz - truth) / err):.2f}")
    assert all(r["status"] == 0 for r in res)
    assert np.all(np.abs(lz - truth) < 3.5 * err + 0.02)
    assert abs(lz.mean() - truth) < 3 * se + 0.05
    ck = np.array([[float(x) for x in l.split()] for l in open(golden_path("oracle_gp_d3_logz.txt"))
                   if not l.startswith("#") and l.strip()])
    assert np.array_equal(ck[:, 0], np.arange(8))
    dz = lz - ck[:, 1]
    print(f"GPU - checker (paired seeds): {dz.mean():+.4f} +- {dz.std(ddof=1) / np.sqrt(8):.4f}")
    assert np.all(np.abs(dz) < 3 * np.hypot(err, ck[:, 2]))
    assert abs(dz.mean()) < 3 * dz.std(ddof=1) / np.sqrt(8)
