"""GPU <-> checker parity of one outer iteration fed the same FP32 state and
the same Philox counters: selection indices, threshold and parents
bit-exact; per-chain accept/eval counters bit-exact except near-ties;
positions and logL of the matching chains within 1e-5 relative; evidence
scalars within FP64 rounding of the FP32 terms."""
import numpy as np
import pytest

import oracle as O
from parity import (MAX_MISMATCH_FRACTION, MAX_TIE_FRACTION, compare_step, near_tie_mask, oracle_opts,
                    oracle_problem)
from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

COUNTERS = ("evals", "accepts", "nulls", "expansions", "shrinks", "cap_out")


def _wl(name, seed):
    if name == "gauss_d2":
        return W.gauss_d2(seed=seed)
    if name == "gmm_d32":
        return W.gmm_d32(seed=seed)
    if name == "gmm_d32_small":
        return W.gmm_d32(seed=seed, n_live=300, k=150).with_(p=12)
    if name == "gauss_d5_odd":
        d = 5
        return W.Workload("gauss_d5", d, "box", np.zeros(d), np.ones(d), "gauss", 64, 33, 7,
                          sigma=0.05, mu=np.full((1, d), 0.4), seed=seed)
    if name == "gauss20":
        return W.gauss20_paper(seed=seed, n_live=256, k=100).with_(p=10)
    if name == "rastrigin_d5":
        return W.rastrigin_mix(5, alpha=0.5, seed=seed, n_live=200, k=100).with_(p=15)
    if name.startswith("rw_"):
        base = _wl(name[3:], seed)
        opts = dict((base.extra or {}).get("options", {}), kernel=1)
        return base.with_(p=3 * base.p, extra=dict(base.extra or {}, options=opts))
    if name in ("gmm_d10_k3", "gmm_d20_k6"):
        d, K = (10, 3) if name == "gmm_d10_k3" else (20, 6)
        mu = np.random.default_rng(seed + 100).uniform(0.2, 0.8, size=(K, d))
        return W.Workload(name, d, "box", np.zeros(d), np.ones(d), "gmm", 300, 150, 2 * d,
                          sigma=0.05, mu=mu, seed=seed)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["gauss_d2", "gauss_d5_odd"])
def test_initial_live_set_matches_checker(gpu_lib, name):
    wl = _wl(name, 3)
    with native.Sampler(wl) as s:
        st = s.export_state()
    pb, op = oracle_problem(wl), oracle_opts(wl)
    ox, _, _ = O.init_live(pb, op)
    # uniform box [0,1]^d: x = u is exact in FP32 on both sides
    assert np.array_equal(st["x"], ox.astype(np.float32))
    ref = pb.loglik(st["x"].astype(np.float64))
    assert np.allclose(st["logL"], ref, rtol=1e-5, atol=1e-5)
    assert np.all(st["birth"] == -np.inf)


@pytest.mark.parametrize("name,seed,warm", [
    ("gauss_d2", 1, 1), ("gauss_d2", 2, 6), ("gauss_d5_odd", 4, 3), ("gmm_d32_small", 5, 4),
    ("gmm_d32", 0, 3), ("gmm_d32", 7, 25), ("gauss20", 2, 5), ("gmm_d10_k3", 3, 4), ("gmm_d20_k6", 6, 4),
    ("rw_gauss_d5_odd", 4, 3), ("rw_gmm_d32_small", 5, 4), ("rw_gauss20", 2, 5),
    ("rastrigin_d5", 3, 4), ("rw_rastrigin_d5", 3, 4)])
def test_one_step_parity(gpu_lib, name, seed, warm):
    wl = _wl(name, seed)
    rep = compare_step(wl, warm)
    g, t = rep["gpu"], rep["orc"]
    key = wl.name if wl.name in ("gauss_d2", "gmm_d32", "gauss20") else "gmm_d32"
    if name.startswith("rw_"):
        # a random-walk step is one proposal: no bracket, no shrinkage
        assert np.all(g["expansions"] == 0) and np.all(g["shrinks"] == 0)
        assert np.array_equal(g["evals"], np.full(wl.k, wl.p))
    # (i) selection and threshold: bit-exact
    assert np.array_equal(g["dead_idx"], t["dead_idx"])
    assert g["logLstar"] == np.float32(t["logLstar"])
    # (ii) parents: bit-exact
    assert np.array_equal(g["parent"], t["parent"])
    # metric factor
    scale = np.abs(t["L"]).max()
    lerr = np.abs(g["L"] - t["L"]).max() / scale
    # (iii) counters: exact for every chain that had no near-tie
    tie = near_tie_mask(rep, key)
    same = np.ones(wl.k, bool)
    for c in COUNTERS:
        same &= g[c] == t[c]
    ok = same
    xerr = np.abs(g["new_x"][ok] - t["new_x"][ok]).max() if ok.any() else 0.0
    # logL = (log peak density) - (quadratic term): FP32 rounding, and the
    # slope times the position differences, scale with the larger of the two
    # terms, bounded by the best live logL of the iteration
    top = float(np.max(rep["l32"][np.isfinite(rep["l32"])]))
    scale = np.maximum(max(1.0, abs(top)), np.abs(t["new_logL"][ok]))
    lrel = (np.abs(g["new_logL"][ok] - t["new_logL"][ok]) / scale).max()
    print(f"\n{name} seed={seed} warm={warm}: L rel err {lerr:.2e}, ties {tie.mean():.4f}, "
          f"mismatch {np.mean(~same):.4f}, x err {xerr:.2e}, logL rel err {lrel:.2e}, "
          f"logZ err {abs(rep['info']['logZ'] - rep['orc_logZ']):.2e}, "
          f"evals gpu {g['evals'].sum()} orc {t['evals'].sum()}")
    assert lerr < 2e-5
    assert np.all(same | tie), np.nonzero(~(same | tie))[0][:10]
    assert tie.mean() <= MAX_TIE_FRACTION
    assert np.mean(~same) <= MAX_MISMATCH_FRACTION
    width = np.max(wl.b - wl.a) if wl.prior == "box" else 1.0
    assert xerr <= 1e-5 * width
    assert lrel <= 1e-5
    # every chain (tied or not) ends strictly inside the constrained set
    moved = g["nulls"] < wl.p
    ll64 = oracle_problem(wl).loglik(g["new_x"][moved].astype(np.float64))
    assert np.all(ll64 > t["logLstar"] - 1e-4 * max(1.0, abs(t["logLstar"])))
    # evidence scalars
    assert abs(rep["info"]["logX"] - rep["orc_logX"]) < 1e-12
    assert abs(rep["info"]["logZ"] - rep["orc_logZ"]) < 1e-6 * max(1.0, abs(rep["orc_logZ"]))
    # the state left behind: dead slots hold the chain results, born at logL*
    gs = rep["gstate"]
    assert np.array_equal(gs["x"][g["dead_idx"]], g["new_x"])
    assert np.all(gs["birth"][g["dead_idx"]] == g["logLstar"])
    keep = np.setdiff1d(np.arange(wl.n_live), g["dead_idx"])
    assert np.array_equal(gs["x"][keep], rep["x32"][keep])


@pytest.mark.parametrize("name", ["gauss_d2", "gauss_d5_odd", "gauss20", "gmm_d32", "gmm_d20_k6", "rastrigin_d5"])
def test_one_step_parity_every_sweep_configuration(gpu_lib, name):
    """Every (lanes per chain, dims per lane) configuration that fits d gives
    the same selection and parents and counters matching the checker; d = 5
    and d = 20 leave the last lanes of a group a partial (or empty) slice."""
    wl = _wl(name, 31)
    key = name if name in ("gauss_d2", "gmm_d32", "gauss20") else "gmm_d32"
    with native.Sampler(wl) as s:
        cands = [q for q in range(25) if _fits(s, q, wl.d)]
    assert len(cands) >= 2
    for q in cands:
        with native.Sampler(wl) as s:
            s.set_cfg(0, q)
            rep = compare_step(wl, 3, sampler=s)
        g, t = rep["gpu"], rep["orc"]
        assert np.array_equal(g["dead_idx"], t["dead_idx"]) and np.array_equal(g["parent"], t["parent"])
        tie = near_tie_mask(rep, key)
        same = np.ones(wl.k, bool)
        for c in COUNTERS:
            same &= g[c] == t[c]
        print(f"\n{name} cfg {native.Sampler.cfg_info(q)}: mismatch {np.mean(~same):.4f} ties {tie.mean():.4f}")
        assert np.all(same | tie)
        assert tie.mean() <= MAX_TIE_FRACTION and np.mean(~same) <= MAX_MISMATCH_FRACTION
        ok = same
        assert np.abs(g["new_x"][ok] - t["new_x"][ok]).max() <= 1e-5
        # slots that were not replaced keep their positions bit for bit
        keep = np.setdiff1d(np.arange(wl.n_live), g["dead_idx"])
        assert np.array_equal(rep["gstate"]["x"][keep], rep["x32"][keep])


def _fits(s, q, d):
    info = native.Sampler.cfg_info(q)
    cap = 4
    while cap < d:
        cap *= 2
    return info["lanes_per_chain"] * info["dims_per_lane"] == cap


def test_autotune_keeps_runs_correct(gpu_lib):
    wls = [W.gauss_d2(seed=s) for s in range(4)] + [W.gmm_d32(seed=s, n_live=200, k=100).with_(p=12, run_id=9)
                                                    for s in range(2)]
    with native.Sampler(wls) as s:
        chosen = s.autotune(iters=2)
        res = s.run()
    print("\nautotune:", chosen)
    for r in res:
        assert r["status"] == 0 and r["n_dead"] > 0


def test_batched_runs_equal_single_runs(gpu_lib):
    wls = [W.gauss_d2(seed=11), W.gmm_d32(seed=12, n_live=200, k=100).with_(p=8, run_id=1),
           W.gauss_d2(seed=13).with_(run_id=2)]
    with native.Sampler(wls) as b:
        b.run()
        dead_b = [b.dead(r) for r in range(3)]
    for r, wl in enumerate(wls):
        with native.Sampler(wl) as s:
            res = s.run()
            d1 = s.dead(0)
        for key in ("x", "logL", "nlive", "birth", "log_w"):
            assert np.array_equal(d1[key], dead_b[r][key]), (r, key)


# tiny batches: a warp's last groups without a chain of their own (k not a
# multiple of the chains per warp, down to k = 1), d below one lane's float4
TINY = [(1, 8, 4, 3), (2, 8, 1, 2), (3, 9, 7, 4), (3, 40, 13, 3), (4, 16, 9, 5)]


@pytest.mark.parametrize("d,m,k,p", TINY)
def test_one_step_parity_tiny_batches(gpu_lib, d, m, k, p):
    """m, k, p and d at their small ends, in every configuration that fits:
    selection, parents and the logical counters as the checker, positions
    within 1e-5, and the slots not replaced untouched."""
    wl = W.Workload("tiny", d, "box", np.zeros(d), np.ones(d), "gauss", m, k, p, sigma=0.2,
                    mu=np.full((1, d), 0.45), seed=11 + d + k)
    with native.Sampler(wl) as s:
        cands = [q for q in range(25) if _fits(s, q, d)]
    assert cands
    for q in cands:
        with native.Sampler(wl) as s:
            s.set_cfg(0, q)
            rep = compare_step(wl, 1, sampler=s)
        g, t = rep["gpu"], rep["orc"]
        assert np.array_equal(g["dead_idx"], t["dead_idx"]) and np.array_equal(g["parent"], t["parent"])
        tie = near_tie_mask(rep, "gauss_d2")
        same = np.ones(k, bool)
        for c in COUNTERS:
            same &= g[c] == t[c]
        assert np.all(same | tie), (q, np.nonzero(~(same | tie))[0])
        ok = same
        if ok.any():
            assert np.abs(g["new_x"][ok] - t["new_x"][ok]).max() <= 1e-5
        gs = rep["gstate"]
        assert np.array_equal(gs["x"][g["dead_idx"]], g["new_x"])
        keep = np.setdiff1d(np.arange(m), g["dead_idx"])
        assert np.array_equal(gs["x"][keep], rep["x32"][keep])
        assert abs(rep["info"]["logZ"] - rep["orc_logZ"]) < 1e-6 * max(1.0, abs(rep["orc_logZ"]))


# the largest sizes the library accepts: d = 128 (directions and the factor
# through shared memory, 128-wide groups) and m = 4096 (the block sort through
# shared memory); a Gaussian prior at d = 64
LARGE = [("box", 128, 300, 150, 3), ("box", 2, 4096, 2048, 3), ("gauss", 64, 256, 128, 4)]


@pytest.mark.parametrize("prior,d,m,k,p", LARGE)
def test_one_step_parity_maximum_sizes(gpu_lib, prior, d, m, k, p):
    if prior == "box":
        a, b = np.zeros(d), np.ones(d)
        mu = np.full((1, d), 0.45)
        sigma = 0.25 if d > 2 else 0.1
    else:  # prior N(0, I); likelihood N(x; 0.5, 0.5^2 I)
        a, b = np.zeros(d), np.ones(d)
        mu = np.full((1, d), 0.5)
        sigma = 0.5
    wl = W.Workload("large", d, prior, a, b, "gauss", m, k, p, sigma=sigma, mu=mu, seed=5 + d)
    rep = compare_step(wl, 2)
    g, t = rep["gpu"], rep["orc"]
    assert np.array_equal(g["dead_idx"], t["dead_idx"]) and np.array_equal(g["parent"], t["parent"])
    assert g["logLstar"] == np.float32(t["logLstar"])
    lerr = np.abs(g["L"] - t["L"]).max() / np.abs(t["L"]).max()
    tie = near_tie_mask(rep, "gmm_d32")
    same = np.ones(k, bool)
    for c in COUNTERS:
        same &= g[c] == t[c]
    ok = same
    print(f"\nlarge {prior} d={d} m={m} k={k}: L rel err {lerr:.2e}, ties {tie.mean():.4f}, "
          f"mismatch {np.mean(~same):.4f}")
    assert lerr < 2e-5
    assert np.all(same | tie)
    assert tie.mean() <= MAX_TIE_FRACTION and np.mean(~same) <= MAX_MISMATCH_FRACTION
    assert np.abs(g["new_x"][ok] - t["new_x"][ok]).max() <= 1e-5 * (1.0 if prior == "box" else 10.0)
    keep = np.setdiff1d(np.arange(m), g["dead_idx"])
    assert np.array_equal(rep["gstate"]["x"][keep], rep["x32"][keep])
    assert abs(rep["info"]["logZ"] - rep["orc_logZ"]) < 1e-6 * max(1.0, abs(rep["orc_logZ"]))


# the step directions' whitening L z on the tensor cores (16 < d <= 64, the
# default) and on the FP32 CUDA cores (dir_fp32 = 1): d = 17 and 48 leave the
# factor's padded rows and columns zero, d = 64 fills two K-chunks; both
# direction normalisations
@pytest.mark.parametrize("d,dir_norm", [(17, 0), (48, 0), (64, 0), (48, 1)])
@pytest.mark.parametrize("fp32", [0, 1])
def test_one_step_parity_direction_whitening(gpu_lib, d, dir_norm, fp32):
    wl = W.Workload(f"gauss_d{d}", d, "box", np.zeros(d), np.ones(d), "gauss", 300, 150, d,
                    sigma=0.08, mu=np.full((1, d), 0.45), seed=5 + d,
                    extra={"options": {"dir_fp32": fp32, "dir_norm": dir_norm}})
    rep = compare_step(wl, 3)
    g, t = rep["gpu"], rep["orc"]
    assert np.array_equal(g["dead_idx"], t["dead_idx"]) and np.array_equal(g["parent"], t["parent"])
    tie = near_tie_mask(rep, "gauss20")
    same = np.ones(wl.k, bool)
    for c in COUNTERS:
        same &= g[c] == t[c]
    xerr = np.abs(g["new_x"][same] - t["new_x"][same]).max()
    print(f"\ndirections d={d} norm={dir_norm} fp32={fp32}: ties {tie.mean():.4f} mismatch {np.mean(~same):.4f} "
          f"x err {xerr:.2e}")
    assert np.all(same | tie)
    assert tie.mean() <= MAX_TIE_FRACTION and np.mean(~same) <= MAX_MISMATCH_FRACTION
    assert xerr <= 1e-5
