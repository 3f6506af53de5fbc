"""The plain single-run FP32 GPU path (one kernel per phase, one thread per
chain in lockstep evaluation rounds, every candidate's likelihood from
scratch, a host loop per iteration) against the batched sweep: in the same
sweep configuration both take the same decisions, so every dead point
matches bit for bit and the evidence is identical."""
import numpy as np
import pytest

from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _runs(wls, path, cfg):
    out = []
    opts = lambda: {"sweep_cfg": cfg, "path": path}
    wls = [w.with_(extra={**w.extra, "options": opts()}) for w in wls]
    if path == native.PATH_PLAIN:
        for w in wls:
            with native.Sampler(w) as s:
                r = s.run()[0]
                out.append((r, s.dead(0)))
    else:
        with native.Sampler(wls) as s:
            res = s.run()
            out = [(res[i], s.dead(i)) for i in range(len(wls))]
    return out


def _same(a, b):
    ra, da = a
    rb, db = b
    assert ra["n_dead"] == rb["n_dead"] and ra["iters"] == rb["iters"]
    for key in ("x", "logL", "birth", "nlive", "log_w"):
        assert np.array_equal(da[key], db[key]), key
    for key in ("logZ", "logZ_err", "logZ_det", "evals", "nulls", "cap_out"):
        assert ra[key] == rb[key], key
    assert rb["spec_evals"] == 0  # the plain path tests one candidate at a time


@pytest.mark.parametrize("cfg", [3, 9, 16])
def test_plain_path_bit_identical_to_batched_gmm(gpu_lib, cfg):
    """4 seeds of the 32-d four-component mixture (500 live points, k = 250,
    p = 3d) in sweep configurations 8x4, 16x2 and 4x8."""
    wls = [W.gmm_d32(seed=s, n_live=500, k=250) for s in range(4)]
    bat = _runs(wls, native.PATH_BATCHED, cfg)
    pl = _runs(wls, native.PATH_PLAIN, cfg)
    for a, b in zip(bat, pl):
        _same(a, b)


def test_plain_path_bit_identical_to_batched_gaussians(gpu_lib):
    """Gaussian runs of the batched-serving workload of several dimensions
    (ragged d: a lane's slice partly or wholly past d), each in its default
    grouped configuration."""
    b64 = W.batch64(seed=0)
    pick = [w for w in b64 if w.d in {w.d for w in b64[:12]}][:4]
    for w in pick:
        cfg = [q for q in range(22) if native.lib().nss_cfg_lanes(q) * native.lib().nss_cfg_dims(q)
               == max(4, 1 << (w.d - 1).bit_length())][0]
        _same(_runs([w], native.PATH_BATCHED, cfg)[0], _runs([w], native.PATH_PLAIN, cfg)[0])


def test_plain_path_gaussian_prior_and_step_trace(gpu_lib):
    """The 20-d Gaussian of the overhead study (Gaussian prior: the slice
    height enters every test): bit-identical to the batched sweep, and the
    per-chain record of an iteration matches too."""
    w = W.gauss20_paper(seed=2)
    cfg = 3  # 8 lanes x 4 dims
    _same(_runs([w], native.PATH_BATCHED, cfg)[0], _runs([w], native.PATH_PLAIN, cfg)[0])
    traces = []
    for path in (native.PATH_BATCHED, native.PATH_PLAIN):
        with native.Sampler(w.with_(extra={"options": {"sweep_cfg": cfg, "path": path}})) as s:
            for _ in range(3):
                s.step()
            traces.append(s.trace(0))
    for key, val in traces[0].items():
        assert np.array_equal(np.asarray(val), np.asarray(traces[1][key])), key


def _small_logreg(seed):
    return W.logreg_d100(seed=seed, n_rows=1000, d=10, n_live=200, k=100).with_(name="logreg_small")


def test_plain_logistic_one_step_parity(gpu_lib):
    """The plain path's logistic step (lockstep evaluation rounds, each slice
    test's logits recomputed from the candidate point by one tensor-core GEMM
    over all chains) against the FP64 checker on the same state and counters."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from parity import MAX_MISMATCH_FRACTION, MAX_TIE_FRACTION, compare_step, near_tie_mask
    wl = _small_logreg(5)
    wl = wl.with_(extra={**wl.extra, "options": {"path": native.PATH_PLAIN}})
    rep = compare_step(wl, 3)
    g, t = rep["gpu"], rep["orc"]
    assert np.array_equal(g["dead_idx"], t["dead_idx"]) and np.array_equal(g["parent"], t["parent"])
    tie = near_tie_mask(rep, "logreg_small")
    same = np.ones(wl.k, bool)
    for c in ("evals", "accepts", "nulls", "expansions", "shrinks", "cap_out"):
        same &= g[c] == t[c]
    xerr = np.abs(g["new_x"][same] - t["new_x"][same]).max()
    print(f"\nplain logistic step: ties {tie.mean():.3f} mismatch {np.mean(~same):.3f} x err {xerr:.2e}")
    assert np.all(same | tie)
    assert tie.mean() <= MAX_TIE_FRACTION and np.mean(~same) <= MAX_MISMATCH_FRACTION
    assert xerr <= 1e-5 * max(1.0, np.abs(t["new_x"][same]).max())


def test_plain_logistic_run_against_batched(gpu_lib):
    """Whole runs of the small logistic problem on both paths: the same
    method, so the evidences agree within the runs' combined errors (the two
    form the logits differently -- from the candidate point, or line-affine --
    and part ways after their first near-tie)."""
    seeds = range(4)
    lz_b, lz_p = [], []
    with native.Sampler([_small_logreg(s) for s in seeds]) as s:
        res_b = s.run()
    for sd in seeds:
        w = _small_logreg(sd)
        w = w.with_(extra={**w.extra, "options": {"path": native.PATH_PLAIN}})
        with native.Sampler(w) as s:
            res_p = s.run()[0]
        assert res_p["status"] == 0 and res_p["spec_evals"] == 0
        lz_p.append((res_p["logZ"], res_p["logZ_err"]))
    for (zp, ep), rb in zip(lz_p, res_b):
        d = zp - rb["logZ"]
        print(f"plain {zp:.3f} +- {ep:.3f}, batched {rb['logZ']:.3f} +- {rb['logZ_err']:.3f}")
        assert abs(d) < 3.0 * 1.25 * np.hypot(ep, rb["logZ_err"])
