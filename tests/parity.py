"""Helpers that drive the CUDA path and the CPU checker on the same seeded
state and compare them.  Used by the GPU parity tests and the smoke check."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

# Per-workload near-tie thresholds (nats, prior log-density, box units): a
# chain whose checker comparisons came within these margins may take the
# other branch in FP32, so its counts are compared only for validity.  Each is
# a few times the FP32 error budget of one comparison: ~4 ulp of the largest
# term of logL plus |grad logL| times the position error (<= 1e-6 of the box):
#   gauss_d2 (logL ~ 3, |grad| ~ 10):        ~3e-6 + 2e-6  -> 2e-5
#   gmm_d32 (logL ~ 90, |grad| ~ 300):       ~3e-5 + 2e-4  -> 1e-3
#   gauss20 (logL ~ 30, |grad| ~ 100):       ~1e-5 + 1e-4  -> 5e-4
#   batch64 (logL ~ 200, sigma >= 0.01):     ~1e-4 + 1e-3  -> 5e-3
#   logreg (N rows, |z| ~ 3..10): FP32 logits 1e-6 |z| per row, FP32 sums of
#   N terms of ~1 nat, fast exp/log in softplus: ~sqrt(N) 1e-5 -> 2e-3 (N=1e3), 1e-2 (N=1e4)
TIES = {"gauss_d2": (2e-5, 2e-5, 2e-6), "gmm_d32": (1e-3, 1e-3, 2e-6), "batch64": (5e-3, 5e-3, 2e-6),
        "gauss20": (5e-4, 5e-4, 2e-6), "logreg_small": (2e-3, 1e-4, 0.0), "logreg_d100": (1e-2, 1e-4, 0.0),
        "gp_d3": (2e-3, 0.0, 2e-6)}
#   gp_d3 (FP32 Cholesky of K, n <= 256, logL ~ 1e1..1e2): ~1e-4 |logL| -> 2e-3 (well-conditioned K)


# Measured over every one-step parity case: at most 5.2% of chains had a
# comparison inside these margins (the 32-d mixture, ~540 slice tests per
# chain) and at most 0.2% of chains took another branch than the checker.
# A chain whose counters match is compared in full (positions and logL) even
# if it had a near-tie; only chains whose counters differ are excluded, and
# each of those must have had a near-tie.
MAX_TIE_FRACTION = 0.06
MAX_MISMATCH_FRACTION = 0.01


def oracle_problem(wl):
    return O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())


def oracle_opts(wl, **kw):
    o = (wl.extra or {}).get("options", {})
    for key in ("kernel", "rw_scale", "dir_norm"):
        if key in o and key not in kw:
            kw[key] = o[key]
    return O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed, run_id=wl.run_id, w=wl.w, tol=wl.tol, **kw)


def fp32_state(wl, warm_iters):
    """A live set reached by the checker after `warm_iters` iterations, rounded
    to FP32 (positions and logL), together with its FP64 scalars."""
    pb, op = oracle_problem(wl), oracle_opts(wl)
    x, logL, birth = O.init_live(pb, op)
    st = (x, logL, birth, -np.inf, 0.0)
    for it in range(warm_iters):
        st, _ = O.step(pb, op, it, *st)
    x, logL, birth, logZ, logX = st
    return (x.astype(np.float32), logL.astype(np.float32), birth.astype(np.float32), logZ, logX)


def compare_step(wl, warm_iters=2, sampler=None, run=0):
    """Feed one FP32 state to both sides, take one iteration, return a report."""
    x32, l32, b32, logZ, logX = fp32_state(wl, warm_iters)
    own = sampler is None
    s = sampler if sampler is not None else native.Sampler(wl)
    try:
        s.import_state(run, x32, l32, b32, iter=warm_iters, logZ=logZ, logX=logX, n_dead=0)
        done, info = s.step()
        g = s.trace(run)
        gstate = s.export_state(run)
    finally:
        if own:
            s.close()
    pb, op = oracle_problem(wl), oracle_opts(wl)
    (ox, ol, ob, oz, oxx), t = O.step(pb, op, warm_iters, x32.astype(np.float64), l32.astype(np.float64),
                                       b32.astype(np.float64), logZ, logX)
    return {"gpu": g, "orc": t, "info": info[run], "gstate": gstate, "orc_logZ": oz, "orc_logX": oxx,
            "x32": x32, "l32": l32}


def near_tie_mask(rep, name):
    tl, tp, tb = TIES.get(name, (1e-3, 1e-3, 2e-6))
    t = rep["orc"]
    return (t["margin"] <= tl) | (t["pmargin"] <= tp) | (t["bmargin"] <= tb)
