"""Writes logreg_d100_is.txt: the evidence of the full-size logistic-regression
workload (logreg_d100 seed 0 data: d = 100, N = 10000 bf16-exact rows, N(0, I)
prior; the Sec. 4.2 shape) by importance sampling, independent of the nested
sampler:

    Z = E_q[ L(w) pi(w) / q(w) ],   q = multivariate t (nu degrees of freedom)
    centred on the posterior mode with scale matrix H^-1 (H the Hessian of the
    negative log posterior there, found by Newton's method),

with the weights' log L + log pi evaluated by the checker (oracle/, FP64; the
mode and Hessian only shape the proposal and use numpy's restatement of the
same log posterior).  With 10^4 rows the posterior is close to Gaussian, so
the weights are well behaved; the estimate is repeated for two proposals (nu = 8 and 30, the scale
inflated by 1.1 and 1.0) and its standard error (delta method over the
weights) and effective sample size are written beside it.

    python tests/golden/make_logreg_is.py
"""
import os
import sys
from multiprocessing import get_context

import numpy as np
from scipy import special

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def log_post_many(X, y, W):
    """log L(w) + log N(w; 0, I) for the columns of W (d x s), FP64."""
    Z = X @ W                                          # N x s logits
    ll = (y[:, None] * Z - np.logaddexp(0.0, Z)).sum(axis=0)
    d = W.shape[0]
    return ll - 0.5 * (W * W).sum(axis=0) - 0.5 * d * np.log(2.0 * np.pi)


_PB = None


def _checker_log_post(W):
    """log L(w) + log pi(w) for the columns of W, by the checker."""
    global _PB
    if _PB is None:
        import oracle as O
        from paper_2601_23252_gb300 import workloads as Wk
        wl = Wk.logreg_d100(seed=0)
        _PB = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    return np.array([_PB.loglik(W[:, i]) + _PB.log_prior(W[:, i]) for i in range(W.shape[1])])


def mode_and_hessian(X, y):
    d = X.shape[1]
    w = np.zeros(d)
    for _ in range(100):
        z = X @ w
        p = special.expit(z)
        g = X.T @ (y - p) - w
        H = (X * (p * (1.0 - p))[:, None]).T @ X + np.eye(d)
        step = np.linalg.solve(H, g)
        w = w + step
        if np.max(np.abs(step)) < 1e-12:
            break
    z = X @ w
    p = special.expit(z)
    H = (X * (p * (1.0 - p))[:, None]).T @ X + np.eye(d)
    return w, H


def importance(pool, w0, H, nu, infl, n, seed, chunk=2000):
    d = len(w0)
    cov = infl * np.linalg.inv(H)
    L = np.linalg.cholesky(cov)
    logdet = 2.0 * np.sum(np.log(np.diag(L)))
    g = np.random.default_rng(seed)
    blocks, logqs = [], []
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        u = g.standard_normal((d, m))
        c = g.chisquare(nu, size=m)
        dev = (L @ u) * np.sqrt(nu / c)
        W = w0[:, None] + dev
        # multivariate t log density at W
        q2 = np.sum(np.linalg.solve(L, dev) ** 2, axis=0)
        logq = (special.gammaln((nu + d) / 2) - special.gammaln(nu / 2) - 0.5 * d * np.log(nu * np.pi)
                - 0.5 * logdet - 0.5 * (nu + d) * np.log1p(q2 / nu))
        blocks.append(W)
        logqs.append(logq)
    lp = pool.map(_checker_log_post, blocks)
    lw = np.concatenate([a - b for a, b in zip(lp, logqs)])
    mx = lw.max()
    wt = np.exp(lw - mx)
    mean = wt.mean()
    logZ = float(mx + np.log(mean))
    se = float(np.sqrt(wt.var(ddof=1) / n) / mean)
    ess = float(wt.sum() ** 2 / np.sum(wt * wt))
    return logZ, se, ess


def main():
    from paper_2601_23252_gb300 import workloads as W
    wl = W.logreg_d100(seed=0)
    X = wl.X.astype(np.float64)
    y = wl.y.astype(np.float64)
    w0, H = mode_and_hessian(X, y)
    lp0 = float(log_post_many(X, y, w0[:, None])[0])
    d = X.shape[1]
    laplace = lp0 + 0.5 * d * np.log(2.0 * np.pi) - 0.5 * np.linalg.slogdet(H)[1]
    rows = []
    with get_context("spawn").Pool(os.cpu_count()) as pool:
        for nu, infl, seed in ((8.0, 1.1, 1), (30.0, 1.0, 2)):
            rows.append((nu, infl, 200000) + importance(pool, w0, H, nu, infl, 200000, seed))
    z = np.array([r[3] for r in rows])
    se = np.array([r[4] for r in rows])
    best = float(np.sum(z / se**2) / np.sum(1 / se**2))
    best_se = float(1.0 / np.sqrt(np.sum(1 / se**2)))
    path = os.path.join(HERE, "logreg_d100_is.txt")
    with open(path, "w") as f:
        f.write("# evidence of the logreg_d100 workload, seed 0 data (d = 100, N = 10000 bf16-exact rows, N(0, I) prior),\n")
        f.write("# by importance sampling (multivariate t proposals at the posterior mode, scale H^-1), weights from\n")
        f.write("# the FP64 checker's log likelihood and log prior;\n")
        f.write("# written by tests/golden/make_logreg_is.py\n")
        f.write(f"# mode: log posterior {lp0:.6f}; Laplace logZ {laplace:.6f}\n")
        for nu, infl, n, lz, s, ess in rows:
            f.write(f"# t proposal nu = {nu:g}, scale x {infl:g}, {n} samples: logZ {lz:.6f} +- {s:.6f}, ESS {ess:.0f}\n")
        f.write("# name value standard_error\n")
        f.write(f"logreg_d100_seed0_logZ {best:.6f} {best_se:.6f}\n")
    print(open(path).read())


if __name__ == "__main__":
    main()
