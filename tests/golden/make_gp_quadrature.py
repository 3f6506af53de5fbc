"""Writes gp_d3_quadrature.txt: the evidence of the full-size GP hyperparameter
workload (n = 256 data of gp_d3 seed 0: RBF + white kernel, log-uniform
priors on lengthscale, amplitude and noise, Sec. 4.3 shape) by brute-force
quadrature of the oracle's FP64 marginal likelihood.  Calls only the checker
(oracle/) and the input generators.

    Z = (1 / vol) int_box L(theta) d theta      (theta = log hyperparameters)

1. A coarse grid of cell centres over the whole prior box locates the mass
   (and would show a second mode).
2. The mode is refined by Nelder-Mead and the posterior covariance taken from
   a finite-difference Hessian of log L there.
3. Tensor Gauss-Legendre quadrature in the Hessian's principal axes over
   +-R standard deviations (points outside the prior box count zero), at two
   resolutions and two radii; their spread is the quadrature error.

    python tests/golden/make_gp_quadrature.py [n_workers]
"""
import os
import sys
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

_PB = None


def _problem():
    global _PB
    if _PB is None:
        import oracle as O
        from paper_2601_23252_gb300 import workloads as W
        wl = W.gp_d3(seed=0)
        _PB = (O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs()), wl.a, wl.b)
    return _PB


def _loglik_many(thetas):
    pb, a, b = _problem()
    out = np.empty(len(thetas))
    for i, th in enumerate(thetas):
        inside = np.all(th >= a) and np.all(th <= b)
        out[i] = pb.loglik(np.asarray(th, float)) if inside else -np.inf
    return out


def loglik_par(pool, thetas, chunks=64):
    parts = np.array_split(np.asarray(thetas), chunks)
    return np.concatenate(pool.map(_loglik_many, [p for p in parts if len(p)]))


def gl_axis(half, panels, order):
    xq, wq = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(-half, half, panels + 1)
    pts = np.concatenate([(e0 + e1) / 2 + (e1 - e0) / 2 * xq for e0, e1 in zip(edges[:-1], edges[1:])])
    wts = np.concatenate([(e1 - e0) / 2 * wq for e0, e1 in zip(edges[:-1], edges[1:])])
    return pts, wts


def main():
    from scipy import optimize, special
    n = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    _, a, b = _problem()
    vol = float(np.prod(b - a))
    with get_context("spawn").Pool(n) as pool:
        # 1. coarse cell-centre grid over the box
        nc = 28
        axes = [a[i] + (np.arange(nc) + 0.5) * (b[i] - a[i]) / nc for i in range(3)]
        grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
        lc = loglik_par(pool, grid)
        cell = vol / nc**3
        coarse_logZ = float(special.logsumexp(lc) + np.log(cell) - np.log(vol))
        top = grid[np.argsort(lc)[::-1][:5]]
        # 2. mode and Hessian
        pb, _, _ = _problem()
        f = lambda th: -pb.loglik(th) if np.all(th >= a) and np.all(th <= b) else np.inf
        res = optimize.minimize(f, top[0], method="Nelder-Mead",
                                options={"xatol": 1e-8, "fatol": 1e-10, "maxiter": 20000, "maxfev": 40000})
        mode = res.x
        h = 1e-3
        H = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                e_i, e_j = np.eye(3)[i] * h, np.eye(3)[j] * h
                H[i, j] = (f(mode + e_i + e_j) - f(mode + e_i - e_j) - f(mode - e_i + e_j) + f(mode - e_i - e_j)) / (4 * h * h)
        cov = np.linalg.inv(0.5 * (H + H.T))
        evals, evecs = np.linalg.eigh(cov)
        sd = np.sqrt(evals)
        laplace = float(-res.fun + 0.5 * np.log(np.linalg.det(2 * np.pi * cov)) - np.log(vol))
        # 3. Gauss-Legendre in the principal axes, theta = mode + V diag(sd) u
        rows = []
        for R, panels, order in ((8.0, 8, 6), (10.0, 10, 6), (10.0, 8, 8)):
            u, w = gl_axis(R, panels, order)
            U = np.stack(np.meshgrid(u, u, u, indexing="ij"), -1).reshape(-1, 3)
            Wt = np.prod(np.stack(np.meshgrid(w, w, w, indexing="ij"), -1).reshape(-1, 3), axis=1)
            TH = mode + (U * sd) @ evecs.T
            lv = loglik_par(pool, TH)
            jac = float(np.prod(sd))
            lz = float(special.logsumexp(lv + np.log(Wt)) + np.log(jac) - np.log(vol))
            rows.append((R, panels, order, len(U), lz))
    vals = np.array([r[4] for r in rows])
    best = float(vals[-1])
    spread = float(vals.max() - vals.min())
    with open(os.path.join(HERE, "gp_d3_quadrature.txt"), "w") as fo:
        fo.write("# evidence of the gp_d3 workload, seed 0 data (n = 256, RBF + white kernel, log-uniform priors),\n")
        fo.write("# by quadrature of the FP64 checker's marginal likelihood; written by tests/golden/make_gp_quadrature.py\n")
        fo.write(f"# coarse {nc}^3 cell-centre grid over the box: logZ {coarse_logZ:.6f}; top cells {np.round(top, 3).tolist()}\n")
        fo.write(f"# mode (log l, log a, log sn) {np.round(mode, 6).tolist()}, logL max {-res.fun:.6f}, "
                 f"principal sd {np.round(sd, 6).tolist()}, Laplace logZ {laplace:.6f}\n")
        for R, panels, order, npts, lz in rows:
            fo.write(f"# Gauss-Legendre in principal axes, +-{R:g} sd, {panels} panels x {order} nodes per axis "
                     f"({npts} points): logZ {lz:.8f}\n")
        fo.write("# name value quadrature_spread\n")
        fo.write(f"gp_d3_seed0_logZ {best:.8f} {spread:.2e}\n")
    print(open(os.path.join(HERE, "gp_d3_quadrature.txt")).read())


if __name__ == "__main__":
    main()
