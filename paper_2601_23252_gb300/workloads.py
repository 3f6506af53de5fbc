"""Seeded synthetic workloads shaped like the paper's problems.

This module only draws inputs: problem definitions (prior bounds, likelihood
parameters, data sets) and the sampler settings of each workload.  It holds
none of the sampling method's arithmetic, so both the CUDA path and the CPU
checker can be fed from it.  Setup data come from numpy's PCG64 stream seeded
with ``[seed, workload id]``; the sampler's own random numbers are drawn by
each implementation from the counter-based Philox stream keyed by
``(seed, run_id)``.

Workloads (sizes follow Sec. 4 and App. B.3 of arxiv 2601.23252):

* ``gauss_d2``   -- d=2, uniform prior on [0,1]^2, isotropic Gaussian
  likelihood N(0.5, 0.1^2 I) (normalised); m=500, k=250, p=5d.
* ``gmm_d32``    -- d=32, uniform prior on [0,1]^32, equal-weight mixture of 4
  isotropic Gaussians, sigma=0.02, means uniform in [0.2,0.8]^32;
  m=1000, k=500, p=3d.
* ``logreg_d100`` -- d=100, N(0,1) prior, N=10000 rows of i.i.d. N(0,1)
  features rounded to bfloat16 (the data set is the rounded matrix), labels
  Bernoulli(sigmoid(X w_true)), w_true ~ N(0, I); m=2000, k=1000, p=2d.
* ``gp_d3``      -- d=3, GP regression, n=256 inputs uniform on [0,10],
  y = sin(x) + N(0, 0.1^2); log-uniform priors on lengthscale [0.01,10],
  amplitude [0.01,10] and noise [1e-3,1] (uniform boxes in log space);
  m=500, k=250, p=15.
* ``batch64``    -- 64 independent Gaussian problems under uniform priors on
  [0,1]^d, d uniform in {4..64}, sigma log-uniform in [0.01,0.1], mean 0.5;
  m=500, k=250, p=3d each.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    d: int
    prior: str                      # "box" or "gauss"
    a: np.ndarray                   # box lower bounds / prior means
    b: np.ndarray                   # box upper bounds / prior std devs
    lik: str                        # "gauss", "gmm", "logreg", "gp", "flat"
    n_live: int
    k: int
    p: int
    sigma: float = 1.0
    mu: Optional[np.ndarray] = None     # [n_comp, d]
    X: Optional[np.ndarray] = None      # logistic design [N, d] (float32, bf16-exact)
    y: Optional[np.ndarray] = None      # logistic labels / GP targets
    t: Optional[np.ndarray] = None      # GP inputs
    w: float = 1.0                      # slice width in the whitened metric
    tol: float = 1e-3
    seed: int = 0
    run_id: int = 0
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def oracle_kwargs(self) -> dict:
        """Keyword arguments for the CPU checker's problem constructor."""
        kw = {"sigma": self.sigma}
        if self.mu is not None:
            kw["mu"] = self.mu
        if self.lik == "logreg":
            kw["X"], kw["y"] = self.X.astype(np.float64), self.y.astype(np.float64)
        if self.lik == "gp":
            kw["t"], kw["y"] = self.t, self.y
        if self.lik == "rastrigin":
            kw["alpha"] = float(self.extra.get("alpha", 0.5))
        return kw


def _rng(seed: int, wid: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(wid)])


def to_bf16_exact(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); float32 out."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = ((u >> 16) & 1) + 0x7FFF
    r = ((u + bias) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def gauss_d2(seed: int = 0, run_id: int = 0) -> Workload:
    d = 2
    return Workload("gauss_d2", d, "box", np.zeros(d), np.ones(d), "gauss", 500, 250, 5 * d,
                    sigma=0.1, mu=np.full((1, d), 0.5), seed=seed, run_id=run_id)


def gmm_d32(seed: int = 0, run_id: int = 0, n_live: int = 1000, k: int = 500) -> Workload:
    d, K = 32, 4
    mu = _rng(seed, 2).uniform(0.2, 0.8, size=(K, d))
    return Workload("gmm_d32", d, "box", np.zeros(d), np.ones(d), "gmm", n_live, k, 3 * d,
                    sigma=0.02, mu=mu, seed=seed, run_id=run_id)


def logreg_d100(seed: int = 0, run_id: int = 0, n_rows: int = 10000, d: int = 100,
                n_live: int = 2000, k: int = 1000) -> Workload:
    g = _rng(seed, 3)
    X = to_bf16_exact(g.standard_normal((n_rows, d)).astype(np.float32))
    w_true = g.standard_normal(d)
    logits = X.astype(np.float64) @ w_true
    y = (g.uniform(size=n_rows) < 1.0 / (1.0 + np.exp(-logits))).astype(np.float32)
    return Workload("logreg_d100", d, "gauss", np.zeros(d), np.ones(d), "logreg", n_live, k,
                    2 * d, X=X, y=y, seed=seed, run_id=run_id, extra={"w_true": w_true})


def gp_d3(seed: int = 0, run_id: int = 0, n: int = 256) -> Workload:
    g = _rng(seed, 4)
    t = g.uniform(0.0, 10.0, size=n)
    y = np.sin(t) + 0.1 * g.standard_normal(n)
    a = np.log(np.array([0.01, 0.01, 1e-3]))
    b = np.log(np.array([10.0, 10.0, 1.0]))
    return Workload("gp_d3", 3, "box", a, b, "gp", 500, 250, 15, t=t, y=y, seed=seed,
                    run_id=run_id)


def rastrigin_mix(d: int, alpha: float = 0.5, seed: int = 0, run_id: int = 0, n_live: int = 500,
                  k: int = 250) -> Workload:
    """Gaussian-Rastrigin mixture of App. F.3 on the box [-5.14, 5.14]^d, p = 3d."""
    r = 5.14
    return Workload("rastrigin", d, "box", np.full(d, -r), np.full(d, r), "rastrigin", n_live, k, 3 * d,
                    seed=seed, run_id=run_id, extra={"alpha": float(alpha)})


def batch64(seed: int = 0, n_runs: int = 64) -> list[Workload]:
    g = _rng(seed, 5)
    out = []
    for r in range(n_runs):
        d = int(g.integers(4, 65))
        sigma = float(np.exp(g.uniform(np.log(0.01), np.log(0.1))))
        out.append(Workload("batch64", d, "box", np.zeros(d), np.ones(d), "gauss", 500, 250, 3 * d,
                            sigma=sigma, mu=np.full((1, d), 0.5), seed=seed, run_id=r))
    return out


def gauss20_paper(seed: int = 0, n_live: int = 500, k: int = 250) -> Workload:
    """20-d Gaussian of the overhead study (App. B.2): prior N(0, I), likelihood
    N(x; 1, 0.01 I), normalised."""
    d = 20
    return Workload("gauss20", d, "gauss", np.zeros(d), np.ones(d), "gauss", n_live, k, d,
                    sigma=0.1, mu=np.ones((1, d)), seed=seed)


WORKLOADS = {"gauss_d2": gauss_d2, "gmm_d32": gmm_d32, "logreg_d100": logreg_d100,
             "gp_d3": gp_d3}
