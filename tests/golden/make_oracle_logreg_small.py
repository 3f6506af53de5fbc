"""Writes oracle_logreg_small_logz.txt: the FP64 CPU checker's evidence for 12
seeds of the reduced logistic-regression workload (N = 1000 rows, d = 10,
N(0,1) prior, n_live = 200, k = 100, p = 2d).  Calls only the checker
(oracle/) and the input generators.

    python tests/golden/make_oracle_logreg_small.py [n_workers]
"""
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def one(seed):
    import oracle as O
    from paper_2601_23252_gb300 import workloads as W
    wl = W.logreg_d100(seed=seed, n_rows=1000, d=10, n_live=200, k=100)
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed, run_id=wl.run_id, w=wl.w, tol=wl.tol)
    r = O.run(pb, op)
    lz, err, _ = O.finalise(r["logL"], r["nlive"], 100, wl.seed, wl.run_id)
    return seed, lz, err, r["logZ_det"], r["iters"], r["evals"]


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    with get_context("spawn").Pool(n) as pool:
        rows = sorted(pool.map(one, range(12)))
    with open(os.path.join(HERE, "oracle_logreg_small_logz.txt"), "w") as f:
        f.write("# FP64 checker, logistic regression N=1000 d=10 (bf16-exact X), N(0,1) prior, m=200, k=100, p=20\n")
        f.write("# written by tests/golden/make_oracle_logreg_small.py\n")
        f.write("# seed logZ logZ_err logZ_det iters evals\n")
        for s, lz, err, det, it, ev in rows:
            f.write(f"{s} {lz:.10f} {err:.10f} {det:.10f} {it} {ev}\n")
