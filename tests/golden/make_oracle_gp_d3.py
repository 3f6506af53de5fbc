"""Writes oracle_gp_d3_logz.txt: the FP64 CPU checker's evidence for 8
sampling seeds of the full-size GP hyperparameter workload (gp_d3 seed 0
data: n = 256, m = 500, k = 250, p = 15).  Calls only the checker (oracle/)
and the input generators.  About half an hour per run on one core.

    python tests/golden/make_oracle_gp_d3.py [n_workers]
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
    wl = W.gp_d3(seed=0).with_(seed=seed)
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed, run_id=wl.run_id, w=wl.w, tol=wl.tol)
    r = O.run(pb, op)
    lz, err, _ = O.finalise(r["logL"], r["nlive"], 100, wl.seed, wl.run_id)
    return seed, lz, err, r["logZ_det"], r["iters"], r["evals"]


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    with get_context("spawn").Pool(n) as pool:
        rows = sorted(pool.map(one, range(8)))
    with open(os.path.join(HERE, "oracle_gp_d3_logz.txt"), "w") as f:
        f.write("# FP64 checker, gp_d3 (seed 0 data: n = 256, RBF + white kernel, log-uniform priors), m=500, k=250, p=15\n")
        f.write("# sampling seeds 0..7; written by tests/golden/make_oracle_gp_d3.py\n")
        f.write("# seed logZ logZ_err logZ_det iters evals\n")
        for s, lz, err, det, it, ev in rows:
            f.write(f"{s} {lz:.10f} {err:.10f} {det:.10f} {it} {ev}\n")
