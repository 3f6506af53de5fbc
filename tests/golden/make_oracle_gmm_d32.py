"""Writes oracle_gmm_d32_logz.txt: the FP64 CPU checker's evidence for the
20 seeds of the gmm_d32 workload (d = 32, 4-component mixture, n_live = 1000,
k = 500, p = 3d), or oracle_gmm_d32_p<c>d_logz.txt for the same seeds at
p = c d.  Calls only the checker (oracle/) and the input generators.

    python tests/golden/make_oracle_gmm_d32.py [n_workers] [c]
"""
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def one(args):
    seed, c = args
    import oracle as O
    from paper_2601_23252_gb300 import workloads as W
    wl = W.gmm_d32(seed=seed)
    if c != 3:
        wl = wl.with_(p=c * wl.d)
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed, run_id=wl.run_id, w=wl.w, tol=wl.tol)
    r = O.run(pb, op)
    lz, err, _ = O.finalise(r["logL"], r["nlive"], 100, wl.seed, wl.run_id)
    return seed, lz, err, r["logZ_det"], r["iters"], r["evals"]


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    c = int(sys.argv[2]) if len(sys.argv) > 2 else 3
    name = "oracle_gmm_d32_logz.txt" if c == 3 else f"oracle_gmm_d32_p{c}d_logz.txt"
    with get_context("spawn").Pool(n) as pool:
        rows = sorted(pool.map(one, [(s, c) for s in range(20)], chunksize=1))
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# FP64 checker, gmm_d32 workload (d=32, 4 comps, sigma 0.02, m=1000, k=500, p={32 * c}),\n")
        f.write("# written by tests/golden/make_oracle_gmm_d32.py\n")
        f.write("# seed logZ logZ_err logZ_det iters evals\n")
        for s, lz, err, det, it, ev in rows:
            f.write(f"{s} {lz:.10f} {err:.10f} {det:.10f} {it} {ev}\n")
