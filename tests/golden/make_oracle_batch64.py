"""Writes oracle_batch64_logz.txt: the FP64 CPU checker's evidence for each of
the 64 runs of the batch64 workload (seed 0: d uniform in {4..64}, sigma
log-uniform in [0.01, 0.1], uniform prior on [0,1]^d, n_live = 500, k = 250,
p = 3d), or oracle_batch64_p<c>d_logz.txt for the same runs at p = c d.
Calls only the checker (oracle/) and the input generators.

    python tests/golden/make_oracle_batch64.py [n_workers] [c]
"""
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def one(args):
    r, c = args
    import oracle as O
    from paper_2601_23252_gb300 import workloads as W
    wl = W.batch64(seed=0)[r]
    if c != 3:
        wl = wl.with_(p=c * wl.d)
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed, run_id=wl.run_id, w=wl.w, tol=wl.tol)
    res = O.run(pb, op)
    lz, err, _ = O.finalise(res["logL"], res["nlive"], 100, wl.seed, wl.run_id)
    return r, wl.d, wl.sigma, lz, err, res["logZ_det"], res["iters"], res["evals"]


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    c = int(sys.argv[2]) if len(sys.argv) > 2 else 3
    name = "oracle_batch64_logz.txt" if c == 3 else f"oracle_batch64_p{c}d_logz.txt"
    # costliest runs first, so the pool's tail is short
    from paper_2601_23252_gb300 import workloads as W
    order = sorted(range(64), key=lambda r: -W.batch64(seed=0)[r].d)
    with get_context("spawn").Pool(n) as pool:
        rows = sorted(pool.map(one, [(r, c) for r in order], chunksize=1))
    with open(os.path.join(HERE, name), "w") as f:
        f.write("# FP64 checker, batch64 workload seed 0 (64 Gaussian runs, d in {4..64}, sigma in [0.01, 0.1],\n")
        f.write(f"# m=500, k=250, p={c}d), written by tests/golden/make_oracle_batch64.py\n")
        f.write("# run d sigma logZ logZ_err logZ_det iters evals\n")
        for r, d, sg, lz, err, det, it, ev in rows:
            f.write(f"{r} {d} {sg:.10f} {lz:.10f} {err:.10f} {det:.10f} {it} {ev}\n")
