#!/usr/bin/env python3
"""Throughput of the batched Nested Slice Sampling sweep on GB300.

Metric: NS dead points per second (all deaths, including the final live
set) and logical likelihood evaluations per second.  One step is one whole
pass of the hot path -- initial prior draw, every outer iteration (selection,
evidence, metric, parents, HRSS sweep with the likelihood fused in,
replacement, termination test) and the post-hoc volume simulation -- over one
batch of independent runs of the workload:

  gmm_d32: d = 32, uniform prior on [0,1]^32, equal-weight mixture of 4
  isotropic Gaussians (sigma 0.02, means uniform in [0.2,0.8]^32 drawn from
  the seed), n_live = 1000, k = 500, p = 3d = 96; 20 seeds per batch.

`value` is measured with the inputs resident on the device (context created
before the timed region); `e2e` goes through the public API from host
buffers: create (problem upload), run, dead-point read-back, destroy.
Multi-GPU: independent replicas (one batch of different seeds per rank), no
data-path collective.  `--impl reference` times the FP64 CPU checker of the
same workload on the host cores (the slow reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NS dead points/s and logL evals/s vs plain path at |\u0394logZ|\u22640.1 nat, % roofline"
UNIT = "dead points/s"


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--runs", type=int, default=20, help="independent seeds per batch (per rank)")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-run-at-a-time comparator")
    ap.add_argument("--sweep-cfg", type=int, default=-1,
                    help="force this sweep configuration id instead of autotuning (profiling runs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU checker baseline")
    ap.add_argument("--ncu-case", action="store_true",
                    help="no timing: the bench batch for a few iterations, small dead stores "
                         "(the case captured by ncu)")
    ap.add_argument("--ncu-cfg", type=int, default=-1,
                    help="with --ncu-case: force this sweep configuration id instead of autotuning")
    ap.add_argument("--ncu-case-logreg", action="store_true",
                    help="no timing: one outer iteration of the full-size logistic-regression "
                         "workload (d=100, N=10000, k=1000, p=200), for ncu captures of its kernels")
    ap.add_argument("--ncu-case-gp", action="store_true",
                    help="no timing: two outer iterations of the GP workload (n=256, k=250, p=15), "
                         "for ncu captures of its sweep kernel")
    return ap.parse_args()


def gmm_logZ(mu, sigma):
    """Closed-form evidence of the equal-weight mixture under the [0,1]^d box."""
    from scipy import special
    lo = special.log_ndtr((0.0 - mu) / sigma)
    hi = special.log_ndtr((1.0 - mu) / sigma)
    per = np.sum(hi + np.log1p(-np.exp(lo - hi)), axis=1)
    return float(special.logsumexp(per) - np.log(len(per)))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources the sweep kernel is compiled from (its own files and the headers
# they include); a change elsewhere does not change the sweep's counters
SWEEP_SOURCES = ("nss_device.cuh", "nss_internal.h", "nss_kernels.h", "nss_sweep.cu", "nss_sweep_chain.cuh",
                 "nss_sweep_common.cuh", "nss_sweep_k1.cu", "nss_sweep_k4.cu", "nss_sweep_k8.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_23252_gb300", "csrc")
    for f in SWEEP_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_sweep_gmm_d32.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def sweep_flops(wl, evals, chain_steps):
    """Algorithmic FP32 operations of the sweep kernel: per logical evaluation
    the line point (2d) and K squared distances (3Kd) plus the K scalings and
    log-sum-exp adds (2K); per HRSS step the direction's norm, the box
    interval and the move (4d).  The whitening L z of each step (d(d+1)) is
    done by the direction kernel and is not counted here."""
    d, K = wl.d, (wl.mu.shape[0] if wl.mu is not None else 1)
    return evals * (2 * d + 3 * K * d + 2 * K) + chain_steps * (4 * d)


def cpu_checker_rate(budget_s=12.0, seed=0):
    """The FP64 checker on one seed of the workload, from the start, for about
    budget_s seconds of iterations: dead points per second on one core."""
    import oracle as O
    from paper_2601_23252_gb300 import workloads as W
    wl = W.gmm_d32(seed=seed)
    pb = O.Problem((wl.prior, wl.a, wl.b), wl.lik, **wl.oracle_kwargs())
    op = O.make_opts(wl.n_live, wl.k, wl.p, seed=wl.seed)
    t0 = time.perf_counter()
    x, l, b = O.init_live(pb, op)
    st, it, ev = (x, l, b, -np.inf, 0.0), 0, 0
    while time.perf_counter() - t0 < budget_s:
        st, tr = O.step(pb, op, it, *st)
        ev += int(tr["evals"].sum())
        it += 1
    dt = time.perf_counter() - t0
    return {"value": wl.k * it / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"gmm_d32 seed {seed}: prior draw + first {it} iterations ({wl.k * it} dead points, "
                      f"{ev} evals) in {dt:.1f} s, one thread", "evals_per_s": ev / dt}


def _cpu_worker(args):
    budget_s, seed = args
    return cpu_checker_rate(budget_s=budget_s, seed=seed)


def cpu_checker_rate_all_cores(budget_s=10.0, seed0=0):
    """The FP64 checker on every host core at once, one seed per process
    (spawned, so no CUDA state is inherited): the summed dead points/s."""
    import multiprocessing as mp
    import oracle as O
    O.lib()  # build once before the workers load it
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        rs = pool.map(_cpu_worker, [(budget_s, seed0 + i) for i in range(n)])
    v = float(sum(r["value"] for r in rs))
    ev = float(sum(r["evals_per_s"] for r in rs))
    return {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"gmm_d32 seeds {seed0}..{seed0 + n - 1}, one process per core, each the prior draw + "
                      f"the first iterations for {budget_s:.0f} s; summed dead points/s", "evals_per_s": ev}


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def rank_seeds(rank, nrun):
    """Each rank runs its own replicas: seeds rank*nrun .. rank*nrun + nrun - 1."""
    return [rank * nrun + s for s in range(nrun)]


def aggregate(total_ms, dead, evals, world, device):
    """Whole-job figures: the slowest rank's time, the dead points and
    evaluations summed over ranks (no exchange inside the timed region)."""
    import torch
    if world == 1:
        return float(total_ms), float(dead), float(evals)
    t = torch.tensor([total_ms, dead, evals], dtype=torch.float64, device=device)
    mx = t.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = t.clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_checker_rate(budget_s=1.0, seed=99)
    rates, evr, samples, cores = [], [], [], 1
    for s in range(args.steps):
        r = cpu_checker_rate_all_cores(budget_s=8.0, seed0=100 * s)
        rates.append(r["value"])
        evr.append(r["evals_per_s"])
        samples.append(r["sample"])
        cores = r["cores"]
    v = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 8000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "gmm_d32 (d=32, 4-component mixture, m=1000, "
                                            "k=500, p=96)", "sample_per_step": "8 s of checker iterations on every host core"},
            "evals_per_s": float(np.mean(evr)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": samples[0]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_native(args):
    import torch
    from paper_2601_23252_gb300 import native
    from paper_2601_23252_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    nrun = args.runs
    seeds = rank_seeds(rank, nrun)
    wls = [W.gmm_d32(seed=s) for s in seeds]
    truth = np.array([gmm_logZ(w.mu, w.sigma) for w in wls])
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 2**20 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    if args.sweep_cfg >= 0:
        wls = [w.with_(extra={"options": {"sweep_cfg": args.sweep_cfg}}) for w in wls]
    sampler = native.Sampler(wls, stream=stream.cuda_stream)
    chosen = sampler.autotune(iters=3) if args.sweep_cfg < 0 else [sampler.cfg(r) for r in range(nrun)]
    tune = {f"{native.Sampler.cfg_info(q)['lanes_per_chain']}x{native.Sampler.cfg_info(q)['dims_per_lane']}": round(v, 4)
            for q, v in sampler.autotune_report().items()}
    for _ in range(args.warmup):
        sampler.reset()
        sampler.run()
    torch.cuda.synchronize()
    sampler.set_profiling(True)
    clocks = Clocks(local)
    times, dead, evals, flops, launches, spec = [], 0, 0, 0.0, 0, 0
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    res = None
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))          # L2 flush between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sampler.reset()
        res = sampler.run()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        for wl, r in zip(wls, res):
            dead += r["n_dead"]
            evals += r["evals"]
            spec += r["spec_evals"]
            flops += sweep_flops(wl, r["evals"], r["iters"] * wl.k * wl.p)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof = sampler.profile()
    total_ms = float(np.sum(times))
    total_ms_all, dead_all, evals_all = aggregate(total_ms, dead, evals, world, dev)
    value = dead_all / (total_ms_all / 1e3)
    dlogZ = np.array([r["logZ"] for r in res]) - truth
    errs = np.array([r["logZ_err"] for r in res])

    # dominant kernel: the sweep
    sweep_ms = prof["ms"]["sweep"]
    sweep_launches = max(1, prof["launches"]["sweep"])
    peaks, src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = flops / (sweep_ms / 1e3) / 1e12 if sweep_ms > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (achieved / fp32_peak) if achieved else None, "traffic": ncu_traffic(),
                "kernel": f"k_sweep<{chosen[0]['lanes_per_chain']},{chosen[0]['dims_per_lane']}> (HRSS sweep, fused mixture likelihood)",
                "peak_source": f"FP32 FMA pipe: {sms} SMs x 128 lanes x 2 flop x "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({src} max clock)",
                "avg_launch_ms": sweep_ms / sweep_launches,
                "launch_ms_over_step_ms": sweep_ms / total_ms if total_ms > 0 else None}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gmm_d32", "d": 32, "n_comp": 4, "sigma": 0.02, "n_live": 1000,
                       "k": 500, "p": 96, "runs_per_gpu": nrun, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (512 MB write)",
                       "sweep_cfg": chosen[0], "autotune_ms_per_Meval": tune,
                       "evidence_accumulation": "f64"},
            "evals_per_s": evals_all / (total_ms_all / 1e3),
            "speculative_tests_per_eval": spec / max(1, evals),
            "gate": logz_gate(seeds, res, dlogZ, errs),
            "roofline": roofline, "gpu_launches": prof["total_launches"] // 1,
            "clocks": clk,
            "kernel_ms_per_step": {k: v / args.steps for k, v in prof["ms"].items() if v > 0}}
    sampler.close()

    # end to end through the public API from host buffers
    if rank == 0 or world > 1:
        e2e_t, e2e_dead, h2d, d2h = [], 0, 0, 0
        # the caller's pinned result buffers, allocated once (the seeds are the
        # timed steps', so every run's dead count is known)
        outs = [{"x": torch.empty((r["n_dead"], 32), dtype=torch.float32).pin_memory(),
                 "logL": torch.empty(r["n_dead"], dtype=torch.float32).pin_memory(),
                 "log_w": torch.empty(r["n_dead"], dtype=torch.float64).pin_memory()} for r in res]
        for s in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            wls_cfg = [w.with_(extra={"options": {"sweep_cfg": chosen[r]["id"]}}) for r, w in enumerate(wls)]
            with native.Sampler(wls_cfg, stream=stream.cuda_stream) as sm:
                rr = sm.run()
                for r in range(nrun):
                    n = rr[r]["n_dead"]
                    out = outs[r] if outs[r]["logL"].numel() == n else {
                        "x": torch.empty((n, 32), dtype=torch.float32).pin_memory(),
                        "logL": torch.empty(n, dtype=torch.float32).pin_memory(),
                        "log_w": torch.empty(n, dtype=torch.float64).pin_memory()}
                    sm.dead(r, out=out)
                p = sm.profile()
                h2d, d2h = p["h2d_bytes"], p["d2h_bytes"]
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
            e2e_dead = sum(r["n_dead"] for r in rr)
        line["e2e"] = {"value": e2e_dead / float(np.mean(e2e_t)), "unit": UNIT,
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": 1e3 * float(np.mean(e2e_t))}

    # plain comparator: the same runs one at a time (single-run contexts)
    if rank == 0 and world == 1 and not args.no_plain:
        t_plain, dead_plain, plain_dz = 0.0, 0, []
        for wl in wls[:4]:
            with native.Sampler(wl, stream=stream.cuda_stream) as sp:
                sp.autotune(iters=3)
                sp.run()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                sp.reset()
                e0.record(stream)
                r = sp.run()[0]
                e1.record(stream)
                e1.synchronize()
                t_plain += e0.elapsed_time(e1)
                dead_plain += r["n_dead"]
            # the same run alone in a context, in the batch's configuration:
            # batching itself must not move logZ
            q = len(plain_dz)
            with native.Sampler(wl.with_(extra={"options": {"sweep_cfg": chosen[q]["id"]}}),
                                stream=stream.cuda_stream) as sp:
                plain_dz.append(abs(sp.run()[0]["logZ"] - res[q]["logZ"]))
        line["single_run_path"] = {"value": dead_plain / (t_plain / 1e3), "unit": UNIT,
                                   "what": "the same kernels, one run per context (autotuned for one run), "
                                           "4 seeds one after another"}
        g = line["gate"]
        g["max_abs_dlogZ_vs_plain_path"] = float(max(plain_dz))
        g["pass"] = bool(g["max_abs_dlogZ_vs_plain_path"] <= 0.1 and g.get("checker_within_3se", True))
    if rank == 0 and world == 1 and not args.no_cpu:
        one = cpu_checker_rate()
        line["cpu_baseline"] = cpu_checker_rate_all_cores()
        line["cpu_baseline"]["one_thread"] = {"value": one["value"], "sample": one["sample"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def logz_gate(seeds, res, dlogZ, errs):
    """logZ of the batched runs against (i) the FP64 checker's runs of the same
    seeds (stored by tests/golden/make_oracle_gmm_d32.py; paired difference,
    its standard error over seeds), (ii) the closed form (the method's own
    bias on this workload, context only).  The plain single-run path is
    added by the caller when it runs."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_gmm_d32_logz.txt")
    ref = {}
    if os.path.exists(path):
        for ln in open(path):
            if ln.strip() and not ln.startswith("#"):
                f = ln.split()
                ref[int(f[0])] = (float(f[1]), float(f[2]))
    g = {"mean_dlogZ_vs_closed_form": float(dlogZ.mean()), "mean_err": float(errs.mean())}
    pairs = [(r["logZ"] - ref[sd][0]) for sd, r in zip(seeds, res) if sd in ref]
    if pairs:
        dz = np.array(pairs)
        se = float(dz.std(ddof=1) / np.sqrt(len(dz))) if len(dz) > 1 else float("nan")
        g.update({"mean_dlogZ_vs_checker": float(dz.mean()), "se_vs_checker": se, "n_checker_seeds": len(dz),
                  "checker_within_3se": bool(abs(dz.mean()) <= 3 * se)})
    g["pass"] = bool(g.get("checker_within_3se", False))
    return g


def run_ncu_case(args):
    """The bench's batch of runs for 6 outer iterations, then exit; dead
    stores sized for those iterations so the device footprint stays small."""
    from paper_2601_23252_gb300 import native
    from paper_2601_23252_gb300 import workloads as W
    opts = {"dead_capacity": 8 * 500 + 1000}
    if args.ncu_cfg >= 0:
        opts["sweep_cfg"] = args.ncu_cfg
    wls = [W.gmm_d32(seed=s).with_(extra={"options": dict(opts)}) for s in range(args.runs)]
    with native.Sampler(wls) as s:
        if args.ncu_cfg < 0:
            s.autotune(iters=2)
        for _ in range(6):
            s.step()
    return 0


def run_ncu_case_logreg(args):
    from paper_2601_23252_gb300 import native
    from paper_2601_23252_gb300 import workloads as W
    wl = W.logreg_d100(seed=0).with_(extra={"options": {"dead_capacity": 4 * 1000 + 2000}})
    with native.Sampler(wl) as s:
        s.set_profiling(True)   # launch by launch (no graph), so ncu sees each kernel
        s.step()
    return 0


def run_ncu_case_gp(args):
    from paper_2601_23252_gb300 import native
    from paper_2601_23252_gb300 import workloads as W
    wl = W.gp_d3(seed=0).with_(extra={"options": {"dead_capacity": 4 * 250 + 500}})
    with native.Sampler(wl) as s:
        s.step()
        s.step()
    return 0


def main():
    args = parse()
    if args.ncu_case:
        return run_ncu_case(args)
    if args.ncu_case_logreg:
        return run_ncu_case_logreg(args)
    if args.ncu_case_gp:
        return run_ncu_case_gp(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
