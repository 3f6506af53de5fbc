"""Thin ctypes binding over the C ABI of ``include/nss.h``.

Argument marshalling only: every step of the sampler runs in the CUDA
library ``libnss_gb300.so``.  There is no CPU fallback -- if the library is
missing or the GPU is absent the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnss_gb300.so")

NSS_OK, NSS_DONE = 0, 1
# posterior expectation kinds (include/nss.h)
GRAD_LIK_SIGMA, GRAD_LIK_MU, GRAD_PRIOR_LOG_PREC, GRAD_GP_NOISE_SCALE, MOMENT_MEAN = 0, 1, 2, 3, 4
STATUS = {0: "ok", 1: "done", -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
          -4: "dead-point store full", -5: "iteration cap reached", -6: "non-finite evidence",
          -7: "call out of order"}
PRIOR = {"box": 0, "gauss": 1}
LOGLIK = {"gauss": 0, "gmm": 1, "logreg": 2, "gp": 3, "flat": 4, "fault": 5, "rastrigin": 6}
K_NAMES = ["init", "prologue", "sweep", "terminate", "final_sort", "volsim", "weights", "other",
           "dirgen", "logits", "lr_slice", "gp_sweep"]
N_KINDS = len(K_NAMES)
PATH_BATCHED, PATH_PLAIN = 0, 1

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


class Prior(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int), ("a", _dp), ("b", _dp)]


class Loglik(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_comp", C.c_int), ("n_data", C.c_int), ("sigma", C.c_double),
                ("mu", _dp), ("X", _fp), ("y", _fp), ("gp_t", _dp), ("gp_y", _dp),
                ("fault_mode", C.c_int), ("fault_param", C.c_double), ("alpha", C.c_double)]


class Options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("run_id", C.c_uint32), ("w", C.c_double), ("w_rule", C.c_int),
                ("dir_norm", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("dead_capacity", C.c_longlong), ("n_sim", C.c_int), ("cov_eps", C.c_double),
                ("cuda_stream", C.c_void_p), ("sweep_cfg", C.c_int), ("kernel", C.c_int),
                ("rw_scale", C.c_double), ("path", C.c_int), ("run_groups", C.c_int),
                ("dir_fp32", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("iter", C.c_int), ("done", C.c_int), ("logLstar", C.c_float), ("logZ", C.c_double),
                ("logX", C.c_double), ("n_dead", C.c_longlong), ("evals", C.c_longlong),
                ("nulls", C.c_longlong), ("cap_out", C.c_longlong), ("nan_evals", C.c_longlong),
                ("spec_evals", C.c_longlong), ("group_rounds", C.c_longlong),
                ("active_group_rounds", C.c_longlong), ("metric_status", C.c_int), ("status", C.c_int)]


class Result(C.Structure):
    _fields_ = [("logZ", C.c_double), ("logZ_err", C.c_double), ("logZ_det", C.c_double),
                ("n_dead", C.c_longlong), ("iters", C.c_int), ("evals", C.c_longlong),
                ("nulls", C.c_longlong), ("cap_out", C.c_longlong), ("nan_evals", C.c_longlong),
                ("spec_evals", C.c_longlong), ("group_rounds", C.c_longlong),
                ("active_group_rounds", C.c_longlong), ("status", C.c_int)]


class State(C.Structure):
    _fields_ = [("iter", C.c_int), ("logZ", C.c_double), ("logX", C.c_double), ("n_dead", C.c_longlong)]


class Trace(C.Structure):
    _fields_ = [("dead_idx", _ip), ("parent", _ip), ("L", _fp), ("evals", _ip), ("accepts", _ip),
                ("nulls", _ip), ("expansions", _ip), ("shrinks", _ip), ("cap_out", _ip),
                ("new_x", _fp), ("new_logL", _fp), ("logLstar", C.c_float)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_longlong * 12), ("ms", C.c_double * 12), ("total_launches", C.c_longlong),
                ("h2d_bytes", C.c_longlong), ("d2h_bytes", C.c_longlong)]


_lib = None


def lib():
    """Load libnss_gb300.so (built in-tree by ``paper_2601_23252_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2601_23252_gb300.build` (there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    L.nss_options_default.argtypes = [P(Options)]
    L.nss_create.argtypes = [P(Prior), P(Loglik), C.c_int, C.c_int, C.c_int, P(Options), P(C.c_void_p)]
    L.nss_create_batch.argtypes = [C.c_int, P(Prior), P(Loglik), _ip, _ip, _ip, P(Options), P(C.c_void_p)]
    L.nss_step.argtypes = [C.c_void_p, P(StepInfo)]
    L.nss_run.argtypes = [C.c_void_p, P(Result)]
    L.nss_finalise.argtypes = [C.c_void_p, P(Result)]
    L.nss_reset.argtypes = [C.c_void_p, P(C.c_uint64)]
    L.nss_autotune.argtypes = [C.c_void_p, C.c_int, _ip]
    L.nss_set_cfg.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.nss_autotune_report.argtypes = [C.c_void_p, _dp]
    L.nss_get_cfg.argtypes = [C.c_void_p, C.c_int]
    L.nss_cfg_lanes.argtypes = [C.c_int]
    L.nss_cfg_dims.argtypes = [C.c_int]
    L.nss_get_dead.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_size_t, P(C.c_size_t)]
    L.nss_posterior_expectation.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]
    L.nss_reweight.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
    L.nss_export_state.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, P(State)]
    L.nss_import_state.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, P(State)]
    L.nss_step_trace.argtypes = [C.c_void_p, C.c_int, P(Trace)]
    L.nss_set_profiling.argtypes = [C.c_void_p, C.c_int]
    L.nss_get_profile.argtypes = [C.c_void_p, P(Profile)]
    L.nss_n_runs.argtypes = [C.c_void_p]
    L.nss_logreg_logits.argtypes = [_fp, C.c_int, C.c_int, _fp, C.c_int, _fp]
    L.nss_gp_loglik.argtypes = [_dp, _dp, C.c_int, _dp, C.c_int, _fp]
    L.nss_wait_selftest.argtypes = [C.c_uint, C.POINTER(C.c_int)]
    L.nss_volume_sim_static.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_uint64, C.c_uint32,
                                        C.c_void_p, C.c_void_p, C.c_void_p]
    L.nss_run_width.argtypes = [C.c_void_p, C.c_int]
    L.nss_run_width.restype = C.c_double
    L.nss_destroy.argtypes = [C.c_void_p]
    L.nss_destroy.restype = None
    L.nss_status_string.argtypes = [C.c_int]
    L.nss_status_string.restype = C.c_char_p
    L.nss_last_error.argtypes = [C.c_void_p]
    L.nss_last_error.restype = C.c_char_p
    _lib = L
    return L


class NSSError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)} ({status}): {msg}")
        self.status = status


def _ptr(a):
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class _Spec:
    """Marshalled problem of one run; keeps its arrays alive for the call."""

    def __init__(self, wl):
        self.a = np.ascontiguousarray(wl.a, dtype=np.float64)
        self.b = np.ascontiguousarray(wl.b, dtype=np.float64)
        self.prior = Prior(PRIOR[wl.prior], int(wl.d), self.a.ctypes.data_as(_dp), self.b.ctypes.data_as(_dp))
        lk = Loglik()
        lk.kind = LOGLIK[wl.lik]
        lk.sigma = float(wl.sigma)
        lk.n_comp = 1
        self.keep = []
        if wl.mu is not None:
            mu = np.ascontiguousarray(np.atleast_2d(np.asarray(wl.mu, dtype=np.float64)))
            self.keep.append(mu)
            lk.mu = mu.ctypes.data_as(_dp)
            lk.n_comp = mu.shape[0]
        if wl.lik == "logreg":
            X = np.ascontiguousarray(wl.X, dtype=np.float32)
            y = np.ascontiguousarray(wl.y, dtype=np.float32)
            self.keep += [X, y]
            lk.X, lk.y, lk.n_data = X.ctypes.data_as(_fp), y.ctypes.data_as(_fp), X.shape[0]
        if wl.lik == "gp":
            t = np.ascontiguousarray(wl.t, dtype=np.float64)
            y = np.ascontiguousarray(wl.y, dtype=np.float64)
            self.keep += [t, y]
            lk.gp_t, lk.gp_y, lk.n_data = t.ctypes.data_as(_dp), y.ctypes.data_as(_dp), t.size
        if wl.lik == "rastrigin":
            lk.alpha = float(wl.extra.get("alpha", 0.5))
        if wl.lik == "fault":
            lk.fault_mode = int(wl.extra.get("fault_mode", 1))
            lk.fault_param = float(wl.extra.get("fault_param", 0.0))
        self.loglik = lk
        o = Options()
        lib().nss_options_default(C.byref(o))
        o.seed, o.run_id, o.w, o.tol = int(wl.seed), int(wl.run_id), float(wl.w), float(wl.tol)
        for key, val in wl.extra.get("options", {}).items():
            setattr(o, key, val)
        self.opts = o


def volume_sim_static(logL, nlive, n_sim, seed, run_id, log_w, logZ_stats, n=None, stream=None):
    """Volume simulation into caller device buffers, with no device allocation
    (fixed library scratch).  logL (float32), nlive (int32), log_w (float64)
    and logZ_stats (float64, 2) are device tensors; n defaults to logL's size."""
    n = int(logL.numel()) if n is None else int(n)
    st = lib().nss_volume_sim_static(_ptr(logL), _ptr(nlive), n, int(n_sim), int(seed), int(run_id),
                                     _ptr(log_w), _ptr(logZ_stats), stream)
    if st != NSS_OK:
        raise NSSError(st, "nss_volume_sim_static")


def wait_selftest(max_polls=2000):
    """Device bounded-wait self-test: 2 when a wait on an mbarrier that nothing
    completes gave up after max_polls polls (the designed outcome), 1 if it
    completed."""
    out = C.c_int(0)
    st = lib().nss_wait_selftest(int(max_polls), C.byref(out))
    if st != NSS_OK:
        raise NSSError(st, "nss_wait_selftest")
    return out.value


def logreg_logits(X, U):
    """Z = U X^T by the tensor-core contraction of the logistic sweep (X as bf16,
    U split into three bf16 parts, FP32 accumulation)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    U = np.ascontiguousarray(U, dtype=np.float32)
    n, d = X.shape
    nu = U.shape[0]
    Z = np.empty((nu, n), np.float32)
    st = lib().nss_logreg_logits(X.ctypes.data_as(_fp), n, d, U.ctypes.data_as(_fp), nu, Z.ctypes.data_as(_fp))
    if st != NSS_OK:
        raise NSSError(st, "nss_logreg_logits")
    return Z


def gp_loglik(t, y, theta):
    """GP log-likelihood at each row of theta [m][3] = (ln l, ln a, ln s) by the
    tensor-core factorisation of the GP sweep (nss_gp_loglik); float32 [m]."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    out = np.empty(th.shape[0], np.float32)
    st = lib().nss_gp_loglik(t.ctypes.data_as(_dp), y.ctypes.data_as(_dp), t.size, th.ctypes.data_as(_dp),
                             th.shape[0], out.ctypes.data_as(_fp))
    if st != NSS_OK:
        raise NSSError(st, "nss_gp_loglik")
    return out


class Sampler:
    """One or many independent Nested Slice Sampling runs on the GPU.

    ``workloads``: a Workload (see ``workloads.py``) or a sequence of them; all
    of a batch advance together, one launch per kernel per iteration.
    """

    def __init__(self, workloads, stream: Optional[int] = None):
        wls = [workloads] if not isinstance(workloads, (list, tuple)) else list(workloads)
        self.workloads = wls
        self.n_runs = len(wls)
        specs = [_Spec(w) for w in wls]
        if stream is not None:
            for s in specs:
                s.opts.cuda_stream = C.c_void_p(int(stream))
        n = len(wls)
        pri = (Prior * n)(*[s.prior for s in specs])
        lik = (Loglik * n)(*[s.loglik for s in specs])
        opt = (Options * n)(*[s.opts for s in specs])
        m = (C.c_int * n)(*[w.n_live for w in wls])
        k = (C.c_int * n)(*[w.k for w in wls])
        p = (C.c_int * n)(*[w.p for w in wls])
        h = C.c_void_p()
        st = lib().nss_create_batch(n, pri, lik, m, k, p, opt, C.byref(h))
        if st != NSS_OK:
            raise NSSError(st, "nss_create_batch failed")
        self._h = h
        self._specs = specs

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().nss_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st, what):
        if st not in (NSS_OK, NSS_DONE):
            raise NSSError(st, f"{what}: {lib().nss_last_error(self._h).decode()}")
        return st

    # -- iteration ---------------------------------------------------------
    def step(self):
        info = (StepInfo * self.n_runs)()
        st = self._check(lib().nss_step(self._h, info), "nss_step")
        return st == NSS_DONE, [{f: getattr(i, f) for f, _ in StepInfo._fields_} for i in info]

    def run(self):
        res = (Result * self.n_runs)()
        self._check(lib().nss_run(self._h, res), "nss_run")
        return [{f: getattr(r, f) for f, _ in Result._fields_} for r in res]

    def reset(self, seeds=None):
        """Start every run again from a fresh prior draw (optionally new seeds)."""
        arr = None
        if seeds is not None:
            arr = (C.c_uint64 * self.n_runs)(*[int(v) for v in seeds])
        self._check(lib().nss_reset(self._h, arr), "nss_reset")

    def autotune(self, iters=3):
        """Pick the fastest sweep configuration per dimension class; resets the runs."""
        out = (C.c_int * self.n_runs)()
        self._check(lib().nss_autotune(self._h, int(iters), out), "nss_autotune")
        return [self.cfg_info(q) for q in out]

    def autotune_report(self):
        """Cost of every configuration tried by the last autotune (ms per 1e6 evals)."""
        arr = (C.c_double * 25)()
        self._check(lib().nss_autotune_report(self._h, arr), "nss_autotune_report")
        return {i: arr[i] for i in range(25) if arr[i] > 0}

    def set_cfg(self, run, cfg):
        self._check(lib().nss_set_cfg(self._h, run, cfg), "nss_set_cfg")

    def cfg(self, run=0):
        return self.cfg_info(lib().nss_get_cfg(self._h, run))

    @staticmethod
    def cfg_info(q):
        return {"id": int(q), "lanes_per_chain": lib().nss_cfg_lanes(q), "dims_per_lane": lib().nss_cfg_dims(q)}

    def finalise(self):
        res = (Result * self.n_runs)()
        self._check(lib().nss_finalise(self._h, res), "nss_finalise")
        return [{f: getattr(r, f) for f, _ in Result._fields_} for r in res]

    def width(self, run=0):
        return lib().nss_run_width(self._h, run)

    # -- data out ----------------------------------------------------------
    def n_dead(self, run=0):
        n = C.c_size_t()
        self._check(lib().nss_get_dead(self._h, run, None, None, None, None, None, 0, C.byref(n)), "nss_get_dead")
        return n.value

    def dead(self, run=0, weights=True, out=None):
        """Dead points of a run in death order (numpy host arrays, or caller
        buffers given in ``out``: dict of arrays/tensors, host or device)."""
        n = self.n_dead(run)
        d = self.workloads[run].d
        if out is None:
            out = {"x": np.empty((n, d), np.float32), "logL": np.empty(n, np.float32),
                   "birth": np.empty(n, np.float32), "nlive": np.empty(n, np.int32)}
            if weights:
                out["log_w"] = np.empty(n, np.float64)
        nn = C.c_size_t()
        self._check(lib().nss_get_dead(self._h, run, _ptr(out.get("x")), _ptr(out.get("logL")),
                                       _ptr(out.get("log_w")), _ptr(out.get("birth")),
                                       _ptr(out.get("nlive")), n, C.byref(nn)), "nss_get_dead")
        return out

    def posterior(self, kind, run=0):
        """Posterior expectation of a finished run computed on the device
        (nss_posterior_expectation): the Fisher-identity gradient of log Z for
        the GRAD_* kinds, the posterior mean for MOMENT_MEAN.  numpy FP64."""
        wl = self.workloads[run]
        k = wl.mu.shape[0] if (wl.mu is not None and wl.lik == "gmm") else 1
        count = {GRAD_LIK_SIGMA: 1, GRAD_LIK_MU: k * wl.d, GRAD_PRIOR_LOG_PREC: 1,
                 GRAD_GP_NOISE_SCALE: 1, MOMENT_MEAN: wl.d}[kind]
        out = np.empty(count, np.float64)
        self._check(lib().nss_posterior_expectation(self._h, run, int(kind), _ptr(out), count),
                    "nss_posterior_expectation")
        return out

    def reweight(self, beta, run=0):
        """log Z at inverse temperature beta from the same dead points, its
        spread over the simulated volumes, and the Kish ESS of the weights
        (nss_reweight)."""
        out = np.empty(3, np.float64)
        self._check(lib().nss_reweight(self._h, run, float(beta), _ptr(out)), "nss_reweight")
        return {"logZ": out[0], "logZ_err": out[1], "ess": out[2]}

    def export_state(self, run=0):
        wl = self.workloads[run]
        x = np.empty((wl.n_live, wl.d), np.float32)
        l = np.empty(wl.n_live, np.float32)
        b = np.empty(wl.n_live, np.float32)
        s = State()
        self._check(lib().nss_export_state(self._h, run, _ptr(x), _ptr(l), _ptr(b), C.byref(s)), "nss_export_state")
        return {"x": x, "logL": l, "birth": b, "iter": s.iter, "logZ": s.logZ, "logX": s.logX,
                "n_dead": s.n_dead}

    def import_state(self, run, x, logL, birth=None, iter=0, logZ=-np.inf, logX=0.0, n_dead=0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        logL = np.ascontiguousarray(logL, dtype=np.float32)
        bp = None
        if birth is not None:
            birth = np.ascontiguousarray(birth, dtype=np.float32)
            bp = _ptr(birth)
        s = State(int(iter), float(logZ), float(logX), int(n_dead))
        self._check(lib().nss_import_state(self._h, run, _ptr(x), _ptr(logL), bp, C.byref(s)), "nss_import_state")

    def trace(self, run=0):
        wl = self.workloads[run]
        k, d = wl.k, wl.d
        arrs = {f: np.empty(k, np.int32) for f in
                ("dead_idx", "parent", "evals", "accepts", "nulls", "expansions", "shrinks", "cap_out")}
        arrs["L"] = np.empty((d, d), np.float32)
        arrs["new_x"] = np.empty((k, d), np.float32)
        arrs["new_logL"] = np.empty(k, np.float32)
        t = Trace()
        for f, a in arrs.items():
            setattr(t, f, a.ctypes.data_as(_fp if a.dtype == np.float32 else _ip))
        self._check(lib().nss_step_trace(self._h, run, C.byref(t)), "nss_step_trace")
        arrs["logLstar"] = t.logLstar
        return arrs

    # -- profiling ---------------------------------------------------------
    def set_profiling(self, on=True):
        self._check(lib().nss_set_profiling(self._h, int(on)), "nss_set_profiling")

    def profile(self):
        p = Profile()
        self._check(lib().nss_get_profile(self._h, C.byref(p)), "nss_get_profile")
        return {"launches": {K_NAMES[i]: p.launches[i] for i in range(N_KINDS)},
                "ms": {K_NAMES[i]: p.ms[i] for i in range(N_KINDS)},
                "total_launches": p.total_launches, "h2d_bytes": p.h2d_bytes, "d2h_bytes": p.d2h_bytes}
