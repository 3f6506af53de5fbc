"""FP64 CPU oracle of Nested Slice Sampling (arxiv 2601.23252), ctypes binding.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the product path never
does.  The arithmetic lives in ``nss_oracle.c`` (plain C, double precision);
this file only marshals numpy arrays.  It shares nothing with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nss_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PRIOR_BOX, PRIOR_GAUSS = 0, 1
LIK_GAUSS, LIK_GMM, LIK_LOGREG, LIK_GP, LIK_FLAT, LIK_RASTRIGIN = 0, 1, 2, 3, 4, 5

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Problem(C.Structure):
    _fields_ = [
        ("prior_kind", C.c_int), ("d", C.c_int), ("a", _dp), ("b", _dp),
        ("lik_kind", C.c_int), ("n_comp", C.c_int), ("n_data", C.c_int),
        ("sigma", C.c_double), ("alpha", C.c_double),
        ("mu", _dp), ("X", _dp), ("y", _dp), ("t", _dp),
    ]


class _Opts(C.Structure):
    _fields_ = [
        ("n_live", C.c_int), ("k", C.c_int), ("p", C.c_int), ("w", C.c_double),
        ("dir_norm", C.c_int), ("cov_eps", C.c_double), ("tol", C.c_double),
        ("max_iter", C.c_int), ("seed", C.c_uint64), ("run_id", C.c_uint32),
        ("kernel", C.c_int), ("rw_scale", C.c_double),
    ]


class _Trace(C.Structure):
    _fields_ = [
        ("dead_idx", _ip), ("parent", _ip), ("L", _dp), ("new_x", _dp), ("new_logL", _dp),
        ("evals", _ip), ("accepts", _ip), ("nulls", _ip), ("expansions", _ip),
        ("shrinks", _ip), ("cap_out", _ip),
        ("margin", _dp), ("pmargin", _dp), ("bmargin", _dp),
        ("logLstar", C.c_double), ("logZ", C.c_double), ("logX", C.c_double), ("done", C.c_int),
    ]


class _Summary(C.Structure):
    _fields_ = [
        ("n_dead", C.c_longlong), ("iters", C.c_int), ("evals", C.c_longlong),
        ("nulls", C.c_longlong), ("cap_out", C.c_longlong),
        ("logZ_det", C.c_double), ("logX", C.c_double), ("status", C.c_int),
    ]


class _Counts(C.Structure):
    _fields_ = [
        ("evals", C.c_int), ("accepts", C.c_int), ("nulls", C.c_int), ("expansions", C.c_int),
        ("shrinks", C.c_int), ("cap_out", C.c_int),
        ("margin", C.c_double), ("pmargin", C.c_double), ("bmargin", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile nss_oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.orc_u24.restype = C.c_double
            L.orc_u24.argtypes = [C.c_uint32]
            L.orc_u53.restype = C.c_double
            L.orc_u53.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_loglik.restype = C.c_double
            L.orc_loglik.argtypes = [C.POINTER(_Problem), _dp]
            L.orc_log_prior.restype = C.c_double
            L.orc_log_prior.argtypes = [C.POINTER(_Problem), _dp]
            L.orc_in_support.argtypes = [C.POINTER(_Problem), _dp]
            L.orc_prior_draw.argtypes = [C.POINTER(_Problem), C.c_uint64, C.c_uint32, C.c_uint32, _dp]
            L.orc_select.argtypes = [C.c_int, C.c_int, _dp, _ip, _ip, _dp]
            L.orc_evidence_death.argtypes = [C.c_double, C.c_int, _dp, _dp]
            L.orc_should_stop.argtypes = [C.c_int, _dp, C.c_double, C.c_double, C.c_double]
            L.orc_covariance.argtypes = [C.c_int, C.c_int, _dp, _dp]
            L.orc_metric.argtypes = [C.c_int, C.c_int, _dp, C.c_double, _dp]
            L.orc_parents.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, _ip, _ip]
            L.orc_hrss_step.argtypes = [C.POINTER(_Problem), _dp, C.c_double, C.c_int, C.c_double,
                                        C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                        _dp, _dp, C.POINTER(_Counts)]
            L.orc_step.argtypes = [C.POINTER(_Problem), C.POINTER(_Opts), C.c_uint32,
                                   _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _ip,
                                   C.POINTER(C.c_longlong), C.c_longlong, C.POINTER(_Trace),
                                   C.POINTER(C.c_longlong)]
            L.orc_init_live.argtypes = [C.POINTER(_Problem), C.POINTER(_Opts), _dp, _dp, _dp]
            L.orc_run.argtypes = [C.POINTER(_Problem), C.POINTER(_Opts), _dp, _dp, _dp, _ip,
                                  C.c_longlong, C.POINTER(_Summary)]
            L.orc_finalise.argtypes = [C.c_longlong, _dp, _ip, C.c_int, C.c_uint64, C.c_uint32,
                                       _dp, _dp, _dp, _dp]
            L.orc_volume_trajectory.argtypes = [C.c_longlong, _ip, C.c_int, C.c_uint64, C.c_uint32,
                                                _dp]
            L.orc_rw_step.argtypes = [C.POINTER(_Problem), _dp, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                      C.c_uint32, C.c_uint32, C.c_uint32, _dp, _dp, C.POINTER(_Counts)]
            L.orc_posterior_expectation.argtypes = [C.POINTER(_Problem), C.c_int, C.c_longlong, _dp, _dp, _dp]
            L.orc_posterior_expectation.restype = C.c_int
            L.orc_u_star.restype = C.c_double
            L.orc_phi.restype = C.c_double
            L.orc_phi.argtypes = [C.c_double]
            L.orc_kappa_inf.restype = C.c_double
            L.orc_mean_chord_ball.restype = C.c_double
            L.orc_mean_chord_ball.argtypes = [C.c_int, C.c_double]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


class Problem:
    """A prior and a likelihood in FP64, holding its arrays alive.

    prior: ("box", a, b) or ("gauss", mean, sd); likelihood kinds:
    gauss (mu, sigma), gmm (mu[K,d], sigma), logreg (X[N,d], y[N]),
    gp (t[n], y[n]), flat, rastrigin (alpha).
    """

    def __init__(self, prior, lik, **kw):
        kind, a, b = prior
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.d = int(self.a.size)
        self._keep = []
        s = _Problem()
        s.prior_kind = PRIOR_BOX if kind == "box" else PRIOR_GAUSS
        s.d = self.d
        s.a, s.b = _d(self.a), _d(self.b)
        s.lik_kind = {"gauss": LIK_GAUSS, "gmm": LIK_GMM, "logreg": LIK_LOGREG, "gp": LIK_GP,
                      "flat": LIK_FLAT, "rastrigin": LIK_RASTRIGIN}[lik]
        s.sigma = float(kw.get("sigma", 1.0))
        s.alpha = float(kw.get("alpha", 0.0))
        s.n_comp = 1
        s.n_data = 0
        if "mu" in kw:
            mu = np.ascontiguousarray(kw["mu"], dtype=np.float64).reshape(-1, self.d)
            self._keep.append(mu)
            s.mu = _d(mu)
            s.n_comp = mu.shape[0]
        if "X" in kw:
            X = np.ascontiguousarray(kw["X"], dtype=np.float64)
            y = np.ascontiguousarray(kw["y"], dtype=np.float64)
            self._keep += [X, y]
            s.X, s.y, s.n_data = _d(X), _d(y), X.shape[0]
        if "t" in kw:
            t = np.ascontiguousarray(kw["t"], dtype=np.float64)
            y = np.ascontiguousarray(kw["y"], dtype=np.float64)
            self._keep += [t, y]
            s.t, s.y, s.n_data = _d(t), _d(y), t.size
        self.s = s
        self.nonflat = kind != "box"

    def loglik(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.ndim == 1:
            return lib().orc_loglik(C.byref(self.s), _d(x))
        return np.array([lib().orc_loglik(C.byref(self.s), _d(np.ascontiguousarray(r))) for r in x])

    def log_prior(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return lib().orc_log_prior(C.byref(self.s), _d(x))

    def in_support(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return bool(lib().orc_in_support(C.byref(self.s), _d(x)))


KERNEL_HRSS, KERNEL_RW = 0, 1


def make_opts(n_live, k, p, seed=0, run_id=0, w=1.0, dir_norm=0, cov_eps=1e-6, tol=1e-3,
              max_iter=100000, kernel=KERNEL_HRSS, rw_scale=0.0):
    o = _Opts()
    o.n_live, o.k, o.p, o.w, o.dir_norm = n_live, k, p, float(w), int(dir_norm)
    o.cov_eps, o.tol, o.max_iter = float(cov_eps), float(tol), int(max_iter)
    o.seed, o.run_id = int(seed), int(run_id)
    o.kernel, o.rw_scale = int(kernel), float(rw_scale)
    return o


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u24(w):
    return lib().orc_u24(int(w) & 0xFFFFFFFF)


def u53(a, b):
    return lib().orc_u53(int(a) & 0xFFFFFFFF, int(b) & 0xFFFFFFFF)


def init_live(pb: Problem, opts):
    m, d = opts.n_live, pb.d
    x = np.empty((m, d)); logL = np.empty(m); birth = np.empty(m)
    lib().orc_init_live(C.byref(pb.s), C.byref(opts), _d(x), _d(logL), _d(birth))
    return x, logL, birth


def select(logL, k):
    logL = np.ascontiguousarray(logL, dtype=np.float64)
    m = logL.size
    dead = np.empty(k, np.int32); surv = np.empty(m - k, np.int32); ls = C.c_double()
    lib().orc_select(m, k, _d(logL), _i(dead), _i(surv), C.byref(ls))
    return dead, surv, ls.value


def evidence_death(logL, n, logZ, logX):
    z, x = C.c_double(logZ), C.c_double(logX)
    lib().orc_evidence_death(float(logL), int(n), C.byref(z), C.byref(x))
    return z.value, x.value


def should_stop(logL, logZ, logX, tol):
    logL = np.ascontiguousarray(logL, dtype=np.float64)
    return bool(lib().orc_should_stop(logL.size, _d(logL), float(logZ), float(logX), float(tol)))


def covariance(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    m, d = X.shape
    S = np.empty((d, d))
    lib().orc_covariance(m, d, _d(X), _d(S))
    return S


def metric(X, eps=1e-6):
    X = np.ascontiguousarray(X, dtype=np.float64)
    m, d = X.shape
    L = np.empty((d, d))
    st = lib().orc_metric(m, d, _d(X), float(eps), _d(L))
    return L, st


def parents(seed, run_id, it, m, k, surv):
    surv = np.ascontiguousarray(surv, dtype=np.int32)
    par = np.empty(k, np.int32)
    lib().orc_parents(int(seed), int(run_id), int(it), m, k, _i(surv), _i(par))
    return par


def hrss_step(pb: Problem, L, w, dir_norm, logLstar, seed, run_id, it, chain, step, x, logLx):
    """One HRSS step from x (modified copy returned) and its counters."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    lx = C.c_double(logLx)
    cnt = _Counts()
    cnt.margin = cnt.pmargin = cnt.bmargin = np.inf
    lib().orc_hrss_step(C.byref(pb.s), _d(L), float(w), int(dir_norm), float(logLstar), int(seed),
                        int(run_id), int(it), int(chain), int(step), _d(x), C.byref(lx),
                        C.byref(cnt))
    return x, lx.value, {f: getattr(cnt, f) for f, _ in _Counts._fields_}


def rw_step(pb: Problem, L, scale, logLstar, seed, run_id, it, chain, step, x, logLx):
    """One constrained random-walk step from x (modified copy returned)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    lx = C.c_double(logLx)
    cnt = _Counts()
    cnt.margin = cnt.pmargin = cnt.bmargin = np.inf
    lib().orc_rw_step(C.byref(pb.s), _d(L), float(scale), float(logLstar), int(seed), int(run_id), int(it),
                      int(chain), int(step), _d(x), C.byref(lx), C.byref(cnt))
    return x, lx.value, {f: getattr(cnt, f) for f, _ in _Counts._fields_}


def step(pb: Problem, opts, it, x, logL, birth, logZ, logX):
    """One NS iteration on copies of the state; returns (state, trace dict)."""
    m, d, k = opts.n_live, pb.d, opts.k
    x = np.array(x, dtype=np.float64, order="C"); logL = np.array(logL, dtype=np.float64)
    birth = np.array(birth, dtype=np.float64)
    z, lx = C.c_double(logZ), C.c_double(logX)
    tr = {
        "dead_idx": np.empty(k, np.int32), "parent": np.empty(k, np.int32),
        "L": np.empty((d, d)), "new_x": np.empty((k, d)), "new_logL": np.empty(k),
        "evals": np.empty(k, np.int32), "accepts": np.empty(k, np.int32),
        "nulls": np.empty(k, np.int32), "expansions": np.empty(k, np.int32),
        "shrinks": np.empty(k, np.int32), "cap_out": np.empty(k, np.int32),
        "margin": np.empty(k), "pmargin": np.empty(k), "bmargin": np.empty(k),
    }
    t = _Trace()
    for f, _ in _Trace._fields_:
        if f in tr:
            setattr(t, f, _i(tr[f]) if tr[f].dtype == np.int32 else _d(tr[f]))
    ev = C.c_longlong(0)
    st = lib().orc_step(C.byref(pb.s), C.byref(opts), int(it), _d(x), _d(logL), _d(birth),
                        C.byref(z), C.byref(lx), None, None, None, None, None, 0, C.byref(t),
                        C.byref(ev))
    tr["logLstar"], tr["logZ"], tr["logX"], tr["done"] = t.logLstar, t.logZ, t.logX, t.done
    tr["status"] = st
    return (x, logL, birth, z.value, lx.value), tr


def run(pb: Problem, opts, cap=None):
    """Whole run; returns a dict with the dead points and the summary."""
    d = pb.d
    if cap is None:
        cap = opts.max_iter * opts.k + opts.n_live if opts.max_iter < 10**5 else 2_000_000
    dx = np.empty((cap, d)); dl = np.empty(cap); db = np.empty(cap); dn = np.empty(cap, np.int32)
    s = _Summary()
    lib().orc_run(C.byref(pb.s), C.byref(opts), _d(dx), _d(dl), _d(db), _i(dn), int(cap),
                  C.byref(s))
    n = s.n_dead
    return {
        "x": dx[:n].copy(), "logL": dl[:n].copy(), "birth": db[:n].copy(), "nlive": dn[:n].copy(),
        "n_dead": n, "iters": s.iters, "evals": s.evals, "logZ_det": s.logZ_det,
        "logX": s.logX, "status": s.status,
    }


def finalise(logL, nlive, R, seed, run_id, want_r=False):
    logL = np.ascontiguousarray(logL, dtype=np.float64)
    nlive = np.ascontiguousarray(nlive, dtype=np.int32)
    n = logL.size
    m, s = C.c_double(), C.c_double()
    lw = np.empty(n)
    lz = np.empty(R)
    lib().orc_finalise(n, _d(logL), _i(nlive), int(R), int(seed), int(run_id), C.byref(m),
                       C.byref(s), _d(lw), _d(lz))
    if want_r:
        return m.value, s.value, lw, lz
    return m.value, s.value, lw


GRAD_LIK_SIGMA, GRAD_LIK_MU, GRAD_PRIOR_LOG_PREC, GRAD_GP_NOISE_SCALE, MOMENT_MEAN = 0, 1, 2, 3, 4


def posterior_expectation(pb: Problem, kind, x, log_w):
    """Weighted posterior expectation over dead points (App. D.2 weights) and
    the Fisher-identity gradients of log Z (orc_posterior_expectation)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, pb.d)
    lw = np.ascontiguousarray(log_w, dtype=np.float64)
    out = np.empty(max(1, pb.d * max(1, pb.s.n_comp)))
    n = lib().orc_posterior_expectation(C.byref(pb.s), int(kind), x.shape[0], _d(x), _d(lw), _d(out))
    if n < 0:
        raise ValueError(f"kind {kind} does not apply to this problem")
    return out[:n].copy()


def volume_trajectory(nlive, r, seed, run_id):
    nlive = np.ascontiguousarray(nlive, dtype=np.int32)
    out = np.empty(nlive.size)
    lib().orc_volume_trajectory(nlive.size, _i(nlive), int(r), int(seed), int(run_id), _d(out))
    return out


def u_star():
    return lib().orc_u_star()


def phi(u):
    return lib().orc_phi(float(u))


def kappa_inf():
    return lib().orc_kappa_inf()


def mean_chord_ball(d, R):
    return lib().orc_mean_chord_ball(int(d), float(R))
