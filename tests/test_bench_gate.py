"""The bench's accuracy gate (host logic, no GPU): the closed forms it uses
equal the test suite's own restatement, and `pass` needs every clause the
metric states (|mean dlogZ| <= 0.1 nat against the closed forms, runs within
3 of their reported errors, and the paired checker clauses)."""
import numpy as np
import pytest

import bench
from closed_forms import box_gauss_logZ, box_gmm_logZ
from paper_2601_23252_gb300 import workloads as W


def test_closed_forms_match_the_tests_restatement():
    for w in W.batch64(seed=0):
        assert bench.truth_of(w) == pytest.approx(box_gauss_logZ(w.mu[0], w.sigma, w.a, w.b), abs=1e-10)
    g = W.gmm_d32(seed=3)
    assert bench.truth_of(g) == pytest.approx(box_gmm_logZ(g.mu, g.sigma, g.a, g.b), abs=1e-10)


def _fake(wls, shift, err, rng, noise):
    return [{"logZ": bench.truth_of(w) + shift + noise * rng.standard_normal(), "logZ_err": err} for w in wls]


@pytest.fixture(scope="module")
def wls():
    return W.batch64(seed=0)


def test_unbiased_runs_pass(wls):
    rng = np.random.default_rng(0)
    res = _fake(wls, 0.0, 0.4, rng, 0.4)
    more = [(wls, _fake(wls, 0.0, 0.4, rng, 0.4)) for _ in range(3)]
    g = bench.logz_gate(wls, res, more=more)
    assert g["n_runs"] == 256 and g["pass"]


def test_a_bias_above_0p1_nat_fails_the_gate(wls):
    rng = np.random.default_rng(1)
    res = _fake(wls, 0.25, 0.4, rng, 0.1)
    g = bench.logz_gate(wls, res)
    assert g["closed_form_within_3err"] and not g["mean_within_0p1_nat"] and not g["pass"]


def test_runs_far_outside_their_errors_fail_the_gate(wls):
    rng = np.random.default_rng(2)
    res = _fake(wls, 0.0, 0.05, rng, 0.4)  # scatter 8x the reported error
    g = bench.logz_gate(wls, res)
    assert not g["closed_form_within_3err"] and not g["pass"]


def test_checker_pairing_is_part_of_pass(wls):
    rng = np.random.default_rng(3)
    res = _fake(wls, 0.0, 0.4, rng, 0.05)
    agree = {i: (r["logZ"] + 0.01 * rng.standard_normal(), 0.4) for i, r in enumerate(res)}
    off = {i: (r["logZ"] - 0.5 + 0.01 * rng.standard_normal(), 0.4) for i, r in enumerate(res)}
    assert bench.logz_gate(wls, res, checker=agree)["pass"]
    g = bench.logz_gate(wls, res, checker=off)
    assert g["checker_runs_within_3err"] and not g["checker_mean_within_3se"] and not g["pass"]


class _FakeSampler:
    """Stands in for the CUDA sampler: every run returns its closed form."""

    def __init__(self, ws, stream=None):
        self.ws = ws

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def autotune(self, iters=3):
        return [{"id": 3, "lanes_per_chain": 8, "dims_per_lane": 4} for _ in self.ws]

    def run(self):
        return [{"logZ": bench.truth_of(w), "logZ_err": 0.3, "n_dead": 1000, "evals": 10**6} for w in self.ws]


def test_gmm_leg_pairs_each_p_with_the_checker_where_it_exists(monkeypatch):
    """The bench's gmm_d32 leg, driven by the stand-in sampler: every p row is
    gated against the closed forms, and the rows whose checker file exists
    (p = 3d always) carry the paired gate."""
    import os
    import types
    from conftest import golden_path
    from paper_2601_23252_gb300 import native
    monkeypatch.setattr(native, "Sampler", _FakeSampler)
    monkeypatch.setattr(bench, "timed_run", lambda s, stream, flush, fill=0.0: (10.0, s.run()))
    out = bench.leg_gmm(types.SimpleNamespace(cuda_stream=0), None)
    assert [r["p"] for r in out["rows"]] == [96, 192, 320, 640]
    assert out["gated_p"] == 96 and all(r["closed_form_pass"] for r in out["rows"])
    for r in out["rows"]:
        c = r["p"] // 32
        has = os.path.exists(golden_path("oracle_gmm_d32_logz.txt" if c == 3 else f"oracle_gmm_d32_p{c}d_logz.txt"))
        assert ("gate" in r) == has
        if has:
            assert "mean_dlogZ_vs_checker" in r["gate"]
