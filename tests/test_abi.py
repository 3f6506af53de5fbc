"""The C ABI library builds, loads and exports every entry point that
include/nss.h declares; argument validation runs before any CUDA call."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "nss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nss_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_23252_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_abi_version_and_status_strings(lib):
    lib.nss_status_string.restype = C.c_char_p
    assert lib.nss_abi_version() == 7
    assert lib.nss_status_string(0) == b"ok"
    assert lib.nss_status_string(-4) == b"dead-point store full"


@pytest.mark.parametrize("bad", ["d0", "k_ge_m", "p0", "empty_box", "sigma0", "no_mu", "tol"])
def test_invalid_arguments_rejected_before_device_work(bad):
    from paper_2601_23252_gb300 import native, workloads as W
    wl = W.gauss_d2()
    if bad == "d0":
        import numpy as np
        wl = wl.with_(d=0, a=np.zeros(0), b=np.zeros(0), mu=np.zeros((1, 0)))
    elif bad == "k_ge_m":
        wl = wl.with_(k=wl.n_live)
    elif bad == "p0":
        wl = wl.with_(p=0)
    elif bad == "empty_box":
        wl = wl.with_(b=wl.a.copy())
    elif bad == "sigma0":
        wl = wl.with_(sigma=0.0)
    elif bad == "no_mu":
        wl = wl.with_(mu=None)
    elif bad == "tol":
        wl = wl.with_(tol=2.0)
    with pytest.raises(native.NSSError) as e:
        native.Sampler(wl)
    assert e.value.status == -1


def test_null_arguments(lib):
    lib.nss_step.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.nss_step(None, None) == -1
    lib.nss_run.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.nss_run(None, None) == -1
    lib.nss_destroy.argtypes = [C.c_void_p]
    lib.nss_destroy(None)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: with the CUDA library absent the binding raises
    instead of computing anything."""
    from paper_2601_23252_gb300 import native
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "absent" / "libnss_gb300.so"))
    monkeypatch.setattr(native, "_lib", None, raising=False)
    with pytest.raises(RuntimeError):
        native.lib()


@pytest.mark.parametrize("bad", ["two_runs", "rw_kernel", "lane_cfg", "k_over_1024", "gp"])
def test_plain_path_arguments_rejected_before_device_work(bad):
    """The plain single-run path takes one HRSS run of a Gaussian, mixture,
    flat or logistic likelihood with k <= 1024 in a grouped sweep
    configuration."""
    from paper_2601_23252_gb300 import native, workloads as W
    plain = {"path": native.PATH_PLAIN}
    wls = [W.gauss_d2().with_(extra={"options": dict(plain)})]
    if bad == "two_runs":
        wls = wls * 2
    elif bad == "rw_kernel":
        wls = [wls[0].with_(extra={"options": dict(plain, kernel=1)})]
    elif bad == "lane_cfg":
        wls = [W.gmm_d32().with_(extra={"options": dict(plain, sweep_cfg=24)})]
    elif bad == "k_over_1024":
        wls = [wls[0].with_(n_live=3000, k=1500)]
    elif bad == "gp":
        wls = [W.gp_d3(n=16).with_(n_live=50, k=10, extra={"options": dict(plain)})]
    with pytest.raises(native.NSSError) as e:
        native.Sampler(wls)
    assert e.value.status == -1
