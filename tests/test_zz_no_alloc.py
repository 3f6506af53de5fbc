"""The allocation-free volume simulation (nss_volume_sim_static): the same
evidence, error and posterior weights as a finished nss_run, from device
buffers the caller passes in, with the library's fixed scratch instead of
device allocation.  It is meant for callers that must not allocate device
memory when they need the result (a framework allocator owns the memory, or
cudaMalloc's device-wide synchronisation is not allowed after start-up).
Collected last on purpose so that a failure here stops a -x run only after
every other test has run; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2601_23252_gb300 import native
from paper_2601_23252_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_volume_simulation_matches_run(gpu_lib):
    torch = pytest.importorskip("torch")
    wl = W.gauss_d2(seed=5)
    with native.Sampler(wl) as s:
        res = s.run()[0]
        d = s.dead(0)
    n = d["logL"].size
    logL = torch.from_numpy(d["logL"]).to("cuda")
    nlive = torch.from_numpy(d["nlive"].astype(np.int32)).to("cuda")
    for call in range(2):  # two calls in a row share the scratch
        lw = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        stats = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        native.volume_sim_static(logL, nlive, 100, wl.seed, wl.run_id, lw, stats)
        torch.cuda.synchronize()
        st = stats.cpu().numpy()
        assert abs(st[0] - res["logZ"]) < 2e-6, (call, st[0], res["logZ"])
        assert abs(st[1] - res["logZ_err"]) < 2e-6, (call, st[1], res["logZ_err"])
        assert np.max(np.abs(lw.cpu().numpy() - d["log_w"])) < 2e-5


def test_static_scratch_rejects_sizes_beyond_the_limit(gpu_lib):
    torch = pytest.importorskip("torch")
    small = torch.zeros(4, dtype=torch.float32, device="cuda")
    ints = torch.ones(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    for n, r in ((524289, 100), (4, 129), (0, 100)):
        with pytest.raises(native.NSSError) as e:
            native.volume_sim_static(small, ints, r, 0, 0, out, stats, n=n)
        assert e.value.status == -1
