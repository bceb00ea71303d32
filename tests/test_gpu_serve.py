"""GPU tests of the served form: continuous batching with admission by a
device-memory budget. Every job's counts and window count must be the same
bits alone (plain steps_run) and in the mix, and the mix must really overlap
jobs on the device and admit late arrivals while others run."""
import numpy as np
import pytest

from paper_1610_02258_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import serve as sv
    return sv


def _jobs(n=16):
    return I.served_jobs(n, rate=400.0, seed=5, t_range=(0.5e-3, 6e-3), size_range=(2_000, 40_000))


@pytest.mark.parametrize("realtime", [False, True])
def test_each_job_same_alone_and_in_the_mix(serve, realtime):
    jobs = _jobs()
    protos = serve.Prototypes()
    alone, _ = serve.run_alone(jobs, protos, realtime=False)
    # budget: the prototypes plus about three average jobs, so admission has to wait
    for j in jobs:
        protos.sim(j.kind, j.size)
    per_job = np.mean([protos.sim(j.kind, j.size).device_bytes for j in jobs])
    srv = serve.Server(hbm_budget=int(protos.device_bytes() + 3 * per_job), max_jobs=6, wave_windows=8)
    srv.protos = protos
    mixed = srv.run(jobs, realtime=realtime)
    for j in jobs:
        a, b = alone[j.job_id], mixed[j.job_id]
        assert a.windows == b.windows
        assert np.array_equal(a.counts, b.counts), j
    assert srv.stats["max_active"] > 1           # jobs overlapped on the device
    assert srv.stats["batch_rebuilds"] > 2       # membership changed while serving
    if not realtime:
        assert srv.stats["admit_waits"] > 0      # the memory budget held jobs back
    s = serve.summarize(mixed, srv.stats["makespan"])
    assert s["jobs"] == len(jobs) and s["p99_s"] >= s["p50_s"] > 0
    protos.close()
