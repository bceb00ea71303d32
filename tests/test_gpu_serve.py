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


@pytest.mark.parametrize("realtime,specialize", [(False, 1), (True, 1), (False, -1)])
def test_each_job_same_alone_and_in_the_mix(serve, realtime, specialize):
    """specialize = 1: jobs grouped by model structure, each group on the
    kernel compiled for its model, groups on streams of their own; -1: one
    batch of every job on the generic kernel."""
    jobs = _jobs()
    protos = serve.Prototypes(specialize=1 if specialize >= 0 else 0)
    alone, _ = serve.run_alone(jobs, protos, realtime=False)
    # budget: the prototypes plus about three average jobs, so admission has to wait
    for j in jobs:
        protos.sim(j.kind, j.size)
    per_job = np.mean([protos.sim(j.kind, j.size).device_bytes for j in jobs])
    srv = serve.Server(hbm_budget=int(protos.device_bytes() + 3 * per_job), max_jobs=6, wave_windows=8,
                       specialize=specialize)
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


def test_native_server_jobs_equal_alone_and_budget_admission(serve):
    """steps_server_* directly: jobs on three prototypes (1,920-tet cuboid,
    box, small dendrite) with end times on and off the window grid and one of
    0; each result equals the same simulation run alone with steps_run. A
    budget below two jobs admits one job at a time; a result is taken once."""
    from paper_1610_02258_gb300 import capi
    ws = [I.config1(seed=3), I.config2(seed=9, nx=3, t_end=2e-3), I.config3(h=0.5e-6, t_end=0.1e-3)]
    protos = [capi.from_workload(w) for w in ws]
    specs = [(0, 11, 3.3e-3), (1, 12, 2.0e-3), (2, 13, 0.1e-3), (1, 14, 0.0), (0, 15, 1.48e-3), (2, 16, 0.071e-3)]
    for budget, limit, spec in [(0, 6, -1), (1, 1, -1), (0, 6, 0), (0, 6, 1)]:
        srv = capi.NativeServer(device_budget=budget, max_jobs=4, wave_windows=5, specialize=spec)
        ids = [srv.submit(protos[k], seed, ws[k].counts, t) for k, seed, t in specs]
        assert ids == list(range(len(specs)))
        assert all(srv.state(i)[0] == 0 for i in ids)
        most = 0
        for _ in range(10000):
            running, _ = srv.step()
            most = max(most, running)
            if all(srv.state(i)[0] == 2 for i in ids):
                break
        assert most <= min(limit, 4)
        for i, (k, seed, t) in zip(ids, specs):
            state, windows, tt = srv.state(i)
            assert state == 2 and abs(tt - t) <= 1e-9 * t
            got = srv.take_result(i)
            ref = protos[k].clone(seed)
            ref.set_counts(ws[k].counts)
            ref.run(t)
            assert windows == ref.windows
            assert np.array_equal(got, ref.get_counts()), (budget, spec, i)
            assert srv.state(i)[0] == 3
            with pytest.raises(capi.StepsError):
                capi._check(capi.lib.steps_server_take_result(srv._h, i, None))
        st = srv.stats()
        assert st["running"] == 0 and st["queued"] == 0 and st["device_bytes"] == 0
        srv.close()


def test_native_server_separates_leave_laws(serve):
    """Prototypes of one model under the EULER and the EXP leave law are two
    model structures for the server: their jobs run in two groups, each on
    its own specialised kernel, and every job equals its run alone."""
    from paper_1610_02258_gb300 import capi
    w = I.config2(seed=9, nx=3, t_end=2e-3)
    protos = [capi.from_workload(w, specialize=1), capi.from_workload(w, leave_law=capi.STEPS_LEAVE_EXP)]
    specs = [(0, 21, 1.3e-3), (1, 22, 1.3e-3), (1, 23, 2.0e-3), (0, 24, 0.7e-3)]
    srv = capi.NativeServer(max_jobs=4, wave_windows=3, specialize=1)
    ids = [srv.submit(protos[k], seed, w.counts, t) for k, seed, t in specs]
    for _ in range(1000):
        srv.step()
        if all(srv.state(i)[0] == 2 for i in ids):
            break
    for i, (k, seed, t) in zip(ids, specs):
        got = srv.take_result(i)
        ref = protos[k].clone(seed)
        ref.set_counts(w.counts)
        ref.run(t)
        assert np.array_equal(got, ref.get_counts()), (k, seed)
    srv.close()
