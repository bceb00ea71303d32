"""GPU tests of the time-varying influx and of device-side recording: a
piecewise-constant influx rate (steps_set_reac_rate between runs) and counts
recorded every dt_rec by steps_run_record must equal, bit for bit, the
oracle driven through the same rate changes and stopped at the same times."""
import numpy as np
import pytest

import oracle
from paper_1610_02258_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import capi as c
    return c


@pytest.mark.parametrize("flow", [None, True])
def test_influx_schedule_and_recording_match_the_oracle(capi, flow):
    """flow = True: the model-specialised kernel, full windows as flow launches."""
    import torch
    w = I.config3(h=0.5e-6, t_end=1e-3)  # ~30k-tet dendrite, 20 species, masked influx
    influx = w.model.n_reac - 1
    g = capi.from_workload(w, specialize=1 if flow else 0, flow=flow)
    o = oracle.from_workload(w, prec=32)
    tau = g.tau
    assert g.tau == o.tau
    rng = np.random.default_rng(4)
    rec_tets = np.sort(rng.choice(w.n_tets, 300, replace=False)).astype(np.int32)
    ca = w.model.names.index("Ca")
    rec_species = np.array([ca, w.model.names.index("CaB0"), 19], np.int32)
    dt_rec = 2.5 * tau  # off the window grid: every recording cuts a window
    t = 0.0
    # segments: (rate, length in windows, record?) -- long plain segments take the graph path
    schedule = [(5e-3, 40, False), (4e-2, 7, True), (1e-3, 33, False), (2e-2, 9, True), (0.0, 18, True)]
    for rate, nwin, record in schedule:
        g.set_reac_rate(influx, rate)
        o.set_reac_rate(influx, rate)
        t_seg = g.time + nwin * tau
        if not record:
            g.run(t_seg)
            o.run(t_seg)
        else:
            t0 = g.time
            nrec = int(np.floor((t_seg - t0) / dt_rec + 1e-9))
            buf = torch.full((nrec + 1, rec_species.size, rec_tets.size), -7, dtype=torch.int32, device="cuda")
            n = g.run_record(t_seg, dt_rec, rec_species, rec_tets, buf.data_ptr(), nrec + 1)
            assert n == nrec
            got = buf.cpu().numpy()
            assert np.all(got[nrec:] == -7)  # nothing written past the last recording
            for k in range(1, nrec + 1):
                o.run(t0 + k * dt_rec)
                ref = o.get_counts()[np.ix_(rec_species, rec_tets)]
                assert np.array_equal(got[k - 1], ref), (rate, k)
            o.run(t_seg)
        assert g.time == o.time and g.windows == o.windows
        assert np.array_equal(g.get_counts(), o.get_counts()), rate
    assert o.events > 0


def test_record_rejects_bad_arguments(capi):
    import torch
    w = I.config1()
    g = capi.from_workload(w)
    buf = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.StepsError):
        g.run_record(1e-3, 0.0, [0], [0], buf.data_ptr(), 4)          # dt_rec <= 0
    with pytest.raises(capi.StepsError):
        g.run_record(1e-3, 1e-4, [3], [0], buf.data_ptr(), 100)       # species out of range
    with pytest.raises(capi.StepsError):
        g.run_record(1e-3, 1e-4, [0], [w.n_tets], buf.data_ptr(), 100)  # tet out of range
    with pytest.raises(capi.StepsError):
        g.run_record(1e-3, 1e-4, [0], [0], buf.data_ptr(), 4)         # 10 recordings > 4
    assert g.windows == 0
    with pytest.raises(capi.StepsError):
        g.set_reac_rate(5, 1.0)
    with pytest.raises(capi.StepsError):
        g.set_reac_rate(0, -1.0)
