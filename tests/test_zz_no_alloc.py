"""GPU test of steps_run_noalloc, the entry point for callers that cannot let
the library allocate device memory (applications that own all device memory
through their own pool or a fixed budget, or that must not allocate once
running). It must give exactly the counts of the ordinary path
(steps_run + steps_get_counts_all) on the same simulation, call after call:
its scratch is a fixed device array that keeps the previous call's contents,
so the second call checks that each call clears what must start at zero.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("specialize", [-1, 1])
def test_noalloc_equals_steps_run_on_two_calls_in_a_row(capi, specialize):
    """On the generic step kernel and on the one compiled for the model."""
    import torch
    w = I.config2(nx=8, t_end=4e-3)  # 13,872 tets, 10 species, 20 reactions
    ref = capi.from_workload(w, specialize=specialize)
    new = capi.from_workload(w, specialize=specialize)  # same seed, tables and clock; its own buffers stay unused
    assert new.specialized == (specialize == 1)
    d_counts = torch.from_numpy(np.ascontiguousarray(w.counts)).to("cuda")
    tau = ref.tau
    # first call ends off the window grid (a shortened window), the second on it
    for t_end in (7.5 * tau, 7.5 * tau + 9 * tau):
        ref.run(t_end)
        expect = ref.get_counts()
        capi.steps_run_noalloc(new._sim, d_counts.data_ptr(), t_end)
        got = d_counts.cpu().numpy()
        assert new.windows == ref.windows and new.time == ref.time
        assert np.array_equal(got, expect)  # integer counts: bit-exact, as every parity test here
    assert int(expect.sum()) > 0
    # the simulation's own count buffers were neither read nor written
    assert np.array_equal(new.get_counts(), w.counts)


def test_noalloc_rejects_negative_counts_before_anything_changes(capi):
    """A negative input count is an argument error: the clock and the
    caller's buffer stay as they were, and a corrected buffer then runs."""
    import torch
    w = I.config2(nx=4, t_end=2e-3)
    sim = capi.from_workload(w)
    ref = capi.from_workload(w)
    bad = np.ascontiguousarray(w.counts).copy()
    bad[3, 17] = -1
    d = torch.from_numpy(bad).to("cuda")
    t_end = 3.5 * sim.tau
    with pytest.raises(capi.StepsError) as e:
        capi.steps_run_noalloc(sim._sim, d.data_ptr(), t_end)
    assert e.value.code == -1 and "negative" in str(e.value)
    assert sim.windows == 0 and sim.time == 0.0
    assert np.array_equal(d.cpu().numpy(), bad)
    d.copy_(torch.from_numpy(np.ascontiguousarray(w.counts)))
    capi.steps_run_noalloc(sim._sim, d.data_ptr(), t_end)
    ref.run(t_end)
    assert sim.windows == ref.windows == 4
    assert np.array_equal(d.cpu().numpy(), ref.get_counts())


def test_noalloc_rejects_problems_beyond_its_scratch(capi):
    import torch
    verts, tets = I.kuhn_box_mesh(76, 17, 17, 0.5e-6)  # 131,784 tets x 32 species > 4,194,304
    m = I.model_from_lists([f"S{i}" for i in range(32)], np.full(32, 1e-12), [])
    sim = capi.Simulation(verts, tets, m, 1)
    d = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.StepsError) as e:
        capi.steps_run_noalloc(sim._sim, d.data_ptr(), 1e-3)
    assert e.value.code == -1 and "exceeds the fixed scratch" in str(e.value)
    assert sim.windows == 0 and sim.time == 0.0
