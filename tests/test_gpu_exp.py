"""GPU parity of the EXP leave law (p = 1 - exp(-tau d) for the diffusion
operator's binomial; STEPS_LEAVE_EXP) against the oracle's EXP mode, bit for
bit, on the model-specialised kernels it runs on: plain runs ending on and
off the window grid (the shortened window's table is built on the host
before its launch), the many-species kernel with trial counts in global
memory, a batch of members against each alone, a clone, and the calls that
must refuse it."""
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


def _both(capi, w, seed, ends, **kw):
    g = capi.Simulation(w.verts, w.tets, w.model, seed, leave_law=capi.STEPS_LEAVE_EXP, **kw)
    o = oracle.OracleSim(w.verts, w.tets, w.model, seed=seed, prec=32, leave=oracle.EXP)
    for obj in (g, o):
        obj.set_counts(w.counts)
        for r, m in w.reac_masks.items():
            obj.set_reac_mask(r, m)
    assert g.tau == o.tau and g.specialized
    for t in ends:
        g.run(t)
        o.run(t)
        assert g.windows == o.windows and g.time == o.time
        assert np.array_equal(g.get_counts(), o.get_counts())
    return g, o


@pytest.mark.parametrize("reorder", [0, 1])
def test_exp_cuboid_bit_exact(capi, reorder):
    w = I.config1()
    g, o = _both(capi, w, 5, [2.3e-3, w.t_end], reorder=reorder)
    assert o.events > 0


def test_exp_box_and_dendrite_bit_exact(capi):
    w = I.config2(nx=4, t_end=3e-3)
    _both(capi, w, 7, [1.1e-3, w.t_end])
    d = I.config3(h=0.5e-6, t_end=0.12e-3)
    g, o = _both(capi, d, 8, [0.05e-3, d.t_end])
    # EULER and EXP differ on the same seed
    e = capi.from_workload(d, seed=8)
    e.run(d.t_end)
    assert not np.array_equal(e.get_counts(), g.get_counts())


def test_exp_batch_and_clone_equal_alone(capi):
    ws = [I.config3(seed=300 + j, h=0.55e-6, t_end=0.1e-3 + 0.03e-3 * j) for j in range(3)]
    alone = []
    for w in ws:
        s = capi.from_workload(w, leave_law=capi.STEPS_LEAVE_EXP)
        s.run(w.t_end)
        alone.append(s.get_counts())
    members = [capi.from_workload(w, leave_law=capi.STEPS_LEAVE_EXP) for w in ws]
    b = capi.Batch(members, block=256)
    assert b.specialized
    b.run([w.t_end for w in ws])
    for ref, m in zip(alone, members):
        assert np.array_equal(m.get_counts(), ref)
    c = members[0].clone(300)
    c.set_counts(ws[0].counts)
    for r, m in ws[0].reac_masks.items():
        c.set_reac_mask(r, m)
    c.run(ws[0].t_end)
    assert np.array_equal(c.get_counts(), alone[0])


def test_exp_refusals(capi):
    import torch
    w = I.config1()
    with pytest.raises(capi.StepsError) as e:
        capi.Simulation(w.verts, w.tets, w.model, 1, specialize=-1, leave_law=capi.STEPS_LEAVE_EXP)
    assert e.value.code == -1
    s = capi.from_workload(w, leave_law=capi.STEPS_LEAVE_EXP)
    d = torch.from_numpy(np.ascontiguousarray(w.counts)).to("cuda")
    with pytest.raises(capi.StepsError) as e:
        capi.steps_run_noalloc(s._sim, d.data_ptr(), 1e-3)
    assert e.value.code == -1 and s.windows == 0
    g = capi.from_workload(w)
    with pytest.raises(capi.StepsError):
        capi.Batch([s, g], block=256)  # one EXP member and one EULER: two model structures
