"""GPU tests of the batched form: one launch per window over many
simulations must give, for every member, exactly the counts, window count
and clock of that member run alone with steps_run."""
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


def _workloads():
    ws = []
    for j, nx in enumerate([3, 7, 1, 12, 5]):
        ws.append(I.config2(seed=100 + j, nx=nx, t_end=3e-3 + 0.37e-3 * j))
    ws.append(I.config1(seed=7))                                # another model (3 species, 2 reactions)
    ws.append(I.config3(h=0.5e-6, t_end=0.15e-3))               # 20 species, masked influx
    return ws


@pytest.mark.parametrize("block,use_graph", [(0, True), (128, False), (512, True)])
def test_batch_equals_members_alone(capi, block, use_graph):
    ws = _workloads()
    alone = []
    for w in ws:
        s = capi.from_workload(w)
        s.run(w.t_end)
        alone.append((s.get_counts(), s.windows, s.time))
    members = [capi.from_workload(w) for w in ws]
    b = capi.Batch(members, block=block, use_graph=use_graph)
    b.run([w.t_end for w in ws])
    for (ref, win, t), m in zip(alone, members):
        assert m.windows == win and m.time == t
        assert np.array_equal(m.get_counts(), ref)
    blk, launches, tune = b.info
    assert launches > 0
    if block == 0:
        assert blk in (128, 256, 512) and all(x > 0 for x in tune)
    else:
        assert blk == block


def test_batch_resume_and_mixed_end_times(capi):
    """Two batch runs in a row (second one ending off the window grid for some
    members, on it for others) equal one run per member alone."""
    ws = _workloads()[:4]
    members = [capi.from_workload(w) for w in ws]
    b = capi.Batch(members, block=256)
    tau = [m.tau for m in members]
    t1 = [5 * t for t in tau]
    t2 = [w.t_end for w in ws]
    b.run(t1)
    b.run(t2)
    for w, m, t1j in zip(ws, members, t1):
        s = capi.from_workload(w)
        s.run(t1j)
        s.run(w.t_end)
        assert m.windows == s.windows
        assert np.array_equal(m.get_counts(), s.get_counts())


def test_plain_batched_plain_handoff(capi):
    """A member that runs alone, then in a batch of block size 128 for an odd
    number of windows (its count buffers swap), then alone again equals the
    same member run alone throughout."""
    ws = [I.config3(h=0.5e-6, t_end=0.2e-3), I.config2(seed=41, nx=4, t_end=3e-3)]
    for spec in (-1, 1):
        for w in ws:
            s = capi.from_workload(w, specialize=spec)
            tau = s.tau
            s.run(4 * tau)
            b = capi.Batch([s], block=128)
            b.run([9 * tau])
            b.close()
            s.run(w.t_end)
            ref = capi.from_workload(w, specialize=spec)
            ref.run(4 * tau)
            ref.run(9 * tau)
            ref.run(w.t_end)
            assert s.windows == ref.windows
            assert np.array_equal(s.get_counts(), ref.get_counts()), (w.name, spec)


@pytest.mark.parametrize("block", [128, 512])
def test_specialised_batch_equals_members_alone(capi, block):
    """Members sharing one model structure (the box network, different sizes,
    seeds and end times): the batched kernel compiled for the model gives every
    member's counts bit for bit as it runs alone; so does the generic one."""
    ws = [I.config2(seed=200 + j, nx=nx, t_end=2e-3 + 0.41e-3 * j) for j, nx in enumerate([2, 9, 4, 1, 6])]
    alone = []
    for w in ws:
        s = capi.from_workload(w, specialize=-1)
        s.run(w.t_end)
        alone.append(s.get_counts())
    for spec in (1, -1):
        members = [capi.from_workload(w) for w in ws]
        b = capi.Batch(members, block=block, specialize=spec)
        b.run([w.t_end for w in ws])
        assert b.specialized == (spec == 1)
        for ref, m in zip(alone, members):
            assert np.array_equal(m.get_counts(), ref), spec


def test_specialised_batch_needs_one_model_structure(capi):
    ws = _workloads()[:2] + [I.config1(seed=3)]
    members = [capi.from_workload(w) for w in ws]
    with pytest.raises(capi.StepsError) as e:
        capi.Batch(members, block=256, specialize=1)
    assert e.value.code == -1
    assert not capi.Batch(members, block=256).specialized  # auto: generic for mixed models


def test_specialised_batch_of_many_species_models(capi):
    """Dendrite replicates (20 species, masked influx): the specialised batched
    kernel keeps trial counts in global memory; members created without a
    specialised kernel of their own get the buffer from the batch. Every
    member equals its run alone."""
    ws = [I.config3(seed=300 + j, h=0.55e-6, t_end=0.1e-3 + 0.03e-3 * j) for j in range(3)]
    alone = []
    for w in ws:
        s = capi.from_workload(w, specialize=-1)
        s.run(w.t_end)
        alone.append(s.get_counts())
    members = [capi.from_workload(w, specialize=-1) for w in ws]
    assert not any(m.specialized for m in members)
    b = capi.Batch(members, block=256, specialize=1)
    assert b.specialized
    b.run([w.t_end for w in ws])
    for ref, m in zip(alone, members):
        assert np.array_equal(m.get_counts(), ref)


def test_full_size_batched_configuration_sampled_against_oracle(capi):
    """The batched benchmark configuration at full size: 256 box replicates
    of 10k-300k tets (20.1M tets), block size autotuned on the first run, the
    model-specialised batched kernel. After 3 ms (about 15 windows each, 12 of
    them inside the autotuner) four members (the smallest, the largest and two
    seeded picks) equal the oracle run on that member alone."""
    import oracle
    sizes = I.batch_sizes(n=256)
    ws = [I.box_for_tets(int(sz), seed=1000 + j) for j, sz in enumerate(sizes)]
    sims = [capi.from_workload(w) for w in ws]
    assert sum(s.nt for s in sims) > 20_000_000
    b = capi.Batch(sims, block=0)
    t_end = 3e-3
    b.run([t_end] * len(sims))
    assert b.specialized
    assert b.info[0] in (128, 256, 512) and max(b.info[2]) > 0  # the autotuner ran
    nts = np.array([s.nt for s in sims])
    picks = {int(nts.argmin()), int(nts.argmax())} | set(np.random.default_rng(4).choice(256, 2, replace=False).tolist())
    for j in sorted(picks):
        w = ws[j]
        o = oracle.OracleSim(w.verts, w.tets, w.model, seed=w.seed, prec=32)
        o.set_counts(w.counts)
        o.run(t_end)
        assert sims[j].windows == o.windows
        assert np.array_equal(sims[j].get_counts(), o.get_counts()), j
    b.close()


def test_batch_tables_survive_a_busy_stream(capi):
    """Rounds in which every member ends off its window grid (a shortened
    window after its full ones), each run queued behind ~0.3 ms of other
    work on the batch's stream, so the uploads of the window tables run long
    after the host has filled them in: the full-window table must not change
    under its queued upload. Every member equals its runs alone."""
    import torch
    ws = [I.config1(seed=20 + j) for j in range(6)] + [I.config2(seed=30 + j, nx=2, t_end=1e-3) for j in range(3)]
    members = [capi.from_workload(w) for w in ws]
    alone = [capi.from_workload(w) for w in ws]
    busy = torch.cuda.Stream()
    b = capi.Batch(members, block=256, use_graph=False, cuda_stream=busy.cuda_stream)
    big = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    for r in range(4):
        targets = [m.time + (1 + (j + r) % 3 + 0.5) * m.tau for j, m in enumerate(members)]
        with torch.cuda.stream(busy):
            big.zero_()
            big.add_(1)
        b.run(targets)
        for s, t in zip(alone, targets):
            s.run(t)
        for j, (m, s) in enumerate(zip(members, alone)):
            assert m.windows == s.windows and m.time == s.time, (r, j)
            assert np.array_equal(m.get_counts(), s.get_counts()), (r, j)


def test_batch_flow_groups_equal_window_launches(capi):
    """The batched flow form: members of one model structure with different
    mesh spacings (so different windows and window counts: members that end
    earlier skip their later items), about 1.3M tets in all (more than one
    L2-sized group), over a run that ends off every member's window grid and
    a second one. Every member equals the same batch in window launches and,
    for a sample, the member run alone."""
    hs = [10 / 17, 10 / 15, 10 / 19, 10 / 17, 10 / 13, 10 / 21, 10 / 17, 10 / 16]
    ws = [I.config2(seed=300 + j, nx=[200, 30, 130, 110, 17, 80, 6, 70][j], h=h * I.UM, t_end=2.1e-3)
          for j, h in enumerate(hs)]
    out = {}
    for flow in (True, False):
        members = [capi.from_workload(w) for w in ws]
        b = capi.Batch(members, block=256, specialize=1, flow=flow)
        b.run([1.7e-3 + 0.05e-3 * j for j in range(len(ws))])
        b.run([w.t_end for w in ws])
        assert b.specialized
        out[flow] = [(m.get_counts(), m.windows, m.time) for m in members]
        b.close()
    assert sum(len(w.tets) for w in ws) > 1_000_000
    assert len({o[1] for o in out[True]}) > 1  # members take different numbers of windows
    for (a, wa, ta), (c, wc, tc) in zip(out[True], out[False]):
        assert wa == wc and ta == tc and np.array_equal(a, c)
    for j in (1, 4, 6):
        s = capi.from_workload(ws[j])
        s.run(1.7e-3 + 0.05e-3 * j)
        s.run(ws[j].t_end)
        assert np.array_equal(s.get_counts(), out[True][j][0])
