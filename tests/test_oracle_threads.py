"""The oracle's threaded windows (the all-core CPU baseline) against its
serial windows: Jacobi in gather form with integer sums (Algorithm 1's
diffusion operator applied after every tet's draws), so counts, reaction
events, windows and time are the same bits for any thread count."""
import numpy as np
import pytest

import oracle
from oracle import END, OCC
from paper_1610_02258_gb300 import inputs as I


def _pair(w, occ, prec, seed):
    a = oracle.from_workload(w, occ=occ, prec=prec, seed=seed)
    b = oracle.from_workload(w, occ=occ, prec=prec, seed=seed)
    return a, b


@pytest.mark.parametrize("occ,prec", [(OCC, 64), (OCC, 32), (END, 64)])
def test_threads_equal_serial_config1(occ, prec):
    w = I.config1()
    a, b = _pair(w, occ, prec, 7)
    a.run(w.t_end)
    b.run(w.t_end, threads=4)
    assert a.windows == b.windows == 14 and a.time == b.time
    assert a.events == b.events > 0
    assert np.array_equal(a.get_counts(), b.get_counts())


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threads_equal_serial_box_network(threads):
    """The benchmark network on a 6x17x17-cube jittered box (10,404 tets),
    run to an end time off the window grid, then on."""
    w = I.config2(nx=6, t_end=2e-3)
    a, b = _pair(w, OCC, 64, 11)
    for t in (1.37e-3, 2e-3):
        a.run(t)
        b.run(t, threads=threads)
        assert a.windows == b.windows and a.time == b.time
        assert a.events == b.events
        assert np.array_equal(a.get_counts(), b.get_counts())
    assert a.events > 1000


def test_threads_equal_serial_masked_calcium():
    """The calcium network with its influx masked to one end of a 10x3x3-cube
    box, one shortened window by step()."""
    verts, tets = I.kuhn_box_mesh(10, 3, 3, 0.5e-6)
    m = I.calcium_model()
    nt = len(tets)
    counts = np.zeros((m.n_species, nt), np.int32)
    ca = m.names.index("Ca")
    counts[ca, :60] = 20
    for s, name in enumerate(m.names):
        if name.startswith("B"):
            counts[s] = I.place_uniform(3 * nt, nt, seed=50 + s)
    mask = np.zeros(nt, np.uint8)
    mask[:60] = 1
    sims = []
    for threads in (1, 5):
        o = oracle.OracleSim(verts, tets, m, seed=3)
        o.set_counts(counts)
        o.set_reac_mask(m.n_reac - 1, mask)
        o.run(0.3e-3, threads=threads)
        o.step(0.4 * o.tau, threads=threads)
        sims.append(o)
    a, b = sims
    assert a.windows == b.windows and a.events == b.events > 0
    assert np.array_equal(a.get_counts(), b.get_counts())
