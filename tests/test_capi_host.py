"""CPU checks of the C ABI: the CUDA library builds for sm_103a, loads, exports
every function include/*.h declares, and its host-only calls (mesh and model
construction, which launch nothing) validate their inputs. No compute call
is made here: that needs a GPU."""
import glob
import os
import re

import numpy as np
import pytest

from paper_1610_02258_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import capi as c
    return c


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(steps_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(capi):
    declared = _declared()
    assert len(declared) >= 20
    for name in sorted(declared):
        assert hasattr(capi.lib, name), name
    assert declared == set(capi.EXPORTS)


def test_options_defaults(capi):
    o = capi.steps_options_default()
    assert (o.occupancy, o.reorder, o.block, o.use_graph) == (1, 1, 256, 1)


def test_mesh_validation_matches_oracle_rules(capi):
    verts, tets = I.kuhn_box_mesh(2, 1, 1, 1.0)
    h = capi.steps_mesh_create(verts, tets)
    assert capi.steps_mesh_num_tets(h) == 12
    capi.steps_mesh_destroy(h)
    with pytest.raises(capi.StepsError) as e:
        capi.steps_mesh_create(verts, np.concatenate([tets, tets[:1]]))
    assert e.value.code == -2 and "more than two" in str(e.value)
    bad = tets.copy()
    bad[3] = [0, 1, 2, 2]
    with pytest.raises(capi.StepsError) as e:
        capi.steps_mesh_create(verts, bad)
    assert e.value.code == -2
    bad = tets.copy()
    bad[0, 1] = len(verts)
    with pytest.raises(capi.StepsError) as e:
        capi.steps_mesh_create(verts, bad)
    assert e.value.code == -2
    with pytest.raises(capi.StepsError) as e:
        capi.steps_mesh_create(verts, tets[:0])
    assert e.value.code == -1


def test_model_validation(capi):
    m = I.config1_model()
    h = capi.steps_model_create(m.diff, m.lhs, m.rhs, m.k)
    capi.steps_model_destroy(h)
    # zero reactions is a valid (pure diffusion) model
    h = capi.steps_model_create([1e-12], np.zeros((0, 1)), np.zeros((0, 1)), np.zeros(0))
    capi.steps_model_destroy(h)
    with pytest.raises(capi.StepsError) as e:  # third order
        capi.steps_model_create([1e-12, 0.0], [[2, 1]], [[0, 0]], [1.0])
    assert e.value.code == -3
    with pytest.raises(capi.StepsError) as e:  # negative rate
        capi.steps_model_create([1e-12], [[1]], [[0]], [-1.0])
    assert e.value.code == -3
    with pytest.raises(capi.StepsError) as e:  # negative D
        capi.steps_model_create([-1e-12], [[1]], [[0]], [1.0])
    assert e.value.code == -3
    with pytest.raises(capi.StepsError) as e:  # too many species
        capi.steps_model_create(np.zeros(33), np.zeros((0, 33)), np.zeros((0, 33)), np.zeros(0))
    assert e.value.code == -1


def test_server_host_side_arguments(capi):
    """The job server's options, empty rounds and job lookups are host work."""
    import ctypes
    lib = capi.lib
    o = capi.steps_server_options()
    lib.steps_server_options_default(ctypes.byref(o))
    assert (o.device_budget, o.max_jobs, o.wave_windows, o.block, o.specialize) == (0, 64, 16, 256, -1)
    h = ctypes.c_void_p()
    assert lib.steps_server_create(ctypes.byref(o), None, ctypes.byref(h)) == 0 and h.value
    r, f = ctypes.c_int32(-1), ctypes.c_int32(-1)
    assert lib.steps_server_step(h, ctypes.byref(r), ctypes.byref(f)) == 0 and (r.value, f.value) == (0, 0)
    assert lib.steps_server_job_state(h, 0, None, None, None) == -1
    assert lib.steps_server_take_result(h, 0, None) == -1
    job = ctypes.c_int64()
    assert lib.steps_server_submit(h, None, 1, None, 1e-3, ctypes.byref(job)) == -1
    q = ctypes.c_int32(-1)
    assert lib.steps_server_stats(h, None, None, None, ctypes.byref(q), None, None) == 0 and q.value == 0
    lib.steps_server_destroy(h)
    for field, bad in [("max_jobs", 0), ("wave_windows", 0), ("block", 96), ("specialize", 2), ("device_budget", -1)]:
        b = capi.steps_server_options()
        lib.steps_server_options_default(ctypes.byref(b))
        setattr(b, field, bad)
        h2 = ctypes.c_void_p()
        assert lib.steps_server_create(ctypes.byref(b), None, ctypes.byref(h2)) == -1, field
    assert lib.steps_server_create(None, None, None) == -1


@pytest.mark.parametrize("case", ["cuboid", "box", "dendrite", "shuffled"])
def test_host_tables_equal_the_oracle(capi, case):
    """The library's host set-up (geometry, tau, fixed-point face thresholds;
    no device work) against the oracle's own: tau and every threshold equal
    bit for bit, and the internal tet order is a permutation that does not
    change them. Morton order brings face neighbours closer in memory."""
    import oracle
    if case == "cuboid":
        w = I.config1()
    elif case == "box":
        w = I.config2(nx=5)
    elif case == "dendrite":
        w = I.config3(h=0.45e-6)
    else:  # the cuboid with its tets listed in a random order
        w = I.config1()
        order = np.random.default_rng(2).permutation(w.n_tets)
        w.tets = w.tets[order]
        w.counts = w.counts[:, order]
    mesh = capi.steps_mesh_create(w.verts, w.tets)
    model = capi.steps_model_create(w.model.diff, w.model.lhs, w.model.rhs, w.model.k)
    try:
        tau, thr, perm = capi.steps_debug_host_tables(mesh, model, w.n_tets)
        tau0, thr0, perm0 = capi.steps_debug_host_tables(mesh, model, w.n_tets, reorder=capi.STEPS_REORDER_NONE)
    finally:
        capi.steps_model_destroy(model)
        capi.steps_mesh_destroy(mesh)
    o = oracle.OracleSim(w.verts, w.tets, w.model, seed=1)
    assert tau == tau0 == o.tau
    assert np.array_equal(thr, o.thresholds()) and np.array_equal(thr0, thr)
    assert np.array_equal(np.sort(perm), np.arange(w.n_tets)) and np.array_equal(perm0, np.arange(w.n_tets))
    # cumulative per face, at most 2^31, and empty for boundary faces: a draw
    # can never select a face without a neighbour (the kernel indexes nxt by it)
    nbr, *_ = oracle.geometry(w.verts, w.tets)
    prev = np.concatenate([np.zeros((w.n_tets, 1), np.uint32), thr[:, :3]], axis=1)
    assert np.all(thr >= prev) and int(thr.max()) <= 2**31
    assert np.array_equal(thr[nbr < 0], prev[nbr < 0])
    assert (nbr < 0).any()
    # face neighbours' distance in memory, caller's order vs Morton order
    inv = np.empty_like(perm)
    inv[perm] = np.arange(w.n_tets)
    i, f = np.nonzero(nbr >= 0)
    d_orig = np.abs(nbr[i, f] - i).mean()
    d_morton = np.abs(inv[nbr[i, f]] - inv[i]).mean()
    if case == "shuffled":
        assert d_morton < 0.1 * d_orig
    else:
        assert d_morton < 2.0 * d_orig


@pytest.mark.parametrize("case", ["box", "dendrite", "two_parts"])
def test_rcm_order_is_a_narrow_band_permutation(capi, case):
    """Reverse Cuthill-McKee order: a permutation of the tets, deterministic,
    with the same tau and thresholds as Morton order, and
    face neighbours a few positions apart: the largest distance is the
    band of the breadth-first levels, far below Morton order's on the
    dendrite. two_parts: two disconnected meshes (two components)."""
    import oracle
    if case == "box":
        w = I.config2(nx=5)
        verts, tets = w.verts, w.tets
    elif case == "dendrite":
        w = I.config3(h=0.45e-6)
        verts, tets = w.verts, w.tets
    else:
        w = I.config1()
        verts, tets = I.replicate_mesh(w.verts, w.tets, 2, spacing=5e-6)
    nt = len(tets)
    mesh = capi.steps_mesh_create(verts, tets)
    model = capi.steps_model_create(w.model.diff, w.model.lhs, w.model.rhs, w.model.k)
    try:
        tau_r, thr_r, perm_r = capi.steps_debug_host_tables(mesh, model, nt, reorder=capi.STEPS_REORDER_RCM)
        tau_r2, _, perm_r2 = capi.steps_debug_host_tables(mesh, model, nt, reorder=capi.STEPS_REORDER_RCM)
        tau_m, thr_m, perm_m = capi.steps_debug_host_tables(mesh, model, nt, reorder=capi.STEPS_REORDER_MORTON)
    finally:
        capi.steps_model_destroy(model)
        capi.steps_mesh_destroy(mesh)
    assert np.array_equal(np.sort(perm_r), np.arange(nt)) and np.array_equal(perm_r, perm_r2)
    assert tau_r == tau_r2 == tau_m
    assert np.array_equal(thr_r, thr_m)  # per tet, in the caller's order: the order does not change them
    nbr, *_ = oracle.geometry(verts, tets)
    i, f = np.nonzero(nbr >= 0)

    def band(perm):
        inv = np.empty_like(perm)
        inv[perm] = np.arange(nt)
        return np.abs(inv[nbr[i, f]] - inv[i]).max()

    assert band(perm_r) <= band(perm_m)
    if case == "dendrite":
        assert band(perm_r) * 20 < band(perm_m)
