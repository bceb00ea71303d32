"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bar: integer counts are compared element by element. Everything the
diffusion operator does is integer work and must be bit-exact. The reaction
operator takes its decisions in float like the oracle's kernel-precision mode
(prec=32), which evaluates the same IEEE operations in the same order, so whole
runs are bit-exact against it; against the FP64 oracle the reaction phase is
compared in distribution (two-sample KS p > 0.01, means within 3 standard
errors over 10^4 replicates)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import END, OCC
from paper_1610_02258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# the oracle's threaded windows give its serial result bit for bit
THREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import capi as c
    return c


def run_both(capi, verts, tets, model, counts, seed, t_end, occ=OCC, masks=None, prec=32, threads=1, leave=0,
             **kw):
    g = capi.Simulation(verts, tets, model, seed, occupancy=occ, leave_law=leave, **kw)
    g.set_counts(counts)
    o = oracle.OracleSim(verts, tets, model, seed=seed, occ=occ, prec=prec, leave=leave)
    o.set_counts(counts)
    for r, m in (masks or {}).items():
        g.set_reac_mask(r, m)
        o.set_reac_mask(r, m)
    assert g.tau == o.tau
    for t in np.atleast_1d(t_end):
        g.run(t)
        o.run(t, threads=threads)
    assert g.windows == o.windows
    assert g.time == o.time
    return g.get_counts(), o.get_counts(), g, o


# ------------------------------------------------------------------ building blocks

def test_philox_bit_exact(capi):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(1 << 16, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for seed in [0, 3, (1 << 64) - 1, 0x0123456789ABCDEF]:
        assert np.array_equal(capi.steps_debug_philox(seed, ctr), oracle.philox_array(seed, ctr))


def test_philox_equals_curand_device_generator(capi, tmp_path_factory):
    """Both Philox4x32-10 implementations (device, oracle) against cuRAND's
    device Philox4x32-10 (curand_kernel.h) for the same key and counters."""
    import ctypes
    import os
    import shutil
    import subprocess
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cuda", "curand_philox.cu")
    lib = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-o", lib, src], check=True, capture_output=True)
    L = ctypes.CDLL(lib)
    L.curand_philox.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2**32, size=(1 << 14, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [5, 0, 0, 0]
    for seed in [0, 3, (1 << 64) - 1, 0x0123456789ABCDEF]:
        ref = np.empty_like(ctr)
        assert L.curand_philox(seed, ctr.ctypes.data, ctr.shape[0], ref.ctypes.data) == 0
        assert np.array_equal(capi.steps_debug_philox(seed, ctr), ref)
        assert np.array_equal(oracle.philox_array(seed, ctr), ref)


def test_logf_bit_exact_on_every_uniform(capi):
    """The kernel's float log agrees bit for bit with the oracle's on all 2^24
    uniforms (m+1)/2^24 the reaction operator can draw, and on random floats."""
    u = ((np.arange(1 << 24, dtype=np.float64) + 1) / 2**24).astype(np.float32)
    assert np.array_equal(capi.steps_debug_logf(u).view(np.uint32), oracle.logf32_array(u).view(np.uint32))
    x = np.exp(np.random.default_rng(4).uniform(-80, 80, 1 << 16)).astype(np.float32)
    assert np.array_equal(capi.steps_debug_logf(x).view(np.uint32), oracle.logf32_array(x).view(np.uint32))


# ------------------------------------------------------------------ whole runs, bit-exact

@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_pure_diffusion_bit_exact(capi, reorder):
    """Diffusion only (no reactions): integer work end to end, including the
    shortened last window."""
    w = I.config1()
    m = I.model_from_lists(["A", "B"], [1e-11, 2.5e-12], [])
    gc, oc, g, o = run_both(capi, w.verts, w.tets, m, w.counts[:2], 17, w.t_end, reorder=reorder)
    assert g.windows == 14
    assert np.array_equal(gc, oc)
    assert np.array_equal(gc.sum(axis=1), w.counts[:2].sum(axis=1))


@pytest.mark.parametrize("occ", [OCC, END])
def test_config1_reaction_diffusion_bit_exact(capi, occ):
    w = I.config1()
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, w.t_end, occ=occ)
    assert o.events > 0
    assert np.array_equal(gc, oc)


@pytest.mark.parametrize("occ", [OCC, END])
def test_irregular_mesh_bit_exact_many_tiles_ragged_tail(capi, occ):
    """Jittered box of 12x17x17 cubes = 20,808 tets (81 blocks of 256 and a
    ragged tail of 72), 10-species / 20-reaction network, 5 ms (24 full
    windows and a shortened one)."""
    w = I.config2(nx=12, t_end=5e-3)
    assert w.n_tets % 256 != 0
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, w.t_end, occ=occ)
    assert o.events > 1000
    assert np.array_equal(gc, oc)


def test_full_size_config2_whole_run_bit_exact(capi):
    """The benchmark workload at full size (294,780 tets, 20 ms, 99 windows),
    default launch configuration (Morton order, CUDA graph, 256 threads, the
    step kernel compiled for the model)."""
    w = I.config2()
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, w.t_end, threads=THREADS)
    assert g.specialized
    assert g.windows == 99
    assert np.array_equal(gc, oc)


def test_full_size_dense_box_whole_run_bit_exact(capi):
    """The benchmark box at ten times its densities (294,780 tets, ~137
    molecules per tet, 20M reaction events over the run), 20 ms: most
    draws take the bit-plane path, the rest one word per molecule."""
    w = I.config2(density_scale=10.0)
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, w.t_end, threads=THREADS)
    assert g.windows == 99 and o.events > 10_000_000
    assert np.array_equal(gc, oc)


@pytest.mark.parametrize("mode", ["exp", "end"])
def test_full_size_box_other_modes_bit_exact(capi, mode):
    """The benchmark box at full size under the EXP leave law, and in the
    end-count trial mode, ending off the window grid."""
    w = I.config2()
    kw = {"leave": oracle.EXP} if mode == "exp" else {"occ": END}
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, [7.3e-3, w.t_end], threads=THREADS, **kw)
    assert np.array_equal(gc, oc)


@pytest.mark.parametrize("which", ["cuboid", "box", "dendrite"])
def test_specialised_kernel_bit_exact(capi, which):
    """The step kernel compiled at run time for the model (forced on small
    meshes) against the oracle: A + B <-> C; the 10-species / 20-reaction
    network; the calcium network with a masked zero-order influx (the order-0
    and dimer-free forms) and immobile species."""
    if which == "cuboid":
        w, masks = I.config1(), {}
    elif which == "box":
        w = I.config2(nx=6, t_end=3e-3)
        masks = {}
    else:
        w = I.config3(h=0.5e-6, t_end=0.2e-3)
        masks = w.reac_masks
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, w.t_end, masks=masks, specialize=1)
    assert g.specialized
    assert o.events > 0
    assert np.array_equal(gc, oc)


def test_specialised_and_generic_kernels_agree(capi):
    """Same simulation on both kernels, several block sizes: the same bits.
    Includes a dimer (2A -> B) and a rate change between runs."""
    w = I.config2(nx=5, t_end=2e-3)
    names, S = w.model.names, w.model.n_species
    rx = [([names[s] for s in range(S) for _ in range(int(w.model.lhs[r, s]))],
           [names[s] for s in range(S) for _ in range(int(w.model.rhs[r, s]))], float(w.model.k[r]))
          for r in range(12)]
    m = I.model_from_lists(names, w.model.diff, [([names[0], names[0]], [names[1]], 3e7)] + rx)
    ref = None
    for kw in [dict(specialize=-1), dict(specialize=1), dict(specialize=1, block=128), dict(specialize=1, block=512)]:
        g = capi.Simulation(w.verts, w.tets, m, 11, **kw)
        assert g.specialized == (kw["specialize"] == 1)
        g.set_counts(w.counts)
        g.run(w.t_end / 2)
        g.set_reac_rate(0, 1e8)
        g.run(w.t_end)
        c = g.get_counts()
        if ref is None:
            ref = c
        assert np.array_equal(c, ref), kw


def test_full_size_dendrite_bit_exact(capi):
    """The dendrite workload at full size (1,034,502 tets, 20 species, influx
    masked to the soma end: the order-0 kernel variant), 20 windows plus a
    shortened one, in the launch configuration the benchmark times."""
    w = I.config3()
    assert w.n_tets > 1_000_000
    g = capi.from_workload(w)
    t_end = 20.5 * g.tau
    gc, oc, g2, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, t_end, masks=w.reac_masks)
    assert g2.specialized
    assert g2.windows == 21
    assert o.events > 0
    assert np.array_equal(gc, oc)


def test_region_mask_and_zero_order_influx_bit_exact(capi):
    """Reaction masks (influx only in the first 5% of tets) on a small
    dendrite-shaped mesh with the 20-species calcium network."""
    w = I.config3(h=0.5e-6, t_end=0.2e-3)
    assert 20000 < w.n_tets < 80000
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, w.seed, w.t_end, masks=w.reac_masks)
    assert o.events > 0
    assert np.array_equal(gc, oc)


def test_cuboid_equals_stored_oracle_values(capi):
    """The CUDA path on the cuboid (A + B <-> C, 1,920 tets, 10 ms) against the
    oracle's stored kernel-precision result in tests/golden/."""
    import importlib.util
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    golden = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(golden)
    ref = golden.read(os.path.join(here, "golden", "cuboid_prec32.txt"))
    w = I.config1()
    g = capi.from_workload(w)
    g.run(w.t_end)
    assert g.windows == ref["windows"] and g.tau == ref["tau"]
    assert np.array_equal(g.get_counts(), ref["counts"])


def test_resume_on_window_grid_equals_single_run(capi):
    w = I.config2(nx=4, t_end=3e-3)
    a = capi.from_workload(w)
    tau = a.tau
    a.run(7 * tau)
    a.run(w.t_end)
    b = capi.from_workload(w)
    b.run(w.t_end)
    assert np.array_equal(a.get_counts(), b.get_counts())
    assert a.windows == b.windows


def test_launch_shape_order_and_graph_do_not_change_results(capi):
    w = I.config2(nx=6, t_end=4e-3)
    ref = None
    for kw in [dict(), dict(use_graph=False), dict(block=64), dict(block=128), dict(block=512),
               dict(reorder=0), dict(reorder=0, use_graph=False, block=512)]:
        s = capi.from_workload(w, **kw)
        s.run(w.t_end)
        c = s.get_counts()
        if ref is None:
            ref = c
        assert np.array_equal(c, ref), kw


# ------------------------------------------------------------------ edge cases

def test_edge_single_tet_and_empty_counts(capi):
    verts, tets = I.isolated_tets(1)
    m = I.config1_model()
    c = np.array([[3], [4], [0]], np.int32)
    gc, oc, *_ = run_both(capi, verts, tets, m, c, 5, 1e-2)
    assert np.array_equal(gc, oc)
    w = I.config1()
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, np.zeros_like(w.counts), 5, 2e-3)
    assert gc.sum() == 0 and np.array_equal(gc, oc)


def test_edge_immobile_species_and_no_diffusion(capi):
    w = I.config1()
    m = I.model_from_lists(["A", "B", "C"], [0.0, 1e-11, 0.0],
                           [(["A", "B"], ["C"], 1e8), (["C"], ["A", "B"], 10.0)])
    gc, oc, *_ = run_both(capi, w.verts, w.tets, m, w.counts, 6, 3e-3)
    assert np.array_equal(gc, oc)
    m = I.model_from_lists(["A", "B", "C"], [0.0, 0.0, 0.0],
                           [(["A", "B"], ["C"], 1e8), (["C"], ["A", "B"], 10.0)])
    gc, oc, g, o = run_both(capi, w.verts, w.tets, m, w.counts, 6, [1e-3, 3e-3])
    assert math.isinf(g.tau) and g.windows == 2
    assert np.array_equal(gc, oc)


def test_edge_large_counts_and_p_equal_one(capi):
    """10^5 molecules in one tet (a long per-molecule loop) and tets whose
    leave probability is exactly 1 (the fastest tets of a regular grid)."""
    w = I.config1()
    m = I.model_from_lists(["A"], [1e-11], [])
    c = np.zeros((1, w.n_tets), np.int32)
    c[0, 777] = 100000
    gc, oc, *_ = run_both(capi, w.verts, w.tets, m, c, 8, [0.0, 3e-3])
    assert np.array_equal(gc, oc) and gc.sum() == 100000


@pytest.mark.parametrize("spec", [-1, 1])
def test_dense_box_bit_exact(capi, spec):
    """The benchmark network at ten times its densities on a 6x17x17-cube
    box (10,404 tets, ~146 molecules per tet): the denser species of most
    tets hold 16 or more trial molecules and draw by bit planes, the rest by
    one word per molecule, with reactions and occupancy rounding on; generic and
    model-specialised kernels, a run ending off the window grid."""
    w = I.config2(nx=6, density_scale=10.0, t_end=1.7e-3)
    assert w.counts.sum() / w.n_tets > 100
    gc, oc, g, o = run_both(capi, w.verts, w.tets, w.model, w.counts, 19, [0.9e-3, w.t_end], specialize=spec)
    assert g.specialized == (spec == 1)
    assert o.events > 10000
    assert np.array_equal(gc, oc)


def test_bulk_threshold_boundary_bit_exact(capi):
    """Counts of 15, 16, 17, 31, 32, 33 and 64 molecules of one species in
    single tets (both sides of the bit-plane threshold and of a group of 32),
    two species diffusing at different rates, a shortened window."""
    w = I.config1()
    m = I.model_from_lists(["A", "B"], [1e-11, 2.7e-12], [])
    c = np.zeros((2, w.n_tets), np.int32)
    for j, n in enumerate([15, 16, 17, 31, 32, 33, 64]):
        c[0, 100 + 37 * j] = n
        c[1, 90 + 41 * j] = n
    gc, oc, *_ = run_both(capi, w.verts, w.tets, m, c, 4, [1.5e-3, 2.6e-3])
    assert np.array_equal(gc, oc)


def max_size_model(seed: int = 17):
    """32 species and 32 reactions, the most a model may have: order-0 influx
    (one masked to a region), a dimerisation 2X -> Y, reactions that change 6
    species (the most one may), species 31 as a reactant, immobile species,
    and seeded first- and second-order conversions for the rest."""
    rng = np.random.default_rng(seed)
    S = 32
    names = [f"X{i}" for i in range(S)]
    diff = np.exp(rng.uniform(np.log(1e-13), np.log(1e-11), S))
    diff[[7, 19, 28]] = 0.0
    rx = [([], ["X0"], 2e-4), ([], ["X1"], 5e-5), (["X2", "X2"], ["X3"], 3e6),
          (["X4", "X5"], ["X6", "X7", "X8", "X9"], 2e6), (["X31"], ["X30", "X29", "X28", "X27", "X26"], 40.0)]
    while len(rx) < 32:
        if len(rx) % 2:
            x, y = rng.choice(S, 2, replace=False)
            rx.append(([names[x]], [names[y]], float(np.exp(rng.uniform(np.log(1.0), np.log(300.0))))))
        else:
            x, y, z = rng.choice(S, 3, replace=False)
            rx.append(([names[x], names[y]], [names[z]], float(np.exp(rng.uniform(np.log(1e5), np.log(1e7))))))
    return I.model_from_lists(names, list(diff), rx)


@pytest.mark.parametrize("specialize,block", [(-1, 256), (-1, 512), (1, 256), (1, 128), (1, 512)])
def test_edge_maximum_model_size_bit_exact(capi, specialize, block):
    """S = 32, R = 32 on an irregular mesh of 5,202 tets (tiles of 128-512
    with a ragged tail), generic and specialised kernels, against the oracle."""
    w = I.config2(nx=3, t_end=1.5e-3)
    m = max_size_model()
    rng = np.random.default_rng(5)
    c = rng.poisson(3.0, size=(32, w.n_tets)).astype(np.int32)
    mask = np.zeros(w.n_tets, np.uint8)
    mask[: w.n_tets // 7] = 1
    gc, oc, g, o = run_both(capi, w.verts, w.tets, m, c, 9, [0.4e-3, w.t_end], masks={0: mask},
                            specialize=specialize, block=block)
    assert g.specialized == (specialize == 1)
    assert o.events > 0 and g.windows >= 3
    assert np.array_equal(gc, oc)


def test_sparse_rows_follow_molecules_across_tiles(capi):
    """Molecules start in a few tets of a 10,404-tet mesh (41 tiles of 256,
    most tiles empty at first) and spread over tiles: A diffuses fast,
    converts to a slower B and to an immobile C. New molecules are added
    between runs (counts reset on the device) and each run is compared with
    the oracle."""
    w = I.config2(nx=6, t_end=6e-3)
    m = I.model_from_lists(["A", "B", "C"], [1e-11, 2e-12, 0.0],
                           [(["A"], ["B"], 300.0), (["B"], ["C"], 100.0)])
    c = np.zeros((3, w.n_tets), np.int32)
    c[0, w.n_tets - 1] = 5000
    c[0, np.random.default_rng(8).choice(w.n_tets, 6, replace=False)] = 800
    for spec in (-1, 1):
        g = capi.Simulation(w.verts, w.tets, m, 13, specialize=spec)
        o = oracle.OracleSim(w.verts, w.tets, m, seed=13, prec=32)
        for obj in (g, o):
            obj.set_counts(c)
        t = 0.0
        for k, dt in enumerate([1.7e-3, 2.0e-3, 2.3e-3]):
            t += dt
            g.run(t)
            o.run(t)
            gc, oc = g.get_counts(), o.get_counts()
            assert np.array_equal(gc, oc), (spec, k)
            # a fresh species-A pulse in the first tet, on top of the state
            nc = gc.copy()
            nc[0, 0] += 3000
            g.set_counts(nc)
            o.set_counts(nc)
        assert (g.get_counts()[2] > 0).sum() > 150


def test_edge_noop_and_bad_arguments(capi):
    w = I.config1()
    s = capi.from_workload(w)
    s.run(0.0)
    assert s.windows == 0
    s.run(-1.0)
    assert s.windows == 0
    bad = w.counts.copy()
    bad[0, 0] = -1
    with pytest.raises(capi.StepsError) as e:
        s.set_counts(bad)
    assert e.value.code == -1
    with pytest.raises(capi.StepsError):
        s.run(float("nan"))


# ------------------------------------------------------------------ statistics vs the FP64 oracle

def test_reaction_phase_matches_fp64_oracle_in_distribution(capi):
    """10^4 well-mixed replicates (isolated tets) of A + B <-> C: the float
    kernel against the FP64 oracle with a different seed, two-sample KS
    p > 0.01 and means within 3 standard errors; both against the exact CME."""
    n, N0, kf, kb, t = 10000, 30, 1e8, 50.0, 4e-3
    verts, tets = I.isolated_tets(n)
    m = I.model_from_lists(["A", "B", "C"], [0.0, 0.0, 0.0],
                           [(["A", "B"], ["C"], kf), (["C"], ["A", "B"], kb)])
    c = np.zeros((3, n), np.int32)
    c[0] = N0
    c[1] = N0 + 5
    g = capi.Simulation(verts, tets, m, 101)
    g.set_counts(c)
    g.run(t)
    gx = g.get_counts()[2]
    o = oracle.OracleSim(verts, tets, m, seed=202, prec=64)
    o.set_counts(c)
    o.run(t)
    ox = o.get_counts()[2]
    assert stats.ks_2samp(gx, ox).pvalue > 0.01
    se = math.sqrt(gx.var() / n + ox.var() / n)
    assert abs(gx.mean() - ox.mean()) < 3 * se


def test_conservation_full_config2(capi):
    w = I.config2()
    s = capi.from_workload(w)
    s.run(w.t_end)
    c = s.get_counts()
    assert c.min() >= 0
    # each reaction of the random network conserves nothing in general, but
    # without reactions every species total is conserved
    m = I.model_from_lists(w.model.names, w.model.diff, [])
    s2 = capi.Simulation(w.verts, w.tets, m, 1)
    s2.set_counts(w.counts)
    s2.run(w.t_end)
    assert np.array_equal(s2.get_counts().sum(axis=1), w.counts.sum(axis=1))
