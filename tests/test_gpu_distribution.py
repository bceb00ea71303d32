"""The float CUDA path against the FP64 oracle in distribution, on the two
reaction networks the benchmarks run, with diffusion and the occupancy trial
rule on (Algorithm 1; §2.2).

Each test runs 10^4 independent copies of one small jittered mesh from one
initial state: the CUDA path under one seed, the oracle (every reaction
decision in double, libm log) under another. Per species, the copy totals
are compared by a two-sample KS test and by their means; so are a few per-tet
marginals. The family of m comparisons per network is held at a 1 %
familywise level (Bonferroni): each KS p-value must exceed 0.01/m and each
mean difference must lie within z(1 - 0.005/m) standard errors (3.3 SE for
m = 11). Sensitivity checks rerun the oracle with one rate constant changed
(5 % on the fastest first-order reaction, or on the calcium pump; a factor 2,
the size of a pair-counting convention mistake, on the fastest second-order
one) and show that the same comparison rejects it, so the test sees changes
of that size.
"""
import copy
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import OCC
from paper_1610_02258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COPIES = 10_000


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_02258_gb300.build import build
    build()
    from paper_1610_02258_gb300 import capi as c
    return c


def _replicated(base_v, base_t, h, one_copy_counts, masks_one=None):
    nt0 = len(base_t)
    verts, tets = I.replicate_mesh(base_v, base_t, COPIES, spacing=(base_v[:, 0].max() - base_v[:, 0].min()) + 4 * h)
    counts = np.tile(one_copy_counts, (1, COPIES)).astype(np.int32)
    masks = {r: np.tile(m, COPIES).astype(np.uint8) for r, m in (masks_one or {}).items()}
    return verts, tets, counts, masks, nt0


def _run_gpu(capi, verts, tets, model, counts, masks, seed, t_end):
    g = capi.Simulation(verts, tets, model, seed)
    g.set_counts(counts)
    for r, m in masks.items():
        g.set_reac_mask(r, m)
    g.run(t_end)
    return g.get_counts(), g.windows


def _run_oracle(verts, tets, model, counts, masks, seed, t_end):
    o = oracle.OracleSim(verts, tets, model, seed=seed, occ=OCC, prec=64)
    o.set_counts(counts)
    for r, m in masks.items():
        o.set_reac_mask(r, m)
    o.run(t_end, threads=max(1, min(32, os.cpu_count() or 1)))  # the serial result, bit for bit
    return o.get_counts(), o.windows


def _compare(a, b, m):
    """(KS p-value, |mean difference| in standard errors) of two samples;
    None when both are the same constant."""
    if a.var() == 0 and b.var() == 0:
        assert a[0] == b[0]
        return None
    p = stats.ks_2samp(a, b).pvalue
    se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    return p, abs(a.mean() - b.mean()) / se


def _family(gpu, orc, nt0, marginals):
    """Per-species copy totals plus the chosen (species, tet) marginals of
    [S, COPIES * nt0] count arrays."""
    S = gpu.shape[0]
    g = gpu.reshape(S, COPIES, nt0)
    o = orc.reshape(S, COPIES, nt0)
    fam = {f"total[{s}]": (g[s].sum(axis=1), o[s].sum(axis=1)) for s in range(S)}
    for s, t in marginals:
        fam[f"tet[{s},{t}]"] = (g[s, :, t], o[s, :, t])
    return fam


def _check_family(fam, label):
    res = {k: _compare(a, b, None) for k, (a, b) in fam.items()}
    res = {k: v for k, v in res.items() if v is not None}
    m = len(res)
    assert m >= 5, f"{label}: too few non-constant comparisons ({m})"
    alpha = 0.01 / m
    z = stats.norm.isf(alpha / 2)
    worst_p = min(p for p, _ in res.values())
    worst_z = max(zz for _, zz in res.values())
    print(f"{label}: {m} comparisons, smallest KS p {worst_p:.3g} (bar {alpha:.2g}), "
          f"largest mean gap {worst_z:.2f} SE (bar {z:.2f})")
    for k, (p, zz) in res.items():
        assert p > alpha, (label, k, p)
        assert zz < z, (label, k, zz)
    return res


def _sensitivity(gpu, verts, tets, model, counts, masks, seed, t_end, nt0, r, factor):
    """Smallest KS p-value of the copy totals against the oracle run with
    rate constant r multiplied by `factor` (a different law)."""
    m2 = copy.deepcopy(model)
    m2.k = model.k.copy()
    m2.k[r] *= factor
    alt, _ = _run_oracle(verts, tets, m2, counts, masks, seed, t_end)
    ps = [_compare(a, b, None) for a, b in _family(gpu, alt, nt0, []).values()]
    return min(p for p, _ in [x for x in ps if x is not None])


def _fastest(model, order):
    """Index of the reaction of the given order with the largest rate constant."""
    orders = model.lhs.sum(axis=1)
    idx = np.nonzero(orders == order)[0]
    return int(idx[np.argmax(model.k[idx])])


def test_config2_network_in_distribution(capi):
    """The benchmark's 10-species, 20-reaction random network on 10^4 copies
    of a jittered 2x2x2-cube mesh (48 tets, h = 10/17 um, the benchmark box's
    spacing and densities), 6.5 ms (nine full windows and a shortened one)."""
    h = 10.0 / 17.0 * I.UM
    bv, bt = I.kuhn_box_mesh(2, 2, 2, h)
    bv = I.jitter_box_vertices(bv, h, 0.2, seed=31)
    model = I.random_network(5)
    rng = np.random.default_rng(2)
    vol_um3 = 8 * (h / I.UM) ** 3
    dens = rng.uniform(1.0, 100.0, size=model.n_species)
    one = np.stack([I.place_uniform(int(round(d * vol_um3)), len(bt), seed=300 + s) for s, d in enumerate(dens)])
    verts, tets, counts, masks, nt0 = _replicated(bv, bt, h, one)
    t_end = 6.5e-3
    gpu, gw = _run_gpu(capi, verts, tets, model, counts, masks, 1001, t_end)
    orc, ow = _run_oracle(verts, tets, model, counts, masks, 2002, t_end)
    assert gw == ow == 10
    fam = _family(gpu, orc, nt0, [(int(np.argmax(dens)), 0)])
    _check_family(fam, "config-2 network")
    for order, factor in ((1, 1.05), (2, 2.0)):
        r = _fastest(model, order)
        p_alt = _sensitivity(gpu, verts, tets, model, counts, masks, 2002, t_end, nt0, r, factor)
        print(f"config-2 network, oracle with k[{r}] x {factor}: smallest KS p {p_alt:.3g}")
        assert p_alt < 1e-6


def test_calcium_network_in_distribution(capi):
    """The dendrite benchmark's 20-species calcium network (four two-site
    buffers, pump, influx masked to one end) on 10^4 copies of a jittered
    3x2x2-cube mesh of 0.5 um cubes (72 tets). Calcium starts in the masked
    end cube, buffers and tracers everywhere; 0.6 ms (about 16 windows of
    the fast calcium diffusion)."""
    h = 0.5 * I.UM
    bv, bt = I.kuhn_box_mesh(3, 2, 2, h)
    bv = I.jitter_box_vertices(bv, h, 0.2, seed=32)
    model = I.calcium_model()
    nt0 = len(bt)
    bary_x = bv[bt].mean(axis=1)[:, 0]
    end = np.argsort(bary_x, kind="stable")[:6]
    mask = np.zeros(nt0, np.uint8)
    mask[end] = 1
    vol_um3 = 12 * (h / I.UM) ** 3
    rng = np.random.default_rng(4)
    one = np.zeros((model.n_species, nt0), np.int32)
    for s, name in enumerate(model.names):
        if name == "Ca":
            one[s] = I.place_uniform(120, nt0, seed=400, subset=end)
        elif name.startswith("B"):
            one[s] = I.place_uniform(int(round(rng.uniform(200, 600) * vol_um3)), nt0, seed=400 + s)
        elif name.startswith("T"):
            one[s] = I.place_uniform(int(round(rng.uniform(10, 100) * vol_um3)), nt0, seed=400 + s)
    influx = model.n_reac - 1
    verts, tets, counts, masks, _ = _replicated(bv, bt, h, one, {influx: mask})
    t_end = 0.6e-3
    gpu, gw = _run_gpu(capi, verts, tets, model, counts, masks, 1003, t_end)
    orc, ow = _run_oracle(verts, tets, model, counts, masks, 2004, t_end)
    assert gw == ow >= 10
    ca, b0, cab0 = model.names.index("Ca"), model.names.index("B0"), model.names.index("CaB0")
    far = int(np.argmax(bary_x))
    fam = _family(gpu, orc, nt0, [(ca, int(end[0])), (ca, far), (cab0, int(end[1])), (b0, far)])
    _check_family(fam, "calcium network")
    pump = model.reac_names.index("Ca -> ")
    for r, factor in ((pump, 1.05), (_fastest(model, 2), 2.0)):
        p_alt = _sensitivity(gpu, verts, tets, model, counts, masks, 2004, t_end, nt0, r, factor)
        print(f"calcium network, oracle with k[{r}] x {factor}: smallest KS p {p_alt:.3g}")
        assert p_alt < 1e-6
