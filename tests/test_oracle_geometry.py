"""Pins of the oracle's mesh geometry, face rates and time window against
closed forms (§2.1: local diffusion rate d_{S,tet} = sum_f D_S A_f / (V d_f)
and tau = min 1/d_{S,tet})."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_02258_gb300 import inputs as I


def test_kuhn_cube_closed_forms():
    """Unit cube split into 6 Kuhn tets: V = 1/6 each; every tet has two faces
    on the cube surface (area 1/2) and two on diagonal planes (area sqrt(2)/2)
    shared with another tet of the cube; adjacent barycentres are sqrt(2)/4
    apart, so g = A/(V d) = 12 on internal faces."""
    verts, tets = I.kuhn_box_mesh(1, 1, 1, 1.0)
    nbr, vol, area, dist, g = oracle.geometry(verts, tets)
    assert np.allclose(vol, 1.0 / 6.0, rtol=0, atol=1e-15)
    for i in range(6):
        internal = nbr[i] >= 0
        assert internal.sum() == 2
        assert np.allclose(np.sort(area[i]), [0.5, 0.5, math.sqrt(2) / 2, math.sqrt(2) / 2], atol=1e-15)
        assert np.allclose(area[i][internal], math.sqrt(2) / 2, atol=1e-15)
        assert np.allclose(dist[i][internal], math.sqrt(2) / 4, atol=1e-15)
        assert np.allclose(g[i][internal], 12.0, rtol=1e-14)
        assert np.all(g[i][~internal] == 0.0)
    # the 6 tets form a ring around the diagonal
    deg = np.bincount(nbr[nbr >= 0].ravel(), minlength=6)
    assert np.all(deg == 2)


def test_kuhn_grid_face_counts_and_cross_cube_rate():
    """nx*ny*nz Kuhn grid: each cube has 6 internal face pairs, each shared
    square carries 2 triangle pairs; boundary triangles = 4 per boundary square.
    Across a cube face the barycentres are sqrt(6)/4 h apart and the triangle
    has area h^2/2, so g = 2 sqrt(6) / h^2."""
    nx, ny, nz, h = 3, 2, 4, 0.5e-6
    verts, tets = I.kuhn_box_mesh(nx, ny, nz, h)
    nbr, vol, area, dist, g = oracle.geometry(verts, tets)
    n_internal = (nbr >= 0).sum()
    shared_squares = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert n_internal == 2 * (6 * nx * ny * nz + 2 * shared_squares)
    boundary_squares = 2 * (nx * ny + ny * nz + nx * nz)
    assert (nbr < 0).sum() == 2 * boundary_squares
    cross = np.isclose(area, h * h / 2, rtol=1e-12, atol=0) & (nbr >= 0)
    assert cross.sum() == 4 * shared_squares
    assert np.allclose(dist[cross], math.sqrt(6) / 4 * h, rtol=1e-12)
    assert np.allclose(g[cross], 2 * math.sqrt(6) / h**2, rtol=1e-12)
    # every neighbour relation is mutual
    for i in range(len(tets)):
        for f in range(4):
            j = nbr[i, f]
            if j >= 0:
                assert i in nbr[j]


def test_regular_tetrahedron():
    a = 2.0
    verts = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.float64)  # edge 2*sqrt(2)
    e = 2 * math.sqrt(2)
    verts = verts * (a / e)
    nbr, vol, area, dist, g = oracle.geometry(verts, np.array([[0, 1, 2, 3]], np.int32))
    assert vol[0] == pytest.approx(a**3 / (6 * math.sqrt(2)), rel=1e-14)
    assert np.allclose(area[0], math.sqrt(3) / 4 * a * a, rtol=1e-14)
    assert np.all(nbr == -1) and np.all(g == 0)


def test_detailed_balance_and_similarity_on_jittered_mesh():
    """A/d is a property of the shared face: V_i g_ij = V_j g_ji. Scaling the
    mesh by L multiplies V by L^3 and g by 1/L^2; translating changes nothing."""
    h = 0.5e-6
    verts, tets = I.kuhn_box_mesh(5, 4, 3, h)
    verts = I.jitter_box_vertices(verts, h, 0.2, seed=4)
    nbr, vol, area, dist, g = oracle.geometry(verts, tets)
    for i in range(len(tets)):
        for f in range(4):
            j = nbr[i, f]
            if j < 0:
                continue
            fj = list(nbr[j]).index(i)
            assert dist[i, f] == dist[j, fj]
            assert area[i, f] == pytest.approx(area[j, fj], rel=1e-12)
            assert vol[i] * g[i, f] == pytest.approx(vol[j] * g[j, fj], rel=1e-12)
    nbr2, vol2, area2, dist2, g2 = oracle.geometry(verts * 3.0 + 1e-5, tets)
    assert np.array_equal(nbr, nbr2)
    assert np.allclose(vol2, vol * 27, rtol=1e-9)
    assert np.allclose(g2, g / 9, rtol=1e-9)
    assert np.all(vol > 0.1 * h**3 / 6)  # jitter of 0.2h inverts nothing


def test_tau_closed_form_and_thresholds():
    """Interior Kuhn tets have G = (24 + 4 sqrt 6)/h^2, the largest on a regular
    grid, so tau = h^2 / (D (24 + 4 sqrt 6)) (7.3969e-4 s for h = 0.5 um,
    D = 1e-11). The fastest tet has leave probability 1: its cumulative
    threshold is 2^31."""
    w = I.config1()
    sim = oracle.OracleSim(w.verts, w.tets, w.model, seed=1)
    h, D = 0.5e-6, 1e-11
    assert sim.tau == pytest.approx(h * h / (D * (24 + 4 * math.sqrt(6))), rel=1e-12)
    thr = sim.thresholds().astype(np.int64)
    assert thr.max() == 2**31 or thr.max() == 2**31 - 1
    assert np.all(np.diff(thr, axis=1) >= 0)  # cumulative
    # per-face widths are 2^31 * tau * D * g_f
    nbr, vol, area, dist, g = oracle.geometry(w.verts, w.tets)
    width = np.diff(np.concatenate([np.zeros((len(thr), 1)), thr], axis=1), axis=1) / 2**31
    assert np.allclose(width, sim.tau * D * g, atol=2 / 2**31)


def test_tau_min_over_diffusive_species_only():
    verts, tets = I.kuhn_box_mesh(2, 2, 2, 0.5e-6)
    m = I.model_from_lists(["A", "B"], [0.0, 2e-12], [])
    sim = oracle.OracleSim(verts, tets, m, seed=1)
    m2 = I.model_from_lists(["A", "B"], [4e-12, 2e-12], [])
    sim2 = oracle.OracleSim(verts, tets, m2, seed=1)
    assert sim.tau == pytest.approx(2 * sim2.tau, rel=1e-14)
    m3 = I.model_from_lists(["A"], [0.0], [])
    assert math.isinf(oracle.OracleSim(verts, tets, m3, seed=1).tau)


def test_bad_meshes_rejected():
    verts, tets = I.kuhn_box_mesh(1, 1, 1, 1.0)
    m = I.model_from_lists(["A"], [1e-12], [])
    bad = np.concatenate([tets, tets[:1]])  # a face shared by 3 tets
    with pytest.raises(ValueError):
        oracle.OracleSim(verts, bad, m, seed=1)
    flat = tets.copy()
    flat[0] = [0, 1, 2, 2]  # degenerate
    with pytest.raises(ValueError):
        oracle.OracleSim(verts, flat, m, seed=1)
    oob = tets.copy()
    oob[0, 0] = 999
    with pytest.raises(ValueError):
        oracle.OracleSim(verts, oob, m, seed=1)


def test_full_box_jitter_bounds_and_volumes():
    """The benchmark box mesh (294,780 tets, vertices jittered by up to 20 % of
    the spacing h per axis): every vertex moves at most 0.2 h per axis,
    boundary vertices stay in their boundary planes, no tet inverts, and the
    smallest volume stays well above zero (the reading taken for the jitter:
    at 0.2 h a Kuhn tet cannot invert, so nothing is resampled)."""
    from paper_1610_02258_gb300 import inputs as I
    h = 10.0 / 17.0 * I.UM
    v0, tets = I.kuhn_box_mesh(170, 17, 17, h)
    w = I.config2()
    v = w.verts
    assert v.shape == v0.shape and np.array_equal(w.tets, tets)
    d = np.abs(v - v0)
    assert d.max() <= 0.2 * h * (1 + 1e-12)
    lo, hi = v0.min(axis=0), v0.max(axis=0)
    on_face = (np.isclose(v0, lo, rtol=0, atol=1e-3 * h) | np.isclose(v0, hi, rtol=0, atol=1e-3 * h))
    assert np.array_equal(v[on_face], v0[on_face])
    def signed_volume(x):
        p = x[tets]
        return np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0])) / 6.0

    vol, vol0 = signed_volume(v), signed_volume(v0)
    nominal = h ** 3 / 6.0
    assert np.allclose(np.abs(vol0), nominal, rtol=1e-9)
    assert np.all(np.sign(vol) == np.sign(vol0))  # no tet turned inside out
    assert np.abs(vol).min() > 0.1 * nominal
    _, vol_o, *_ = oracle.geometry(v, tets)
    assert np.allclose(vol_o, np.abs(vol), rtol=1e-9, atol=0)
