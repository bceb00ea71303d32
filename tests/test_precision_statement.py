"""The float-vs-double propensity error of the reaction operator.

The kernel evaluates mass-action propensities in float, in a fixed order
(order 0: k / (1/(N_A V)); order 1: k N; order 2: ((k * (1/(N_A V))) N_a) N_b),
from float copies of k and 1/(N_A V); the oracle's reference mode evaluates
them in double. This test measures the relative difference over every
reaction of the benchmark networks, every tet volume of the meshes and
counts up to 1000, and pins the bound stated with the benchmark: at most
3 float roundings of k and 1/(N_A V) plus 3 of the products, i.e. below
6 * 2^-24 = 3.6e-7 relative."""
import numpy as np

from paper_1610_02258_gb300 import inputs as I

NA = 6.02214076e23


def _volumes(verts, tets):
    p = verts[tets]
    u, v, w = p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]
    return np.abs(np.einsum("ij,ij->i", u, np.cross(v, w))) / 6.0


def _rel_err(model, vols, counts):
    f32 = np.float32
    worst = 0.0
    for r in range(model.n_reac):
        reac = [s for s in range(model.n_species) for _ in range(model.lhs[r, s])]
        k = model.k[r]
        nav = NA * (vols * 1000.0)
        inv = (1.0 / nav).astype(f32)
        kf = f32(k)
        for n in counts:
            if len(reac) == 0:
                a32 = kf / inv
                a64 = k * nav
            elif len(reac) == 1:
                a32 = np.full_like(inv, kf * f32(n))
                a64 = np.full_like(nav, k * n)
            else:
                m = n - 1 if reac[0] == reac[1] else n
                a32 = ((kf * inv) * f32(n)) * f32(m)
                a64 = k / nav * n * m
            ok = a64 > 0
            if ok.any():
                worst = max(worst, float(np.max(np.abs(a32[ok].astype(np.float64) - a64[ok]) / a64[ok])))
    return worst


def test_float_propensity_error_bound():
    counts = [1, 2, 3, 7, 10, 33, 100, 999]
    w2 = I.config2(nx=4)
    e2 = _rel_err(w2.model, _volumes(w2.verts, w2.tets), counts)
    w3 = I.config3(h=0.5e-6, t_end=1e-3)
    e3 = _rel_err(w3.model, _volumes(w3.verts, w3.tets), counts)
    assert e2 < 6 * 2.0**-24 and e3 < 6 * 2.0**-24, (e2, e3)
    assert e2 > 0 and e3 > 0
