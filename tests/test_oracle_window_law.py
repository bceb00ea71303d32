"""Pins of the oracle's shortened windows, its fixed-point leave thresholds and
its occupancy trial rule (Algorithm 1: the last window of a run is cut to
t_end - t; the diffusion operator's binomial(Nbar, tau, d_{S,tet}); §2.1 for
d_{S,tet} = sum_f D_S A_f / (V d_f)).

- A window of length c*tau moves each molecule of species S with the one-window
  matrix I + c*tau*Q_S, Q_S the generator of the face rates D_S*A/(V*d). Over
  independent copies the per-tet totals after K such windows are exactly
  Multinomial with a row of (I + c tau Q_S)^K; dropping the tau_k/tau factor
  (a full window's law) fails.
- Every species' cumulative threshold T_f, for a full or a shortened window,
  lies below 2^31 * tau_k * D_S * sum_{f'<=f} g_f' by less than
  1 + p_tet + p_S units of 2^-31 (p_tet = tau D_max G_tet <= 1 and
  p_S = (D_S/D_max)(tau_k/tau) <= 1, the two fixed-point factors), with the
  geometry recomputed here in numpy from the vertices.
- Occupancy (OCC) against end-count (END) trials as tau -> 0: with the same
  seed both modes run the same reactions, and to first order in tau they
  differ only after one B -> A event at a uniform time in the window (an
  A -> B event is clamped back to the end count), which costs half a trial on
  average. So E[M_OCC - M_END] / tau -> -kb N_B / 2, and the trial counts of
  the two modes agree in every tet where no reaction fired.
- The EXP leave law (p = 1 - exp(-tau_k d) instead of tau_k d): counts follow
  I + diag((1 - e^{-tau_k d}) / d) D Q and not the EULER matrix, and its
  thresholds lie within 3 units of 2^31 (1 - e^{-tau_k D G}) cumg_f / G.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import END, OCC
from paper_1610_02258_gb300 import inputs as I
from tests.stats import chi2_table_pvalue

H = 0.5e-6
PAIR_G = 12.0 / H**2  # g of the shared face of two Kuhn tets of one cube

_FACE = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]  # face f is opposite vertex f


def np_geometry(verts, tets):
    """Face neighbours and g = A / (V d) of every local face, recomputed with
    numpy from the vertices (independent of the oracle's C geometry)."""
    nt = len(tets)
    owner = {}
    nbr = -np.ones((nt, 4), np.int64)
    for i in range(nt):
        for f, fv in enumerate(_FACE):
            key = tuple(sorted(int(tets[i, k]) for k in fv))
            if key in owner:
                j, fj = owner.pop(key)
                nbr[i, f], nbr[j, fj] = j, i
            else:
                owner[key] = (i, f)
    p = verts[tets]                                   # [nt, 4, 3]
    vol = np.abs(np.linalg.det(p[:, 1:] - p[:, :1])) / 6.0
    bary = p.mean(axis=1)
    g = np.zeros((nt, 4))
    for f, (a, b, c) in enumerate(_FACE):
        area = 0.5 * np.linalg.norm(np.cross(p[:, b] - p[:, a], p[:, c] - p[:, a]), axis=1)
        ok = nbr[:, f] >= 0
        d = np.linalg.norm(bary[nbr[ok, f]] - bary[ok], axis=1)
        g[ok, f] = area[ok] / (vol[ok] * d)
    return nbr, vol, g


def one_window_matrix(nbr, g, rate):
    """I + rate * Q: rate = tau_k * D_S; Q[i, j] = g over the faces i shares with j."""
    nt = len(nbr)
    P = np.zeros((nt, nt))
    for i in range(nt):
        for f in range(4):
            if nbr[i, f] >= 0:
                P[i, nbr[i, f]] += rate * g[i, f]
        P[i, i] = 1.0 - P[i].sum()
    return P


@pytest.mark.parametrize("c", [0.37, 0.81])
def test_shortened_window_diffusion_law(c):
    """Species A diffuses 2.5 times slower than an empty species F that sets
    tau, so the window's thresholds carry both factors D_A/D_max and
    tau_k/tau. After K windows of c*tau the per-tet totals over 400 copies of
    a jittered 3x3x2-cube mesh are Multinomial(N0 * copies, row of
    (I + c tau D_A Q)^K); with the tau_k/tau factor dropped they are not."""
    bv, bt = I.kuhn_box_mesh(3, 3, 2, H)
    bv = I.jitter_box_vertices(bv, H, 0.2, seed=8)
    copies, N0, K, D = 400, 50, 3, 1e-11
    DA = D / 2.5
    verts, tets = I.replicate_mesh(bv, bt, copies, spacing=3 * H + 4 * H)
    nt0 = len(bt)
    m = I.model_from_lists(["A", "F"], [DA, D], [])
    start = 17
    cnt = np.zeros((2, nt0 * copies), np.int32)
    cnt[0, start::nt0] = N0
    for occ in (OCC, END):
        sim = oracle.OracleSim(verts, tets, m, seed=44 + occ, occ=occ, prec=64)
        sim.set_counts(cnt)
        for _ in range(K):
            sim.step(c * sim.tau)
        out = sim.get_counts()
        assert out[1].sum() == 0
        agg = out[0].reshape(copies, nt0).sum(axis=0)
        assert agg.sum() == N0 * copies
        nbr, vol, g = np_geometry(bv, bt)
        tau = 1.0 / (D * (g.sum(axis=1)).max())
        assert sim.tau == pytest.approx(tau, rel=1e-12)
        law = np.linalg.matrix_power(one_window_matrix(nbr, g, c * tau * DA), K)[start]
        assert law.min() >= 0
        assert chi2_table_pvalue(agg, law) > 1e-3
        # the tau_k/tau factor dropped: every window moves as a full one
        wrong = np.linalg.matrix_power(one_window_matrix(nbr, g, tau * DA), K)[start]
        assert chi2_table_pvalue(agg, wrong) < 1e-6


@pytest.mark.parametrize("c", [1.0, 0.81, 0.37, 1e-3])
def test_species_thresholds_against_fp64(c):
    """Every species of a 10-species model with D spread over two decades, on
    a jittered 6x5x4-cube mesh (720 tets): the window's cumulative threshold
    T_f of every tet and face is floor-quantised from 2^31 tau_k D_S
    sum_{f'<=f} g_f' in two fixed-point factors, so
    0 <= X - T < 1 + p_tet + p_S (units of 2^-31). A species with D = 0
    never leaves."""
    bv, bt = I.kuhn_box_mesh(6, 5, 4, H)
    verts = I.jitter_box_vertices(bv, H, 0.2, seed=12)
    D = np.array([1e-11, 3.7e-12, 1e-13, 5.5e-12, 0.0, 2.2e-13, 9.9e-12, 1e-11, 4e-12, 6.1e-13])
    m = I.model_from_lists([f"S{s}" for s in range(len(D))], D, [])
    sim = oracle.OracleSim(verts, bt, m, seed=1)
    nbr, vol, g = np_geometry(verts, bt)
    cumg = np.cumsum(g, axis=1)
    dmax, gmax = D.max(), cumg[:, 3].max()
    tau = 1.0 / (dmax * gmax)
    assert sim.tau == pytest.approx(tau, rel=1e-13)
    tau_k = c * tau
    p_tet = tau * dmax * cumg[:, 3:4]
    worst = 0.0
    for s, Ds in enumerate(D):
        T, scale = sim.species_thresholds(s, tau_k)
        if Ds == 0.0:
            assert scale == 0 and not T.any()
            continue
        p_s = (Ds / dmax) * c
        assert scale == pytest.approx(p_s * 2**31, abs=1.0 + 1e-6)
        X = 2.0**31 * tau_k * Ds * cumg
        gap = X - T.astype(np.float64)
        assert gap.min() >= -1e-5
        assert np.all(gap < 1.0 + p_tet + p_s + 1e-5)
        assert np.all(np.diff(T.astype(np.int64), axis=1) >= 0)
        worst = max(worst, float(gap.max()))
    assert worst < 3.0


def test_occupancy_trials_approach_end_count():
    """Isolated pairs of Kuhn tets; tet 0 holds 10 A and 10 B with A <-> B
    (kf = 30 /s, kb = 60 /s); A diffuses with leave probability 1 (it sets
    tau), B is immobile, so after one window the A in tet 1 is the trial count
    M_A. tau is shrunk by raising D_A. With eps = (kf N_A + kb N_B) tau the
    mean number of events per tet and window:
    - the ratio r = E[M_OCC - M_END] / (-kb N_B tau / 2) is 1 within eps/2 + 4 SE;
    - the fraction of pairs whose counts differ is at most the probability of
      any event, 1 - exp(-eps), within 4 SE;
    - |E[M_OCC - M_END]| shrinks in proportion to tau.
    A plausible mistake moves r far from 1: occupancy summed with the count
    after the event gives 0, truncation instead of stochastic rounding 2, no
    clamp to the end count 0.5."""
    n, NA0, NB0, kf, kb = 40000, 10, 10, 30.0, 60.0
    verts, tets = I.isolated_pairs(n)
    deltas = []
    for DA in (1.024e-10, 4.096e-10):
        m = I.model_from_lists(["A", "B"], [DA, 0.0], [(["A"], ["B"], kf), (["B"], ["A"], kb)])
        c = np.zeros((2, 2 * n), np.int32)
        c[0, 0::2] = NA0
        c[1, 0::2] = NB0
        moved = {}
        for occ in (OCC, END):
            sim = oracle.OracleSim(verts, tets, m, seed=5, occ=occ, prec=64)
            sim.set_counts(c)
            tau = sim.tau
            assert tau == pytest.approx(1.0 / (DA * PAIR_G), rel=1e-12)
            sim.step(tau)
            out = sim.get_counts()
            assert np.array_equal(out[0].reshape(n, 2).sum(axis=1) + out[1].reshape(n, 2).sum(axis=1),
                                  np.full(n, NA0 + NB0))
            assert not out[1, 1::2].any()
            moved[occ] = out[0, 1::2].astype(np.float64)
        d = moved[OCC] - moved[END]
        eps = (kf * NA0 + kb * NB0) * tau
        pred = -kb * NB0 * tau / 2
        r = d.mean() / pred
        se = d.std(ddof=1) / math.sqrt(n) / abs(pred)
        assert abs(r - 1.0) < eps / 2 + 4 * se, (tau, eps, r, se)
        frac = float((d != 0).mean())
        assert frac <= 1 - math.exp(-eps) + 4 * math.sqrt(frac * (1 - frac) / n)
        deltas.append((tau, d.mean()))
    (t1, d1), (t2, d2) = deltas
    assert d2 / d1 == pytest.approx(t2 / t1, rel=0.35)


def exp_window_matrix(nbr, g, tau_k, D):
    """EXP law: molecule in tet i leaves with 1 - exp(-tau_k d_i), d_i = D G_i,
    through face f in proportion to g_f: P = I + diag((1 - e^{-tau_k d}) / d) D Q."""
    nt = len(nbr)
    G = g.sum(axis=1)
    P = np.zeros((nt, nt))
    for i in range(nt):
        if G[i] <= 0:
            P[i, i] = 1.0
            continue
        p_leave = 1.0 - np.exp(-tau_k * D * G[i])
        for f in range(4):
            if nbr[i, f] >= 0:
                P[i, nbr[i, f]] += p_leave * g[i, f] / G[i]
        P[i, i] = 1.0 - P[i].sum()
    return P


@pytest.mark.parametrize("c", [1.0, 0.6])
def test_exp_law_diffusion_is_multinomial(c):
    """The EXP leave law (p = 1 - exp(-tau d)): per-tet totals over 400
    copies after K windows of c*tau are Multinomial with a row of the EXP
    matrix's K-th power, and not with the EULER law's (p = tau d)."""
    bv, bt = I.kuhn_box_mesh(3, 3, 2, H)
    bv = I.jitter_box_vertices(bv, H, 0.2, seed=8)
    copies, N0, K, D = 400, 40, 3, 1e-11
    verts, tets = I.replicate_mesh(bv, bt, copies, spacing=3 * H + 4 * H)
    nt0 = len(bt)
    m = I.model_from_lists(["A"], [D], [])
    start = 17
    cnt = np.zeros((1, nt0 * copies), np.int32)
    cnt[0, start::nt0] = N0
    sim = oracle.OracleSim(verts, tets, m, seed=61, leave=oracle.EXP)
    sim.set_counts(cnt)
    for _ in range(K):
        sim.step(c * sim.tau)
    agg = sim.get_counts()[0].reshape(copies, nt0).sum(axis=0)
    assert agg.sum() == N0 * copies
    nbr, vol, g = np_geometry(bv, bt)
    tau = 1.0 / (D * g.sum(axis=1).max())
    law = np.linalg.matrix_power(exp_window_matrix(nbr, g, c * tau, D), K)[start]
    assert chi2_table_pvalue(agg, law) > 1e-3
    euler = np.linalg.matrix_power(one_window_matrix(nbr, g, c * tau * D), K)[start]
    assert chi2_table_pvalue(agg, euler) < 1e-6


@pytest.mark.parametrize("c", [1.0, 0.37])
def test_exp_thresholds_against_fp64(c):
    """EXP law thresholds T_f = (share_f * L) >> 31 lie below
    2^31 (1 - exp(-tau_k D_S G)) cumg_f / G by less than 3 units (two floors
    of factors <= 1, and the product's floor)."""
    bv, bt = I.kuhn_box_mesh(6, 5, 4, H)
    verts = I.jitter_box_vertices(bv, H, 0.2, seed=12)
    D = np.array([1e-11, 3.7e-12, 0.0, 2.2e-13])
    m = I.model_from_lists([f"S{s}" for s in range(len(D))], D, [])
    sim = oracle.OracleSim(verts, bt, m, seed=1, leave=oracle.EXP)
    nbr, vol, g = np_geometry(verts, bt)
    cumg = np.cumsum(g, axis=1)
    G = cumg[:, 3:4]
    tau = 1.0 / (D.max() * G.max())
    tau_k = c * tau
    for s, Ds in enumerate(D):
        T, _ = sim.species_thresholds(s, tau_k)
        if Ds == 0.0:
            assert not T.any()
            continue
        X = 2.0**31 * (1.0 - np.exp(-tau_k * Ds * G)) * cumg / G
        gap = X - T.astype(np.float64)
        assert gap.min() >= -1e-5 and gap.max() < 3.0
        assert np.all(np.diff(T.astype(np.int64), axis=1) >= 0)
