"""Pins of the oracle's simulation against laws fixed by the mathematics of
the operator-split method (Algorithm 1), each chosen so that a plausible
mistake in one part fails at least one test:

- conservation (any dropped or doubled molecule in the apply step);
- first-order decay and reversible A<->B: each molecule's identity is an
  independent two-state chain, so totals are exactly binomial whatever the
  mesh and the diffusion (SSA waiting times, selection, stoichiometry signs);
- one well-mixed tet: A + B <-> C against the chemical master equation solved
  by the matrix exponential (second-order propensity convention);
- pure diffusion: molecules are independent walkers with the one-window
  transition matrix P = I + tau*Q (face rates D*A/(V*d)), so per-tet totals
  over independent copies are exactly multinomial with the rows of P^K
  (geometry, neighbour indexing, thresholds, sampler, Jacobi apply);
- occupancy mode: zero-order production gives E[trials] = a*tau/2 against
  a*tau for the end-count mode; pure decay makes the two modes identical;
- two tets, homodimer annihilation + diffusion in end-count mode: the exact
  law of the split chain (reaction operator expm(Q_R tau) per tet, then the
  binomial diffusion operator), composed over windows;
- the window loop: full windows, the shortened last window, resumption.
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import expm

import oracle
from oracle import END, OCC
from paper_1610_02258_gb300 import inputs as I
from tests.stats import chi2_pvalue, chi2_table_pvalue

NA = 6.02214076e23
H = 0.5e-6
V_KUHN_L = H**3 / 6 * 1e3  # litres of one Kuhn tet of a 0.5 um cube
PAIR_G = 12.0 / H**2       # g of the shared face of two Kuhn tets of one cube

MODES = [(OCC, 64), (OCC, 32), (END, 64), (END, 32)]


def _sim(verts, tets, model, counts, seed, occ=OCC, prec=64, masks=None):
    s = oracle.OracleSim(verts, tets, model, seed=seed, occ=occ, prec=prec)
    s.set_counts(counts)
    for r, m in (masks or {}).items():
        s.set_reac_mask(r, m)
    return s


@pytest.mark.parametrize("occ,prec", MODES)
def test_conservation_every_window(occ, prec):
    """A + B <-> C with kf = 1e8 /M/s (about 70 events per window on the
    cuboid, so reactions surely fire): A + C and B + C are conserved."""
    w = I.config1()
    fast = I.model_from_lists(["A", "B", "C"], [1e-11] * 3, [(["A", "B"], ["C"], 1e8), (["C"], ["A", "B"], 10.0)])
    sim = _sim(w.verts, w.tets, fast, w.counts, 9, occ, prec)
    tot = w.counts.sum(axis=1)
    events = 0
    for _ in range(6):
        sim.step(sim.tau)
        c = sim.get_counts()
        assert c.min() >= 0
        assert c[0].sum() + c[2].sum() == tot[0] + tot[2]
        assert c[1].sum() + c[2].sum() == tot[1] + tot[2]
    events = sim.events
    assert events > 0
    # pure diffusion: every species total is constant
    m = I.model_from_lists(["A", "B"], [1e-11, 3e-12], [])
    sim = _sim(w.verts, w.tets, m, w.counts[:2], 9, occ, prec)
    for _ in range(5):
        sim.step(sim.tau)
        assert np.array_equal(sim.get_counts().sum(axis=1), w.counts[:2].sum(axis=1))


@pytest.mark.parametrize("occ,prec", MODES)
def test_first_order_decay_is_binomial(occ, prec):
    """A -> 0 at k: N(t) ~ Bin(N0, exp(-k t)) exactly, per independent pair."""
    n, N0, k, t = 6000, 20, 50.0, 10e-3
    verts, tets = I.isolated_pairs(n)
    m = I.model_from_lists(["A"], [1e-11], [(["A"], [], k)])
    c = np.zeros((1, 2 * n), np.int32)
    c[0, 0::2] = N0
    sim = _sim(verts, tets, m, c, 21, occ, prec)
    sim.run(t)
    assert sim.windows >= 5  # several full windows plus a shortened one
    tot = sim.get_counts()[0].reshape(n, 2).sum(axis=1)
    p = math.exp(-k * t)
    ks = np.arange(N0 + 1)
    assert chi2_pvalue(tot, ks, stats.binom.pmf(ks, N0, p)) > 1e-3


@pytest.mark.parametrize("occ,prec", MODES)
def test_reversible_isomerisation_is_binomial(occ, prec):
    """A <-> B (kf, kb): from all-A, N_A(t) ~ Bin(N, pi + (1 - pi) e^{-(kf+kb) t}),
    pi = kb / (kf + kb), whatever the diffusion."""
    n, N, kf, kb, t = 6000, 10, 80.0, 40.0, 15e-3
    verts, tets = I.isolated_pairs(n)
    m = I.model_from_lists(["A", "B"], [1e-11, 2e-12], [(["A"], ["B"], kf), (["B"], ["A"], kb)])
    c = np.zeros((2, 2 * n), np.int32)
    c[0, 0::2] = N
    sim = _sim(verts, tets, m, c, 22, occ, prec)
    sim.run(t)
    out = sim.get_counts()
    a = out[0].reshape(n, 2).sum(axis=1)
    assert np.all(a + out[1].reshape(n, 2).sum(axis=1) == N)
    pi = kb / (kf + kb)
    p = pi + (1 - pi) * math.exp(-(kf + kb) * t)
    ks = np.arange(N + 1)
    assert chi2_pvalue(a, ks, stats.binom.pmf(ks, N, p)) > 1e-3


@pytest.mark.parametrize("prec", [64, 32])
def test_single_tet_matches_master_equation(prec):
    """A + B <-> C in one well-mixed tet is plain Gillespie SSA (no diffusive
    face, tau = inf: one window). N_C(t) against expm(Q t) of the CME."""
    n, N0, kf, kb, t = 20000, 10, 1e8, 50.0, 5e-3
    verts, tets = I.isolated_tets(n)
    m = I.model_from_lists(["A", "B", "C"], [1e-11, 1e-11, 1e-11],
                           [(["A", "B"], ["C"], kf), (["C"], ["A", "B"], kb)])
    c = np.zeros((3, n), np.int32)
    c[0] = N0
    c[1] = N0
    sim = _sim(verts, tets, m, c, 23, OCC, prec)
    assert math.isinf(sim.tau)
    sim.run(t)
    assert sim.windows == 1
    out = sim.get_counts()
    cf = kf / (NA * V_KUHN_L)
    Q = np.zeros((N0 + 1, N0 + 1))
    for x in range(N0 + 1):  # x = N_C
        up = cf * (N0 - x) * (N0 - x)
        dn = kb * x
        if x < N0:
            Q[x, x + 1] = up
        if x > 0:
            Q[x, x - 1] = dn
        Q[x, x] = -(up + dn)
    p = expm(Q * t)[0]
    assert chi2_pvalue(out[2], np.arange(N0 + 1), p) > 1e-3
    assert np.all(out[0] == N0 - out[2]) and np.all(out[1] == N0 - out[2])


def _transition_matrix(sim_tau, D, nbr, g):
    nt = nbr.shape[0]
    P = np.zeros((nt, nt))
    for i in range(nt):
        for f in range(4):
            j = nbr[i, f]
            if j >= 0:
                P[i, j] += sim_tau * D * g[i, f]
        P[i, i] = 1.0 - P[i].sum()
    return P


@pytest.mark.parametrize("occ", [OCC, END])
def test_pure_diffusion_law_is_multinomial(occ):
    """Independent walkers: summed over independent copies of a jittered
    3x3x2-cube mesh, per-tet counts after K windows are Multinomial with the
    row of P^K of the start tet."""
    h = H
    bv, bt = I.kuhn_box_mesh(3, 3, 2, h)
    bv = I.jitter_box_vertices(bv, h, 0.2, seed=8)
    copies, N0, K, D = 400, 50, 3, 1e-11
    verts, tets = I.replicate_mesh(bv, bt, copies, spacing=3 * h + 4 * h)
    nt0 = bt.shape[0]
    m = I.model_from_lists(["A"], [D], [])
    c = np.zeros((1, nt0 * copies), np.int32)
    start = 17
    c[0, start::nt0] = N0
    sim = _sim(verts, tets, m, c, 24, occ, 64)
    for _ in range(K):
        sim.step(sim.tau)
    agg = sim.get_counts()[0].reshape(copies, nt0).sum(axis=0)
    nbr, vol, area, dist, g = oracle.geometry(bv, bt)
    P = _transition_matrix(sim.tau, D, nbr, g)
    pk = np.linalg.matrix_power(P, K)[start]
    assert pk.min() >= 0
    assert chi2_table_pvalue(agg, pk) > 1e-3
    # the same counts are not multinomial under a plausible mistake
    # (walkers sent to the tet across the *next* local face)
    nbr_bad = np.roll(nbr, 1, axis=1)
    g_bad = g.copy()
    Pb = _transition_matrix(sim.tau, D, np.where(nbr_bad >= 0, nbr_bad, -1), g_bad)
    pkb = np.clip(np.linalg.matrix_power(np.clip(Pb, 0, None), K)[start], 0, None)
    assert chi2_table_pvalue(agg, pkb + 1e-12) < 1e-6


def test_occupancy_mode_production_law():
    """0 -> A and 0 -> B at a (molecules/s) in tet 0 of isolated pairs, B four
    times slower than A (so p_A = 1, p_B = 1/4 over the shared face). After one
    window from empty: OCC trials have mean a tau / 2 (time average of a
    Poisson ramp); END trials are the end count, mean a tau."""
    n, a_rate = 20000, 2000.0
    verts, tets = I.isolated_pairs(n)
    kM = a_rate / (NA * V_KUHN_L)
    DA = 1e-11
    m = I.model_from_lists(["A", "B"], [DA, DA / 4], [([], ["A"], kM), ([], ["B"], kM)])
    mask = np.zeros(2 * n, np.uint8)
    mask[0::2] = 1
    tau = 1.0 / (DA * PAIR_G)
    for occ, frac in [(OCC, 0.5), (END, 1.0)]:
        sim = _sim(verts, tets, m, np.zeros((2, 2 * n), np.int32), 25, occ, 64, masks={0: mask, 1: mask})
        assert sim.tau == pytest.approx(tau, rel=1e-12)
        sim.step(sim.tau)
        out = sim.get_counts()
        for s, p in [(0, 1.0), (1, 0.25)]:
            moved = out[s, 1::2].astype(np.float64)
            total = out[s].reshape(n, 2).sum(axis=1)
            assert total.mean() == pytest.approx(a_rate * tau, abs=4 * total.std() / math.sqrt(n))
            expect = p * frac * a_rate * tau
            assert moved.mean() == pytest.approx(expect, abs=4 * moved.std() / math.sqrt(n) + 1e-12)


@pytest.mark.parametrize("prec", [64, 32])
def test_occupancy_equals_end_count_for_pure_decay(prec):
    """For a species that only decays, the window's time average is >= its end
    count, so the clamped trial count is the end count: OCC == END exactly."""
    w = I.config1()
    m = I.model_from_lists(["A", "B"], [1e-11, 5e-12], [(["A"], [], 30.0), (["B"], [], 80.0)])
    res = []
    for occ in (OCC, END):
        sim = _sim(w.verts, w.tets, m, w.counts[:2], 26, occ, prec)
        sim.run(6e-3)
        res.append(sim.get_counts())
        assert sim.events > 100
    assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("prec", [64, 32])
def test_two_tet_split_chain_exact_law(prec):
    """Two face-sharing tets, A + A -> 0 (homodimer, a = k/(N_A V) N (N-1)) and
    diffusion with p = 1/4 (a fast empty species sets tau), END mode. The law of
    (N_A in tet 0, N_A in tet 1) after K windows equals the composition of
    the exact per-window operators: reaction expm(Q_R tau) in each tet, then
    independent binomial moves across the face."""
    n, N0, K = 20000, 6, 3
    verts, tets = I.isolated_pairs(n)
    c_rate = 20.0
    k2 = c_rate * NA * V_KUHN_L
    DA = 1e-12
    m = I.model_from_lists(["A", "F"], [DA, 4 * DA], [(["A", "A"], [], k2)])
    c = np.zeros((2, 2 * n), np.int32)
    c[0, 0::2] = N0
    sim = _sim(verts, tets, m, c, 27, END, prec)
    tau = sim.tau
    p = DA * PAIR_G * tau
    assert p == pytest.approx(0.25, rel=1e-9)
    for _ in range(K):
        sim.step(tau)
    out = sim.get_counts()[0].reshape(n, 2)

    # exact chain over states (a0, a1), a0 + a1 <= N0
    Qr = np.zeros((N0 + 1, N0 + 1))
    for a in range(2, N0 + 1):
        Qr[a, a - 2] = c_rate * a * (a - 1)
        Qr[a, a] = -c_rate * a * (a - 1)
    Rt = expm(Qr * tau)
    states = [(a0, a1) for a0 in range(N0 + 1) for a1 in range(N0 + 1 - a0)]
    idx = {s: i for i, s in enumerate(states)}
    T = np.zeros((len(states), len(states)))
    for (a0, a1), i in idx.items():
        for b0 in range(a0 + 1):
            for b1 in range(a1 + 1):
                pr = Rt[a0, b0] * Rt[a1, b1]
                if pr == 0:
                    continue
                for n0 in range(b0 + 1):
                    for n1 in range(b1 + 1):
                        q = pr * stats.binom.pmf(n0, b0, p) * stats.binom.pmf(n1, b1, p)
                        T[i, idx[(b0 - n0 + n1, b1 - n1 + n0)]] += q
    dist = np.zeros(len(states))
    dist[idx[(N0, 0)]] = 1.0
    for _ in range(K):
        dist = dist @ T
    obs = np.zeros(len(states))
    for a0, a1 in out:
        obs[idx[(int(a0), int(a1))]] += 1
    assert chi2_table_pvalue(obs, dist) > 1e-3


def test_window_loop_partial_and_resume():
    w = I.config1()
    sim = _sim(w.verts, w.tets, w.model, w.counts, 31)
    tau = sim.tau
    sim.run(2.5 * tau)
    assert sim.windows == 3 and sim.time == 2.5 * tau
    sim.run(5.0 * tau)  # 2.5 -> 3.5 -> 4.5 -> 5.0
    assert sim.windows == 6 and sim.time == 5.0 * tau
    sim.run(5.0 * tau)  # no-op
    assert sim.windows == 6
    # stopping on the window grid and resuming is the same as one run
    a = _sim(w.verts, w.tets, w.model, w.counts, 31)
    a.run(3 * tau)
    a.run(7 * tau)
    b = _sim(w.verts, w.tets, w.model, w.counts, 31)
    b.run(7 * tau)
    assert a.windows == b.windows == 7
    assert np.array_equal(a.get_counts(), b.get_counts())
    # a different seed gives a different trajectory
    c = _sim(w.verts, w.tets, w.model, w.counts, 32)
    c.run(7 * tau)
    assert not np.array_equal(c.get_counts(), b.get_counts())


def test_reaction_only_model_one_window_per_run():
    verts, tets = I.isolated_tets(10)
    m = I.model_from_lists(["A"], [0.0], [(["A"], [], 10.0)])
    sim = _sim(verts, tets, m, np.full((1, 10), 5, np.int32), 1)
    sim.run(1e-3)
    sim.run(4e-3)
    assert sim.windows == 2 and sim.time == 4e-3


@pytest.mark.parametrize("prec", [64, 32])
def test_rate_change_gives_the_piecewise_poisson_law(prec):
    """Zero-order influx 0 -> A into isolated tets, no diffusion (each run is
    one exact SSA window): with rate k1 on [0, t1] and k2 on [t1, t2] the
    count at t2 is Poisson(N_A V (k1 t1 + k2 (t2 - t1))) (a Poisson process
    with a piecewise-constant rate). Ignoring the change (rate k1 throughout)
    predicts a mean 3x smaller on the second piece and fails the test."""
    n, k1, k2, t1, t2 = 4000, 2e-3, 6e-3, 1e-3, 2.5e-3
    verts, tets = I.isolated_tets(n)
    m = I.model_from_lists(["A"], [0.0], [([], ["A"], k1)])
    sim = _sim(verts, tets, m, np.zeros((1, n), np.int32), 31, OCC, prec)
    vol_l = (0.5e-6) ** 3 / 6.0 * 1e3  # a Kuhn tet of a 0.5 um cube, in litres
    nav = 6.02214076e23 * vol_l
    sim.run(t1)
    sim.set_reac_rate(0, k2)
    sim.run(t2)
    assert sim.windows == 2
    a = sim.get_counts()[0]
    lam = nav * (k1 * t1 + k2 * (t2 - t1))
    lam_wrong = nav * k1 * t2
    ks = np.arange(a.max() + 1)
    pmf = stats.poisson.pmf(ks, lam)
    pmf[-1] += stats.poisson.sf(ks[-1], lam)
    assert chi2_pvalue(a, ks, pmf) > 1e-3
    se = math.sqrt(lam / n)
    assert abs(a.mean() - lam) < 4 * se
    assert abs(a.mean() - lam_wrong) > 20 * se


def test_pure_diffusion_msd_exact_law_and_6Dt():
    """Mean-squared displacement of molecules released in the centre tet of a
    regular Kuhn mesh (16^3 cubes of 0.5 um, 24,576 tets), tau << t << L^2/D.
    (1) The sample MSD (barycentres) equals the scheme's exact expectation
        E[MSD] = sum_i (e_0 P^K)_i |b_i - b_0|^2, P = I + tau Q with Q built
        from the mesh's face rates D g_f, within 4 standard errors.
    (2) That expectation is 6 D t within 10 %: the two-point flux on the
        non-orthogonal Kuhn tets is not exact (the deviation is printed)."""
    import scipy.sparse as sp
    n_cube, h, D, N = 16, 0.5e-6, 1e-12, 20000
    verts, tets = I.kuhn_box_mesh(n_cube, n_cube, n_cube, h)
    nt = tets.shape[0]
    bary = verts[tets].mean(axis=1)
    centre = np.full(3, n_cube * h / 2)
    i0 = int(np.argmin(((bary - centre) ** 2).sum(axis=1)))
    m = I.model_from_lists(["A"], [D], [])
    c = np.zeros((1, nt), np.int32)
    c[0, i0] = N
    sim = _sim(verts, tets, m, c, 41)
    tau = sim.tau
    K = 90
    t = K * tau
    for _ in range(K):
        sim.step(tau)
    got = sim.get_counts()[0]
    assert got.sum() == N
    d2 = ((bary - bary[i0]) ** 2).sum(axis=1)
    msd_sample = float((got * d2).sum() / N)
    # the scheme's exact law: each molecule is an independent walker with P = I + tau Q
    nbr, vol, area, dist, g = oracle.geometry(verts, tets)
    rows, cols, vals = [], [], []
    for f in range(4):
        ok = nbr[:, f] >= 0
        rows.append(np.nonzero(ok)[0])
        cols.append(nbr[ok, f])
        vals.append(tau * D * g[ok, f])
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    leave = np.bincount(rows, weights=vals, minlength=nt)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(nt, nt)) + sp.diags(1.0 - leave)
    p = np.zeros(nt)
    p[i0] = 1.0
    PT = P.T.tocsr()
    for _ in range(K):
        p = PT @ p
    msd_exact = float(p @ d2)
    var = float(p @ d2 ** 2) - msd_exact ** 2
    se = math.sqrt(var / N)
    assert abs(msd_sample - msd_exact) < 4 * se, (msd_sample, msd_exact, se)
    rel = msd_exact / (6 * D * t) - 1.0
    print(f"MSD at t = {t:.3g} s: exact scheme {msd_exact:.4g} m^2, 6Dt {6 * D * t:.4g} m^2 ({100 * rel:+.1f} %)")
    assert abs(rel) < 0.10
    # and the sample itself against the physics, with its sampling error
    assert abs(msd_sample / (6 * D * t) - 1.0) < 0.10 + 4 * se / (6 * D * t)
