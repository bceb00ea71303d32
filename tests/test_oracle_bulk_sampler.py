"""Pins of the oracle's bit-plane draws: a species with BULK_MIN or more trial
molecules in a tet (Algorithm 1's diffusion operator, binomial leave count
split over the faces) assembles each molecule's 31-bit uniform x from bit
planes instead of taking one word per molecule. x must still be uniform and
independent between molecules, so the face counts of one draw are exactly
Multinomial(M, p_f) with p_f = (T_f - T_{f-1}) / 2^31 and the stay
probability 1 - T_3 / 2^31 (the same law as the one-word-per-molecule path).
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from tests.stats import chi2_pvalue, chi2_table_pvalue

T_TYPICAL = np.array([90_000_000, 310_000_000, 330_000_000, 700_000_000], np.uint32)


def _draws(M, T, n, seed=5, window=3):
    return np.array([oracle.sample_bulk(seed, window, tet, 2, M, T) for tet in range(n)])


@pytest.mark.parametrize("M", [8, 31, 32, 45, 100])
def test_face_counts_are_multinomial(M):
    """Per draw, the moved count is Binomial(M, T_3/2^31); summed over draws,
    the face totals split in proportion to the threshold widths."""
    n = 3000
    d = _draws(M, T_TYPICAL, n)
    p = np.diff(np.concatenate([[0], T_TYPICAL.astype(np.float64)])) / 2**31
    moved = d.sum(axis=1)
    ks = np.arange(M + 1)
    assert chi2_pvalue(moved, ks, stats.binom.pmf(ks, M, p.sum())) > 1e-3
    tot = d.sum(axis=0)
    assert chi2_table_pvalue(np.append(tot, n * M - tot.sum()), np.append(p, 1 - p.sum())) > 1e-3
    # faces of one draw are negatively correlated like a multinomial's
    c01 = np.cov(d[:, 0], d[:, 1])[0, 1]
    assert c01 == pytest.approx(-M * p[0] * p[1], abs=6 * M * np.sqrt(p[0] * p[1]) / np.sqrt(n))


def test_groups_are_independent():
    """M = 64 is two groups of 32 with their own planes: the moved count is
    Binomial(64, p), not twice one group's (which would double its variance)."""
    n, M = 4000, 64
    T = np.array([0, 0, 0, 1_073_741_824], np.uint32)  # p = 1/2 through face 3
    moved = _draws(M, T, n)[:, 3]
    ks = np.arange(M + 1)
    assert chi2_pvalue(moved, ks, stats.binom.pmf(ks, M, 0.5)) > 1e-3
    assert moved.var() == pytest.approx(M * 0.25, rel=0.1)


def test_special_cases():
    full = np.array([2**31] * 4, np.uint32)
    assert np.array_equal(oracle.sample_bulk(1, 0, 7, 0, 40, full), [40, 0, 0, 0])
    none = np.zeros(4, np.uint32)
    assert np.array_equal(oracle.sample_bulk(1, 0, 7, 0, 40, none), [0, 0, 0, 0])
    last = np.array([0, 0, 0, 2**31], np.uint32)
    assert np.array_equal(oracle.sample_bulk(1, 0, 7, 0, 77, last), [0, 0, 0, 77])
    assert np.array_equal(oracle.sample_bulk(1, 0, 7, 0, 0, last), [0, 0, 0, 0])


def test_planes_restated_with_numpy():
    """The draw restated from its definition with the separately pinned
    Philox: group g's block blk is Philox(seed; window low word, tet,
    g << 3 | blk, 4 << 28 | species << 23 | window bits 32..54); plane k is
    word k of the group's blocks; molecule j's x has bit 30 - k = bit j of
    plane k; it goes through the first face with x < T_f."""
    rng = np.random.default_rng(6)
    for _ in range(40):
        seed = int(rng.integers(0, 2**63))
        window = int(rng.integers(0, 2**40))
        tet = int(rng.integers(0, 2**31))
        sp = int(rng.integers(0, 32))
        M = int(rng.integers(oracle.BULK_MIN, 120))
        T = np.sort(rng.integers(0, 2**31 + 1, 4)).astype(np.uint32)
        want = np.zeros(4, np.int64)
        for g in range((M + 31) // 32):
            ctr = np.array([[window & 0xFFFFFFFF, tet, (g << 3) | blk,
                             (4 << 28) | (sp << 23) | ((window >> 32) & 0x7FFFFF)] for blk in range(8)], np.uint32)
            planes = oracle.philox_array(seed, ctr).reshape(-1)
            for j in range(min(32, M - 32 * g)):
                x = 0
                for k in range(31):
                    x |= ((int(planes[k]) >> j) & 1) << (30 - k)
                f = int(np.searchsorted(T.astype(np.int64), x, side="right"))
                if f < 4:
                    want[f] += 1
        assert np.array_equal(oracle.sample_bulk(seed, window, tet, sp, M, T), want)
