"""Statistical helpers for the tests (scipy only)."""
import numpy as np
from scipy import stats


def chi2_pvalue(observed_samples, pmf_support, pmf, min_expected=5.0):
    """Chi-square goodness of fit of integer samples against a pmf given on
    `pmf_support`; bins with small expected counts are merged into their
    neighbour. Returns the p-value."""
    observed_samples = np.asarray(observed_samples)
    n = observed_samples.size
    support = np.asarray(pmf_support)
    pmf = np.asarray(pmf, dtype=np.float64)
    pmf = pmf / pmf.sum()
    obs = np.array([(observed_samples == v).sum() for v in support], dtype=np.float64)
    assert obs.sum() == n, "samples outside the support"
    exp = pmf * n
    # merge bins from the low end upward, then the remainder into the last kept bin
    ob, eb = [], []
    acc_o = acc_e = 0.0
    for o, e in zip(obs, exp):
        acc_o += o
        acc_e += e
        if acc_e >= min_expected:
            ob.append(acc_o)
            eb.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0 or acc_o > 0:
        if eb:
            ob[-1] += acc_o
            eb[-1] += acc_e
        else:
            ob.append(acc_o)
            eb.append(acc_e)
    ob, eb = np.array(ob), np.array(eb)
    if len(ob) < 2:
        return 1.0
    return float(stats.chisquare(ob, eb).pvalue)


def chi2_table_pvalue(obs_counts, exp_probs, min_expected=5.0):
    """Chi-square of a table of category counts against probabilities."""
    obs_counts = np.asarray(obs_counts, np.float64)
    exp = np.asarray(exp_probs, np.float64)
    exp = exp / exp.sum() * obs_counts.sum()
    keep = exp >= min_expected
    o = np.append(obs_counts[keep], obs_counts[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    return float(stats.chisquare(o, e).pvalue)
