"""The seeded input generators (no arithmetic of the method): the served job
stream has the stated law and every generator is reproducible from its seed."""
import numpy as np

from paper_1610_02258_gb300 import inputs as I


def test_served_job_stream_law():
    """Poisson arrivals at 50 jobs/s (exponential gaps, mean 20 ms), generators
    1-3 about equally often, sizes snapped to log-spaced buckets in [2k, 1M],
    t_end log-uniform in [1, 100] ms, distinct seeds."""
    jobs = I.served_jobs(4000, rate=50.0, seed=21)
    t = np.array([j.arrival for j in jobs])
    gaps = np.diff(t)
    assert t[0] == 0.0 and np.all(gaps >= 0)
    assert abs(gaps.mean() - 0.02) < 4 * 0.02 / np.sqrt(gaps.size)
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.1  # exponential: CV = 1
    kinds = np.bincount([j.kind for j in jobs], minlength=4)[1:]
    assert kinds.min() > 0.3 * len(jobs)
    sizes = np.array([j.size for j in jobs])
    assert set(np.unique(sizes)) <= set(I.SIZE_BUCKETS.tolist())
    assert sizes.min() >= 2000 and sizes.max() <= 1_000_000
    lt = np.log([j.t_end for j in jobs])
    assert lt.min() >= np.log(1e-3) and lt.max() <= np.log(100e-3)
    assert abs(lt.mean() - 0.5 * (np.log(1e-3) + np.log(100e-3))) < 0.1
    assert len({j.seed for j in jobs}) == len(jobs)


def test_generators_are_reproducible():
    for make in (lambda: I.config1(), lambda: I.config2(nx=3), lambda: I.config3(h=0.6e-6)):
        a, b = make(), make()
        assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tets, b.tets)
        assert np.array_equal(a.counts, b.counts)
        assert np.array_equal(a.model.k, b.model.k) and np.array_equal(a.model.diff, b.model.diff)
    sizes = I.batch_sizes(256)
    assert np.array_equal(sizes, I.batch_sizes(256))
    assert sizes.min() >= 1e4 and sizes.max() <= 3e5
