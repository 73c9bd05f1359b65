"""The seeded stand-ins for the paper's SK instances have the shape and the
distribution the paper states (symmetric, zero diagonal, +/-1 with equal
probability or N(0, 1)), and are reproducible from their seed."""
import numpy as np
from scipy import stats

import synth


def test_pm1_instances_are_symmetric_fair_and_seeded():
    J = synth.sk_pm1(500, 3)
    assert J.dtype == np.float32 and J.shape == (500, 500)
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    off = J[np.triu_indices(500, 1)]
    assert set(np.unique(off)) == {-1.0, 1.0}
    # equal probability: the count of +1 over 124750 pairs within 4 sigma
    n = off.size
    assert abs(np.count_nonzero(off > 0) - n / 2) < 4 * np.sqrt(n / 4)
    assert np.array_equal(J, synth.sk_pm1(500, 3))
    assert not np.array_equal(J, synth.sk_pm1(500, 4))


def test_gaussian_instances_are_symmetric_normal_and_seeded():
    J = synth.sk_gauss(400, 2)
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    off = J[np.triu_indices(400, 1)].astype(np.float64)
    assert stats.kstest(off, "norm").pvalue > 1e-3
    assert abs(off.mean()) < 0.02 and abs(off.std() - 1.0) < 0.02
    assert np.array_equal(J, synth.sk_gauss(400, 2))


def test_batch_sizes_uniform_in_range():
    sizes = synth.batch_sizes(256, 4)
    assert len(sizes) == 256 and min(sizes) >= 100 and max(sizes) <= 2000
    assert synth.batch_sizes(256, 4) == sizes
    big = synth.batch_sizes(20000, 1)
    assert stats.kstest((np.array(big) - 100 + 0.5) / 1901, "uniform").pvalue > 1e-3
