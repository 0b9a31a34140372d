"""Seeded input generators (CPU): the large sparse-support generator draws
the family it states."""
import numpy as np

import workloads as W


def test_vectorised_sparse_support_draws_distinct_indices_of_the_stated_family():
    D, d, N, nz = 100, 3, 20000, 10
    s = W.sparse_support_vectorised(3, D, d, N, nz)
    assert s.shape == (N, D) and s.dtype == np.uint16
    assert not s[0].any()                            # the zero index first
    assert np.all((s[1:] != 0).sum(axis=1) == nz)    # exactly nz nonzero components
    assert s.max() == d and s[s != 0].min() == 1      # values in 1..d
    assert len(np.unique(s, axis=0)) == N             # distinct multi-indices
    assert np.array_equal(s, W.sparse_support_vectorised(3, D, d, N, nz))  # seeded


def test_vectorised_sparse_support_uses_every_axis_and_value():
    s = W.sparse_support_vectorised(4, 30, 5, 5000, 3)
    nzr, nzc = np.nonzero(s)
    counts = np.bincount(nzc, minlength=30)
    assert counts.min() > 0.5 * counts.mean()        # axes drawn uniformly
    vals = np.bincount(s[nzr, nzc], minlength=6)[1:]
    assert vals.min() > 0.8 * vals.mean()            # values drawn uniformly
