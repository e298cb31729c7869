"""The seeded input generators: shapes, determinism and the stated distributions."""
import numpy as np

import workloads


def test_plain_small_shape_and_determinism():
    a = workloads.plain_small(0)
    b = workloads.plain_small(0)
    c = workloads.plain_small(1)
    assert a.V.shape == (256, 512) and a.W.shape == (256, 16) and a.H.shape == (16, 512)
    for x in (a.V, a.W, a.H):
        assert x.dtype == np.float32 and x.flags.c_contiguous
    np.testing.assert_array_equal(a.V, b.V)
    np.testing.assert_array_equal(a.W, b.W)
    assert not np.array_equal(a.V, c.V)
    assert np.all(a.V == np.round(a.V)) and a.V.min() >= 0          # Poisson counts
    assert 0.1 <= a.W.min() and a.W.max() <= 1.0                     # U(0.1, 1) start
    assert 0.1 <= a.H.min() and a.H.max() <= 1.0


def test_custom_mean_and_exact():
    p = workloads.custom(64, 96, 8, seed=3, shape=0.3, mean=2.0)
    assert abs(p.meta["mean_V"] - 2.0) < 0.2
    e = workloads.custom(32, 40, 4, seed=1, noise="exact")
    np.testing.assert_allclose(e.V, e.W0.astype(np.float64) @ e.H0, rtol=1e-5)


def test_plain_large_recipe_small_slice():
    p = workloads.plain_large(0, N=256, T=512, R=128)
    assert abs(p.meta["mean_V"] - 2.0) < 0.1
    assert 0.0 < p.meta["zero_fraction"] < 1.0


def test_batched_shapes():
    shapes = workloads.batched_shapes(512, 0)
    assert len(shapes) == 512
    N, T, R = (np.array(x) for x in zip(*shapes))
    assert N.min() >= 64 and N.max() <= 2048
    assert T.min() >= 128 and T.max() <= 8192
    assert set(np.unique(R)) <= {8, 16, 32, 64}


def test_sparse_generators_shape_density_and_csr():
    import numpy as np
    for fn, (N, T, dens) in ((workloads.sparse_tdt2, (36771, 10212, 0.0035)),
                             (workloads.sparse_newsgroup, (61188, 18774, 0.002))):
        sp = fn(0)
        assert (sp.N, sp.T) == (N, T)
        assert abs(sp.nnz / (N * T) - dens) < 0.1 * dens
        assert sp.row_ptr[0] == 0 and sp.row_ptr[-1] == sp.nnz
        assert np.all(np.diff(sp.row_ptr) >= 0)
        assert sp.col_idx.min() >= 0 and sp.col_idx.max() < T
        assert np.all(sp.vals >= 1)
    a, b = workloads.sparse_custom(50, 70, 4, 0.1, seed=2), workloads.sparse_custom(50, 70, 4, 0.1, seed=2)
    assert np.array_equal(a.col_idx, b.col_idx) and np.array_equal(a.vals, b.vals)
