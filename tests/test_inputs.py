"""Structure of the seeded synthetic generators (no solver arithmetic)."""
import numpy as np
import pytest

from paper_1602_04386_gb300 import inputs


def check_csr(g):
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.nnz and np.all(np.diff(g.rowptr) >= 0)
    A = {}
    for i in range(g.n):
        cs = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(cs) > 0) and i not in cs
        for j, w in zip(cs, g.w[g.rowptr[i]:g.rowptr[i + 1]]):
            A[(i, int(j))] = w
    for (i, j), w in A.items():
        assert A[(j, i)] == w and w > 0


def connected(g):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    a = sp.csr_matrix((np.ones(g.nnz), g.col, g.rowptr), shape=(g.n, g.n))
    return connected_components(a, directed=False)[0] == 1


def test_grid_counts_and_weights():
    g = inputs.grid(7, 5, "uniform", seed=3)
    assert g.n == 35 and g.nnz == 2 * (7 * 4 + 6 * 5)
    check_csr(g)
    assert g.w.dtype == np.float32 and g.w.min() >= 0.5 and g.w.max() < 1.5


@pytest.mark.parametrize("scale", [6, 9])
def test_rmat_structure(scale):
    g = inputs.rmat(scale, seed=7)
    check_csr(g)
    assert connected(g) and g.n <= 2 ** scale
    assert g.w.min() >= np.float32(0.1) and g.w.max() < 1.0
    deg = np.diff(g.rowptr)
    assert deg.max() > 3 * deg.mean()  # skewed degrees (a hub of degree > 3x the mean)


def test_knn_structure():
    g = inputs.knn_mixture(3000, seed=5)
    check_csr(g)
    assert connected(g)
    deg = np.diff(g.rowptr)
    assert deg.min() >= 1 and np.median(deg) >= 10
    assert g.w.max() <= 1.0


def test_batch_mix_alternates_families():
    gs = inputs.batch_mix(6, scale_range=(6, 8), side_range=(5, 9))
    assert [g.name.startswith("grid") for g in gs] == [True, False] * 3
    for g in gs:
        check_csr(g)
        assert connected(g)


def test_serving_pool_sizes_and_seeds():
    """The serving pool: point counts log-spaced between nmin and nmax, graph i
    drawn with seed + i (the same graph as knn_mixture with that seed), each
    one connected (its largest component kept) and symmetric."""
    pool = inputs.serving_pool(5, 200, 3200, seed=77)
    assert len(pool) == 5
    want = np.exp(np.linspace(np.log(200), np.log(3200), 5)).round().astype(np.int64)
    assert list(want) == [200, 400, 800, 1600, 3200]
    for i, (g, npts) in enumerate(zip(pool, want)):
        assert npts // 8 <= g.n <= npts  # the largest component: at least one of the 8 clusters
        ref = inputs.knn_mixture(int(npts), seed=77 + i)
        assert g.n == ref.n and np.array_equal(g.col, ref.col) and np.array_equal(g.w, ref.w)
        W = g.dense()
        assert np.array_equal(W, W.T) and (W.diagonal() == 0).all()
        seen = np.zeros(g.n, bool)  # connected: a traversal from vertex 0 reaches all
        stack = [0]
        seen[0] = True
        while stack:
            v = stack.pop()
            for u in g.col[g.rowptr[v]:g.rowptr[v + 1]]:
                if not seen[u]:
                    seen[u] = True
                    stack.append(int(u))
        assert seen.all()
