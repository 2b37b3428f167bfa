"""Spectral partitioning by recursive Fiedler bisection (fiedler_partition),
the application of the Introduction, against the same bisection driven on the
host with the oracle's Fiedler vectors, and against the known components of
a Gaussian-mixture kNN graph.

Bars: labels equal to the oracle-driven bisection's on all but 0.1% of the
vertices (a vertex whose Fiedler entry is near zero may land on either side);
disconnected parts split along their components exactly; cluster recovery on
the 8-component mixture measured by the adjusted Rand index."""
import numpy as np
import pytest

import oracle
from paper_1602_04386_gb300 import inputs

pytestmark = pytest.mark.gpu

fiedler = pytest.importorskip("paper_1602_04386_gb300.fiedler")
torch = pytest.importorskip("torch")

OPTS = dict(refine=1, refine_tol=1e-6)


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    fiedler.load()


def induced(g, verts):
    """Induced subgraph of the ascending vertex list verts (CSR, entries in the
    parent's order)."""
    pos = np.full(g.n, -1, np.int64)
    pos[verts] = np.arange(len(verts))
    rows, cols, ws = [], [], []
    for i, v in enumerate(verts):
        c = g.col[g.rowptr[v]:g.rowptr[v + 1]]
        w = g.w[g.rowptr[v]:g.rowptr[v + 1]]
        keep = pos[c] >= 0
        rows.append(np.full(keep.sum(), i))
        cols.append(pos[c[keep]])
        ws.append(w[keep])
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    rp = np.zeros(len(verts) + 1, np.int32)
    np.add.at(rp, r + 1, 1)
    return inputs.CSR(len(verts), np.cumsum(rp).astype(np.int32), np.concatenate(cols).astype(np.int32),
                      np.concatenate(ws).astype(g.w.dtype))


def components_lowest_first(h):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    A = sp.csr_matrix((np.ones(len(h.col)), h.col, h.rowptr), shape=(h.n, h.n))
    _, comp = connected_components(A, directed=False)
    return comp != comp[0]


def reference_bisection(g, parts, **kw):
    """The bisection rule of fiedler_partition with the oracle's vectors."""
    lab = np.zeros(g.n, np.int32)
    sizes = [g.n]
    while len(sizes) < parts:
        cand = [k for k in range(len(sizes)) if sizes[k] >= 2]
        if not cand:
            break
        pick = max(cand, key=lambda k: (sizes[k], -k))
        verts = np.flatnonzero(lab == pick)
        h = induced(g, verts)
        r = oracle.solve(h, **kw)
        if r.status == oracle.EDISCONNECTED:
            side = components_lowest_first(h)
        else:
            assert r.status == 0
            side = r.x(h.n) < 0
        newp = len(sizes)
        lab[verts[side]] = newp
        sizes[pick] -= int(side.sum())
        sizes.append(int(side.sum()))
    return lab


def ari(a, b):
    """Adjusted Rand index of two labelings."""
    from math import comb
    ua, ia = np.unique(a, return_inverse=True)
    ub, ib = np.unique(b, return_inverse=True)
    M = np.zeros((len(ua), len(ub)), np.int64)
    np.add.at(M, (ia, ib), 1)
    s = sum(comb(int(x), 2) for x in M.ravel())
    sa = sum(comb(int(x), 2) for x in M.sum(1))
    sb = sum(comb(int(x), 2) for x in M.sum(0))
    n2 = comb(len(a), 2)
    exp = sa * sb / n2
    return (s - exp) / (0.5 * (sa + sb) - exp)


@pytest.mark.parametrize("precision", [0, 1])
def test_partition_equals_oracle_driven_bisection(precision):
    g = inputs.knn_mixture(6000, seed=21)
    with fiedler.Plan(precision=precision, **OPTS) as p:
        lab, info = p.partition(g, 8)
    assert info.parts == 8 and info.solves == 7
    ref = reference_bisection(g, 8, **OPTS)
    assert (lab != ref).mean() <= 1e-3
    assert sorted(np.unique(lab)) == list(range(8))


def test_partition_splits_disconnected_parts_along_components():
    g = inputs.disjoint_union(inputs.disjoint_union(inputs.grid(30, 20, "uniform", seed=1), inputs.path(50)),
                              inputs.grid(12, 9))
    with fiedler.Plan(**OPTS) as p:
        lab2, info2 = p.partition(g, 2)
        lab3, info3 = p.partition(g, 3)
    # first split: the component of vertex 0 (the 30 x 20 grid) against the rest
    assert info2.parts == 2 and info2.component_splits == 1
    assert np.array_equal(lab2, np.concatenate([np.zeros(600), np.ones(158)]).astype(np.int32))
    # second split: the largest part, the grid, by its Fiedler vector's sign
    assert info3.parts == 3 and info3.component_splits == 1
    assert np.array_equal(lab3, reference_bisection(g, 3, **OPTS))


def test_partition_recovers_mixture_clusters():
    """Config 3's generator (8 isotropic Gaussians, means uniform in [0,10]^2,
    sigma 0.5) at 20,000 points: the 8-way recursive bisection recovers the
    mixture components (ARI against the generating labels)."""
    g, truth = inputs.knn_mixture(20000, return_labels=True)
    with fiedler.Plan(**OPTS) as p:
        lab, info = p.partition(g, 8, on_device=False)
    assert info.parts == 8
    score = ari(lab, truth)
    ref = reference_bisection(g, 8, **OPTS)
    assert abs(score - ari(ref, truth)) <= 0.01
    assert score >= ARI_MIN


ARI_MIN = 0.6  # the host-side bisection reaches 0.68 on this graph
