"""Seeded synthetic graph generators shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the solver: it only produces symmetric CSR
adjacency matrices (int32 row pointers, int32 column indices sorted ascending
within each row, positive weights) from counter-based random streams, so that
the CUDA path and the CPU oracle can be fed the same inputs.

Random numbers come from the splitmix64 generator (S. Vigna, public-domain
reference ``splitmix64.c``): output k (k = 0, 1, ...) of the stream seeded with
``s`` is ``mix64(s + (k + 1) * 0x9E3779B97F4A7C15)``.  A uniform draw in [0, 1)
is ``(output >> 11) * 2**-53``.  Every weight is rounded to float32 so that the
FP32 and FP64 forms of the solver see the same graph.

Workload shapes:
  * unit 2-D 5-point grids (vertex index r*k + c, r < m, c < k);
  * weighted 2-D grids, edges enumerated horizontal (row-major) then vertical,
    weight_e = f32(0.5 + u_e), u_e the e-th uniform draw of the seed's stream;
  * R-MAT graphs (skewed degrees) and Gaussian-mixture k-nearest-neighbour
    graphs (spectral clustering inputs), largest connected component kept;
  * the batched mix (grids and R-MAT graphs of many sizes) and the serving
    pool (kNN graphs of log-spaced sizes);
  * small closed-form families (path, cycle, complete, star) for pins;
  * random sparse graphs for dense-eigensolver pins.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Base seed of the synthetic workloads; config c uses BASE_SEED + c.
BASE_SEED = 20160214


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64(seed: int, k) -> np.ndarray:
    """Outputs k (array) of the splitmix64 stream seeded with ``seed``."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * GAMMA
    return _mix64(state)


def uniform01(seed: int, k) -> np.ndarray:
    """Uniform doubles in [0, 1) from outputs k of the seed's stream."""
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class CSR:
    """Symmetric adjacency matrix in CSR form (no diagonal unless added on purpose)."""

    __slots__ = ("n", "rowptr", "col", "w", "name")

    def __init__(self, n, rowptr, col, w, name=""):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.w = np.ascontiguousarray(w)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def with_dtype(self, dtype) -> "CSR":
        return CSR(self.n, self.rowptr, self.col, self.w.astype(dtype), self.name)

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.col] = self.w
        return a

    def __repr__(self):
        return f"CSR({self.name or '?'}, n={self.n}, nnz={self.nnz}, w={self.w.dtype})"


def csr_from_edges(n, u, v, w, dtype=np.float32, name="") -> CSR:
    """Symmetric CSR from undirected edge lists (each edge listed once, u != v,
    no duplicates).  Columns end up sorted ascending within every row."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=dtype)
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    vals = np.concatenate([w, w])
    order = np.argsort(rows * n + cols)  # keys are distinct: (row, col) order
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals, name)


def grid_edges(m: int, k: int):
    """Edges of the m x k 5-point grid, horizontal (row-major) first, then vertical."""
    r, c = np.meshgrid(np.arange(m, dtype=np.int64), np.arange(k - 1, dtype=np.int64), indexing="ij")
    hu = (r * k + c).ravel()
    hv = hu + 1
    r, c = np.meshgrid(np.arange(m - 1, dtype=np.int64), np.arange(k, dtype=np.int64), indexing="ij")
    vu = (r * k + c).ravel()
    vv = vu + k
    return np.concatenate([hu, vu]), np.concatenate([hv, vv])


def grid(m: int, k: int, weights: str = "unit", seed: int = BASE_SEED, dtype=np.float32) -> CSR:
    """m x k 5-point grid graph; ``weights`` is "unit" or "uniform" (0.5 + U[0,1), rounded to f32)."""
    u, v = grid_edges(m, k)
    if weights == "unit":
        w = np.ones(u.shape[0], dtype=np.float32)
    elif weights == "uniform":
        w = (0.5 + uniform01(seed, np.arange(u.shape[0]))).astype(np.float32)
    else:
        raise ValueError(weights)
    return csr_from_edges(m * k, u, v, w.astype(dtype), dtype=dtype, name=f"grid{m}x{k}-{weights}")


def path(n: int, dtype=np.float32) -> CSR:
    u = np.arange(n - 1)
    return csr_from_edges(n, u, u + 1, np.ones(n - 1), dtype=dtype, name=f"path{n}")


def cycle(n: int, dtype=np.float32) -> CSR:
    u = np.arange(n)
    v = (u + 1) % n
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    return csr_from_edges(n, lo, hi, np.ones(n), dtype=dtype, name=f"cycle{n}")


def complete(n: int, dtype=np.float32) -> CSR:
    iu, ju = np.triu_indices(n, 1)
    return csr_from_edges(n, iu, ju, np.ones(iu.shape[0]), dtype=dtype, name=f"K{n}")


def star(n: int, dtype=np.float32) -> CSR:
    """Vertex 0 joined to vertices 1..n-1."""
    v = np.arange(1, n)
    return csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), v, np.ones(n - 1), dtype=dtype, name=f"star{n}")


def random_connected(n: int, avg_deg: float, seed: int, wlo=0.1, whi=1.0, dtype=np.float32) -> CSR:
    """Random sparse connected graph: a random spanning tree plus random extra edges,
    weights uniform in [wlo, whi) rounded to f32."""
    k = 0
    perm = np.argsort(uniform01(seed, np.arange(n)), kind="stable")
    k += n
    # tree: perm[i] attaches to perm[j], j uniform in [0, i)
    j = (uniform01(seed, k + np.arange(1, n)) * np.arange(1, n)).astype(np.int64)
    k += n
    tu, tv = perm[1:], perm[j]
    m_extra = max(0, int(n * avg_deg / 2) - (n - 1))
    eu = (uniform01(seed, k + np.arange(m_extra)) * n).astype(np.int64)
    k += m_extra
    ev = (uniform01(seed, k + np.arange(m_extra)) * n).astype(np.int64)
    k += m_extra
    u = np.concatenate([tu, eu])
    v = np.concatenate([tv, ev])
    keep = u != v
    lo, hi = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = _distinct(lo * n + hi)
    lo, hi = key // n, key % n
    w = (wlo + (whi - wlo) * uniform01(seed, k + np.arange(lo.shape[0]))).astype(np.float32)
    return csr_from_edges(n, lo, hi, w.astype(dtype), dtype=dtype, name=f"rand{n}-s{seed}")


def disjoint_union(a: CSR, b: CSR) -> CSR:
    """Block-diagonal union of two graphs (b's vertices shifted by a.n)."""
    rowptr = np.concatenate([a.rowptr[:-1], b.rowptr + a.nnz]).astype(np.int32)
    col = np.concatenate([a.col, b.col + a.n]).astype(np.int32)
    w = np.concatenate([a.w, b.w.astype(a.w.dtype)])
    return CSR(a.n + b.n, rowptr, col, w, name=f"{a.name}+{b.name}")


def with_self_loops(g: CSR, rows, weight=1.0) -> CSR:
    """Copy of g with a diagonal entry added on the given rows (self-loops)."""
    rows = set(int(r) for r in rows)
    rp = [0]
    cols, ws = [], []
    for i in range(g.n):
        cs = list(g.col[g.rowptr[i]:g.rowptr[i + 1]])
        vs = list(g.w[g.rowptr[i]:g.rowptr[i + 1]])
        if i in rows:
            pos = int(np.searchsorted(np.asarray(cs, dtype=np.int64), i))
            cs.insert(pos, i)
            vs.insert(pos, weight)
        cols += cs
        ws += vs
        rp.append(len(cols))
    return CSR(g.n, np.asarray(rp), np.asarray(cols), np.asarray(ws, dtype=g.w.dtype), name=g.name + "+loops")


def _distinct(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values of an integer array."""
    s = np.sort(keys)
    return s[np.concatenate(([True], s[1:] != s[:-1]))] if s.size else s


def largest_component(g: CSR, return_kept: bool = False):
    """Induced subgraph on the largest connected component (vertex order kept);
    with return_kept, also the kept original vertex ids."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    a = sp.csr_matrix((np.ones(g.nnz), g.col, g.rowptr), shape=(g.n, g.n))
    k, lab = connected_components(a, directed=False)
    if k == 1:
        return (g, np.arange(g.n)) if return_kept else g
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    new = np.full(g.n, -1, np.int64)
    new[keep] = np.arange(keep.size)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m = (new[rows] >= 0) & (new[g.col] >= 0)
    r, c, w = new[rows[m]], new[g.col[m]], g.w[m]
    rowptr = np.zeros(keep.size + 1, np.int64)
    rowptr[1:] = np.cumsum(np.bincount(r, minlength=keep.size))
    out = CSR(keep.size, rowptr, c, w, name=g.name + "-lcc")
    return (out, keep) if return_kept else out


def rmat(scale: int, edge_factor: int = 8, a=0.57, b=0.19, c=0.19, seed: int = BASE_SEED + 4,
         wlo=0.1, whi=1.0, dtype=np.float32) -> CSR:
    """R-MAT graph: edge_factor * 2^scale draws, each choosing one quadrant per
    bit level with probabilities (a, b, c, 1-a-b-c); symmetrised, duplicates and
    self-loops removed, weights uniform in [wlo, whi) per undirected edge
    (rounded to f32), largest connected component kept.

    Quadrant draws are 16-bit: output k of the seed's stream supplies the draws
    of levels 4k' .. 4k'+3 of one edge as its four 16-bit words (low word
    first), compared with the thresholds round(65536 * (a, a+b, a+b+c))."""
    n = 1 << scale
    m = edge_factor * n
    wpe = (scale + 3) // 4  # 64-bit outputs per edge
    words = splitmix64(seed, np.arange(m * wpe, dtype=np.int64))
    u = words.view(np.uint16).reshape(m, 4 * wpe)[:, :scale]  # little-endian: low word first
    ta, tb, tc = (int(round(65536 * t)) for t in (a, a + b, a + b + c))
    q = (u >= ta).astype(np.uint8) + (u >= tb) + (u >= tc)  # quadrant 0..3
    pw = (1 << np.arange(scale - 1, -1, -1, dtype=np.int64))
    src = ((q >> 1).astype(np.int64) * pw).sum(axis=1)
    dst = ((q & 1).astype(np.int64) * pw).sum(axis=1)
    keep = src != dst
    lo, hi = np.minimum(src[keep], dst[keep]), np.maximum(src[keep], dst[keep])
    key = _distinct(lo * n + hi)
    lo, hi = key // n, key % n
    w = (wlo + (whi - wlo) * uniform01(seed + 1, np.arange(key.size))).astype(np.float32)
    g = csr_from_edges(n, lo, hi, w.astype(dtype), dtype=dtype, name=f"rmat{scale}-s{seed}")
    return largest_component(g)


def knn_mixture(npts: int = 200_000, k: int = 10, clusters: int = 8, sigma: float = 0.5, box: float = 10.0,
                seed: int = BASE_SEED + 3, dtype=np.float32, return_labels: bool = False):
    """Points from a mixture of isotropic Gaussians (point i in component
    i mod clusters, means uniform in [0, box]^2, Box-Muller normals), exact
    k-nearest-neighbour graph symmetrised by union, weights exp(-d^2 / 0.25)
    rounded to f32, largest connected component kept.  With return_labels,
    also the mixture component of every kept vertex."""
    from scipy.spatial import cKDTree
    means = uniform01(seed, np.arange(2 * clusters)).reshape(clusters, 2) * box
    u1 = uniform01(seed + 1, np.arange(npts))
    u2 = uniform01(seed + 2, np.arange(npts))
    u1 = np.maximum(u1, 2.0 ** -53)
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.stack([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)], axis=1)
    pts = means[np.arange(npts) % clusters] + sigma * z
    d, idx = cKDTree(pts).query(pts, k=k + 1)
    src = np.repeat(np.arange(npts, dtype=np.int64), k)
    dst = idx[:, 1:].ravel().astype(np.int64)
    dd = d[:, 1:].ravel()
    keep = src != dst
    lo, hi, dd = np.minimum(src[keep], dst[keep]), np.maximum(src[keep], dst[keep]), dd[keep]
    key = lo * npts + hi
    order = np.argsort(key, kind="stable")
    key, dd = key[order], dd[order]
    first = np.concatenate(([True], key[1:] != key[:-1]))  # first listing of each edge
    key, dd = key[first], dd[first]
    lo, hi = key // npts, key % npts
    w = np.exp(-dd * dd / 0.25).astype(np.float32)
    w = np.maximum(w, np.float32(np.finfo(np.float32).tiny))  # keep every weight positive
    g = csr_from_edges(npts, lo, hi, w.astype(dtype), dtype=dtype, name=f"knn{npts}-s{seed}")
    if not return_labels:
        return largest_component(g)
    g, kept = largest_component(g, return_kept=True)
    return g, (kept % clusters).astype(np.int64)


def batch_mix_item(i: int, seed: int = BASE_SEED + 4, scale_range=(9, 16), side_range=(20, 300)) -> CSR:
    """Graph i of the batched workload: even i a 2-D grid with sides uniform in
    side_range and unit weights, odd i an R-MAT graph with scale uniform in
    scale_range (edge factor 8, weights uniform [0.1, 1)).  The sizes come from
    draws 3i .. 3i+2 of the seed's stream, the R-MAT edges from seed + 1000 + i."""
    u = uniform01(seed, np.arange(3 * i, 3 * i + 3))
    if i % 2 == 0:
        m = side_range[0] + int(u[0] * (side_range[1] - side_range[0] + 1))
        k = side_range[0] + int(u[1] * (side_range[1] - side_range[0] + 1))
        return grid(m, k, "unit")
    s = scale_range[0] + int(u[2] * (scale_range[1] - scale_range[0] + 1))
    return rmat(s, seed=seed + 1000 + i)


def _batch_items(args):
    lo, hi, seed, scale_range, side_range = args
    return [batch_mix_item(i, seed, scale_range, side_range) for i in range(lo, hi)]


def _batch_items_at(args):
    idx, seed, scale_range, side_range = args
    return [batch_mix_item(i, seed, scale_range, side_range) for i in idx]


def batch_mix(count: int = 4096, seed: int = BASE_SEED + 4, scale_range=(9, 16), side_range=(20, 300),
              procs: int = 1, indices=None):
    """The batched workload: graphs batch_mix_item(0 .. count-1), or the graphs
    of the given global indices (one rank's share).  With procs > 1 they are
    generated by that many worker processes (started with 'spawn', so this is
    safe after CUDA has been initialised in the caller)."""
    if indices is not None:
        idx = list(indices)
        if procs <= 1 or len(idx) < 64:
            return [batch_mix_item(i, seed, scale_range, side_range) for i in idx]
        import concurrent.futures as cf
        import multiprocessing as mp
        step = max(1, len(idx) // (8 * procs))
        parts = [(idx[k:k + step], seed, scale_range, side_range) for k in range(0, len(idx), step)]
        with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
            out = []
            for part in ex.map(_batch_items_at, parts):
                out.extend(part)
        return out
    if procs <= 1 or count < 64:
        return [batch_mix_item(i, seed, scale_range, side_range) for i in range(count)]
    import concurrent.futures as cf
    import multiprocessing as mp
    step = max(1, count // (8 * procs))
    jobs = [(lo, min(count, lo + step), seed, scale_range, side_range) for lo in range(0, count, step)]
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        out = []
        for part in ex.map(_batch_items, jobs):
            out.extend(part)
    return out


def _knn_item(args):
    npts, seed = args
    return knn_mixture(int(npts), seed=seed)


def serving_pool(count: int = 24, nmin: float = 1e3, nmax: float = 2e6, seed: int = BASE_SEED + 5, procs: int = 1):
    """Graphs for the serving workload: Gaussian-mixture kNN graphs (as
    knn_mixture) with point counts log-spaced from nmin to nmax, graph i
    drawn with seed + i.  Requests that pick one of them uniformly at random
    have sizes distributed log-uniformly between nmin and nmax (to the pool's
    resolution)."""
    sizes = np.exp(np.linspace(np.log(nmin), np.log(nmax), count)).round().astype(np.int64)
    jobs = [(int(sz), seed + i) for i, sz in enumerate(sizes)]
    if procs <= 1:
        return [_knn_item(j) for j in jobs]
    import concurrent.futures as cf
    import multiprocessing as mp
    # largest first, so that the longest jobs start early
    order = sorted(range(count), key=lambda i: -sizes[i])
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        res = dict(zip(order, ex.map(_knn_item, [jobs[i] for i in order])))
    return [res[i] for i in range(count)]
