"""Pins of the CPU oracle against facts fixed outside it: published generator
outputs, hand-worked fixtures, closed-form spectra, LAPACK, brute force and the
literal Galerkin product.  No GPU needed."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_1602_04386_gb300 import inputs


# --------------------------------------------------------------------------
# random streams

def test_splitmix64_known_answers():
    for seed, k, out in read_golden("splitmix64.txt"):
        expect = int(out, 0)
        assert oracle.splitmix64(int(seed), int(k)) == expect
        assert int(inputs.splitmix64(int(seed), [int(k)])[0]) == expect


def test_uniform01_is_top_53_bits():
    for k in range(5):
        u = oracle.uniform01(7, k)
        assert u == (oracle.splitmix64(7, k) >> 11) * 2.0 ** -53
        assert 0.0 <= u < 1.0
        assert u == inputs.uniform01(7, [k])[0]


# --------------------------------------------------------------------------
# helpers (independent of the oracle)

def six_vertex_graph():
    rows = [r for r in read_golden("hec_six_vertex.txt") if r[0] == "edges"]
    u = [int(r[1]) for r in rows]
    v = [int(r[2]) for r in rows]
    w = [float(r[3]) for r in rows]
    return inputs.csr_from_edges(6, u, v, w)


def golden_field(name, key):
    return [r[1:] for r in read_golden(name) if r[0] == key]


def laplacian_dense(g):
    W = g.dense()
    return np.diag(W.sum(1)) - W


def edge_hash_py(a, b):
    lo, hi = min(a, b), max(a, b)
    return int(inputs.splitmix64((lo << 32) | hi, [0])[0])


def key_py(w, a, b, tie_rule):
    """Sort key realising the order K(e) = (w desc, h asc, min asc, max asc)."""
    lo, hi = min(a, b), max(a, b)
    h = edge_hash_py(a, b) if tie_rule == 0 else 0
    return (-w, h, lo, hi)


def edges_of(g):
    out = []
    for i in range(g.n):
        for e in range(g.rowptr[i], g.rowptr[i + 1]):
            j = int(g.col[e])
            if j > i:
                out.append((float(g.w[e]), i, j))
    return out


GRAPHS = [
    lambda: inputs.grid(9, 7, "unit"),
    lambda: inputs.grid(12, 10, "uniform", seed=3),
    lambda: inputs.random_connected(120, 5.0, seed=11),
    lambda: inputs.random_connected(60, 3.0, seed=5),
    lambda: inputs.star(17),
    lambda: inputs.complete(9),
    lambda: inputs.path(31),
]


# --------------------------------------------------------------------------
# heavy-edge coarsening (Alg. 1)

def test_hec_golden_six_vertex():
    g = six_vertex_graph()
    mate_expect = [int(t) for t in golden_field("hec_six_vertex.txt", "mate")[0]]
    agg_expect = [int(t) for t in golden_field("hec_six_vertex.txt", "agg")[0]]
    for mode in (oracle.HEC_HANDSHAKE, oracle.HEC_GREEDY):
        for tie in (oracle.TIE_HASHED, oracle.TIE_INDEX):
            mate, rounds = oracle.match(g, mode, tie)
            assert list(mate) == mate_expect
            if mode == oracle.HEC_HANDSHAKE:
                assert rounds == int(golden_field("hec_six_vertex.txt", "handshake_rounds")[0][0])
            agg, nc = oracle.aggregate(g, mate, tie)
            assert list(agg) == agg_expect and nc == 2
    crow, ccol, cw, cd = oracle.galerkin(g, np.array(agg_expect), 2)
    assert list(crow) == [0, 1, 2] and list(ccol) == [1, 0]
    expect = {(int(a), int(b)): float(c) for a, b, c in golden_field("hec_six_vertex.txt", "coarse_row")}
    assert cw[0] == expect[(0, 1)] and cw[1] == expect[(1, 0)]
    assert list(cd) == [1.5, 1.5]
    perms = golden_field("hec_six_vertex.txt", "paper_perm")
    aggs = golden_field("hec_six_vertex.txt", "paper_agg")
    for p, a in zip(perms, aggs):
        agg_p, nc_p = oracle.hec_paper(g, perm=np.array([int(t) for t in p]))
        assert list(agg_p) == [int(t) for t in a]
        assert nc_p == max(int(t) for t in a) + 1


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("tie", [oracle.TIE_HASHED, oracle.TIE_INDEX])
def test_matching_is_greedy_under_K(gi, tie):
    """The handshake rounds and the sorted greedy scan give the same matching,
    and that matching is the greedy matching of the order K checked by brute
    force: every unmatched edge has a matched neighbouring edge earlier in K."""
    g = GRAPHS[gi]()
    m1, rounds = oracle.match(g, oracle.HEC_HANDSHAKE, tie)
    m2, _ = oracle.match(g, oracle.HEC_GREEDY, tie)
    assert np.array_equal(m1, m2)
    mate = m1
    E = edges_of(g)
    keys = {(a, b): key_py(w, a, b, tie) for w, a, b in E}
    matched = {(min(a, b), max(a, b)) for a, b in enumerate(mate) if b >= 0}
    for a, b in enumerate(mate):
        if b >= 0:
            assert mate[b] == a and (min(a, b), max(a, b)) in keys
    for (a, b), k in keys.items():
        if (a, b) in matched:
            continue
        blockers = [e for e in matched if (a in e or b in e) and keys[e] < k]
        assert blockers, f"edge {(a, b)} could have been matched greedily"
    # maximal: no edge with both ends free
    for w, a, b in E:
        assert mate[a] >= 0 or mate[b] >= 0


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_aggregation_rule(gi):
    g = GRAPHS[gi]()
    mate, _ = oracle.match(g)
    agg, nc = oracle.aggregate(g, mate)
    # leaders in ascending index order get ids 0..nc-1
    leaders = [u for u in range(g.n) if (mate[u] >= 0 and u < mate[u]) or
               (mate[u] < 0 and g.rowptr[u + 1] == g.rowptr[u])]
    assert nc == len(leaders)
    for k, u in enumerate(leaders):
        assert agg[u] == k
    for u in range(g.n):
        if mate[u] >= 0:
            assert agg[u] == agg[mate[u]]
        elif g.rowptr[u + 1] > g.rowptr[u]:
            nb = [(key_py(float(g.w[e]), u, int(g.col[e]), 0), int(g.col[e]))
                  for e in range(g.rowptr[u], g.rowptr[u + 1])]
            best = min(nb)[1]
            assert agg[u] == agg[best]


def test_paper_hec_properties():
    g = inputs.random_connected(80, 4.0, seed=2)
    agg, nc = oracle.hec_paper(g, seed=99)
    assert agg.min() == 0 and agg.max() == nc - 1
    assert len(np.unique(agg)) == nc
    # every aggregate contains a vertex and its heaviest neighbour (lowest index on ties)
    for u in range(g.n):
        cs = g.col[g.rowptr[u]:g.rowptr[u + 1]]
        ws = g.w[g.rowptr[u]:g.rowptr[u + 1]].astype(np.float64)
        m = int(cs[np.flatnonzero(ws == ws.max())[0]])
        # u is either paired with / joined to its heaviest neighbour, or was
        # taken as the heaviest neighbour of someone earlier
        partners = [v for v in range(g.n) if agg[v] == agg[u] and v != u]
        assert partners
        assert agg[m] == agg[u] or any(
            int(g.col[g.rowptr[v]:g.rowptr[v + 1]][np.argmax(g.w[g.rowptr[v]:g.rowptr[v + 1]])]) == u
            for v in partners)


# --------------------------------------------------------------------------
# Galerkin coarse operator (Alg. 3)

@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_galerkin_matches_literal_product(gi):
    g = GRAPHS[gi]()
    mate, _ = oracle.match(g)
    agg, nc = oracle.aggregate(g, mate)
    crow, ccol, cw, cd = oracle.galerkin(g, agg, nc)
    P = np.zeros((g.n, nc))
    P[np.arange(g.n), agg] = 1.0
    Lc_lit = P.T @ laplacian_dense(g) @ P       # I L I^T with I = P^T
    Lc = np.diag(cd)
    rows = np.repeat(np.arange(nc), np.diff(crow))
    Lc[rows, ccol] -= cw
    assert np.allclose(Lc, Lc_lit, rtol=0, atol=1e-12 * np.abs(Lc_lit).max())
    # sorted columns, no diagonal, symmetric, zero row sums
    for I in range(nc):
        cs = ccol[crow[I]:crow[I + 1]]
        assert np.all(np.diff(cs) > 0) and I not in cs
    assert np.allclose(Lc, Lc.T, atol=0)
    assert np.allclose(Lc.sum(1), 0, atol=1e-12 * np.abs(cd).max())
    # cross-aggregate weight is conserved
    W = g.dense()
    cross = W[agg[:, None] != agg[None, :]].sum()
    assert np.isclose(cw.sum(), cross, rtol=1e-13)


@pytest.mark.parametrize("make,levels", [
    (lambda: inputs.path(25), 1),     # n = 25 is not coarsened (Alg. 3: while n > 25)
    (lambda: inputs.path(26), 2),     # n = 26 is, once
    (lambda: inputs.random_connected(45, 4.0, seed=2), None),
    (lambda: inputs.grid(7, 6, "uniform", seed=4), None),
])
def test_coarsening_stops_at_25_vertices(make, levels):
    """Alg. 3 coarsens while a level has more than 25 vertices: the coarsest
    level has at most 25 and every other level more than 25."""
    g = make()
    lv = oracle.build_hierarchy(g).levels
    assert lv[-1].n <= 25
    assert all(L.n > 25 for L in lv[:-1])
    if levels is not None:
        assert len(lv) == levels


def test_hierarchy_invariants_and_stop_rule():
    g = inputs.grid(40, 30, "uniform", seed=9)
    r = oracle.build_hierarchy(g)
    assert r.status == 0
    lv = r.levels
    assert lv[-1].n <= 25 < lv[-2].n
    for a, b in zip(lv[:-1], lv[1:]):
        assert a.nc == b.n and a.agg is not None
        assert 2 <= b.n <= 0.9 * a.n
    for L in lv:
        rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
        # d equals the row sums in ascending column order (bit for bit)
        for i in range(L.n):
            s = 0.0
            for e in range(L.rowptr[i], L.rowptr[i + 1]):
                s += L.w[e]
            assert s == L.d[i]
        A = np.zeros((L.n, L.n))
        A[rows, L.col] = L.w
        assert np.array_equal(A, A.T)
        assert L.sigma == 2 * L.d.max()


# --------------------------------------------------------------------------
# colouring

@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_coloring_greedy_equals_jp_and_is_valid(gi):
    g = GRAPHS[gi]()
    c1, n1, _ = oracle.color(g, jp=False)
    c2, n2, rounds = oracle.color(g, jp=True)
    assert np.array_equal(c1, c2) and n1 == n2
    prio = [(int(inputs.splitmix64(v, [0])[0]), v) for v in range(g.n)]
    for v in range(g.n):
        nb = g.col[g.rowptr[v]:g.rowptr[v + 1]]
        assert c1[v] not in c1[nb]
        higher = {int(c1[u]) for u in nb if prio[u] > prio[v]}
        smallest = min(set(range(len(nb) + 2)) - higher)
        assert c1[v] == smallest
    assert rounds >= 1 and n1 == c1.max() + 1


# --------------------------------------------------------------------------
# Gauss-Seidel (Alg. 2)

def test_gs_golden_path3():
    rows = {r[0]: [float(t) for t in r[1:]] for r in read_golden("gs_path3.txt")}
    g = inputs.csr_from_edges(3, [0, 1], [1, 2], [1.0, 2.0])
    d = g.dense().sum(1)
    x = oracle.gauss_seidel(g.rowptr, g.col, g.w, d, None, rows["x0"], 1)
    assert np.allclose(x, rows["x1"], rtol=0, atol=1e-16)


@pytest.mark.parametrize("colored", [False, True])
def test_gs_converges_to_linear_solve(colored):
    """Alg. 2 on an SPD, strictly diagonally dominant system (Thm 2.1) converges
    to the LAPACK solution; colour-class order converges to the same point."""
    g = inputs.random_connected(70, 4.0, seed=21)
    W = g.dense()
    d = W.sum(1) + 0.5
    A = np.diag(d) - W
    b = inputs.uniform01(5, np.arange(g.n)) - 0.5
    order = None
    if colored:
        c, nc, _ = oracle.color(g)
        order = np.concatenate([np.flatnonzero(c == k) for k in range(nc)])
    x = oracle.gauss_seidel(g.rowptr, g.col, g.w, d, b, np.zeros(g.n), 400, order)
    xs = np.linalg.solve(A, b)
    assert np.abs(x - xs).max() < 1e-11 * np.abs(xs).max()


def test_smoothing_sweeps_colour_classes_in_order():
    """With colour-class order, a level's sweep visits the classes in
    ascending colour.  No two vertices of a class are adjacent, so the order
    inside a class cannot change a single bit; the level's smoothed vector must
    equal Alg. 2 (pinned above) run with every class shuffled, and differ from a
    lexicographic sweep."""
    g = inputs.grid(12, 10, "uniform", seed=3)
    r = oracle.solve(g, gs_sweeps=1, forced_pi=[0] * 64)  # no power iteration: the sweep alone
    assert r.status == 0
    lv = r.levels
    rng = np.random.default_rng(0)
    differs = False
    for j in range(len(lv) - 1):
        F, Cl = lv[j], lv[j + 1]
        x0 = Cl.x[F.agg].copy()                 # prolongation, then deflation and normalisation
        x0 -= x0.mean()
        x0 /= np.linalg.norm(x0)
        order = np.concatenate([rng.permutation(np.flatnonzero(F.color == k)) for k in range(F.ncolors)])
        x1 = oracle.gauss_seidel(F.rowptr, F.col, F.w, F.d, None, x0, 1, order)
        x1 -= x1.mean()
        x1 /= np.linalg.norm(x1)
        assert np.abs(x1 - F.x).max() < 1e-12, j
        xl = oracle.gauss_seidel(F.rowptr, F.col, F.w, F.d, None, x0, 1)
        xl -= xl.mean()
        xl /= np.linalg.norm(xl)
        differs |= np.abs(xl - F.x).max() > 1e-6
    assert differs


# --------------------------------------------------------------------------
# dense Jacobi eigensolver (truth reference for small graphs)

def test_jacobi_against_lapack_and_closed_form():
    rng = inputs.uniform01(77, np.arange(40 * 40)).reshape(40, 40) - 0.5
    A = rng + rng.T
    ev, V, sweeps = oracle.jacobi_eig(A)
    ref = np.linalg.eigvalsh(A)
    assert np.allclose(ev, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(A @ V, V * ev, atol=1e-11)
    assert sweeps < 20
    n = 25
    ev, V, _ = oracle.jacobi_eig(laplacian_dense(inputs.path(n)))
    closed = 2 - 2 * np.cos(np.pi * np.arange(n) / n)
    assert np.allclose(ev, np.sort(closed), atol=1e-13)


# --------------------------------------------------------------------------
# whole method: closed forms, brute force, invariants

def angle(x, v):
    return 1 - abs(x @ v) / (np.linalg.norm(x) * np.linalg.norm(v))


TIGHT = dict(resid_tol=1e-10, pi_max_iters=400000, pi_max_iters_coarsest=400000)


@pytest.mark.parametrize("n", [2, 5, 24, 26, 100])
def test_path_closed_form(n):
    g = inputs.path(n)
    r = oracle.solve(g, **TIGHT)
    assert r.status == 0
    lam = 2 - 2 * np.cos(np.pi / n)
    assert abs(r.lam - lam) <= 1e-9 * lam
    v = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    assert angle(r.x(n), v) < 1e-9


@pytest.mark.parametrize("m,k", [(64, 48), (20, 13), (33, 7)])
def test_grid_closed_form(m, k):
    g = inputs.grid(m, k, "unit")
    r = oracle.solve(g, **TIGHT)
    lam = 2 - 2 * np.cos(np.pi / max(m, k))
    assert abs(r.lam - lam) <= 1e-9 * lam
    rr = np.arange(m * k) // k
    v = np.cos(np.pi * (rr + 0.5) / m)
    assert angle(r.x(m * k), v) < 1e-9
    x = r.x(m * k)
    assert abs(np.linalg.norm(x) - 1) < 1e-14 and r.ortho < 1e-12


def test_config1_paper_stop_rule_values():
    """64x48 unit grid with the paper's stop rule: the result is an
    approximation above lambda_2 (variational bound) within a few percent."""
    g = inputs.grid(64, 48, "unit")
    r = oracle.solve(g)
    lam = 2 - 2 * np.cos(np.pi / 64)
    assert lam <= r.lam < 1.05 * lam
    for L in r.levels:
        if L.pi_iters < (100000 if L is r.levels[-1] else 10000):
            assert L.last_cos > 1 - 1e-6


@pytest.mark.parametrize("n", [7, 30])
def test_cycle_and_complete_eigenvalues(n):
    r = oracle.solve(inputs.cycle(n), **TIGHT)
    assert abs(r.lam - (2 - 2 * np.cos(2 * np.pi / n))) < 1e-9
    r = oracle.solve(inputs.complete(n))
    assert abs(r.lam - n) < 1e-12 * n


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_random_graphs_against_dense_jacobi(seed):
    g = inputs.random_connected(150 + 10 * seed, 4.0, seed=seed)
    ev, V, _ = oracle.jacobi_eig(laplacian_dense(g))
    r = oracle.solve(g, **TIGHT)
    assert abs(r.lam - ev[1]) < 1e-8 * ev[1]
    if ev[2] - ev[1] > 1e-3 * ev[1]:
        assert angle(r.x(g.n), V[:, 1]) < 1e-8
    # default stop rule: Rayleigh quotient above lambda_2 (variational bound)
    r2 = oracle.solve(g)
    assert r2.lam >= ev[1] * (1 - 1e-12)
    # reported residual recomputed independently
    x = r2.x(g.n)
    L = laplacian_dense(g)
    assert np.isclose(np.linalg.norm(L @ x - r2.lam * x), r2.residual, rtol=1e-9)
    assert np.isclose(x @ L @ x, r2.lam, rtol=1e-12)


def test_modes_agree_when_tight():
    g = inputs.grid(30, 21, "uniform", seed=4)
    ev = np.linalg.eigvalsh(laplacian_dense(g))
    for kw in (dict(hec_mode=2), dict(gs_order=0), dict(hec_mode=1, tie_rule=1), dict(gs_sweeps=0),
               dict(coarsest_dense=1)):
        r = oracle.solve(g, **TIGHT, **kw)
        assert r.status == 0
        assert abs(r.lam - ev[1]) < 1e-8 * ev[1], kw


def test_sign_and_normalisation():
    g = inputs.grid(17, 11, "uniform", seed=8)
    r = oracle.solve(g)
    x = r.x(g.n)
    i = int(np.argmax(np.abs(x)))
    assert x[i] > 0
    assert abs(np.linalg.norm(x) - 1) < 1e-14 and abs(x.sum()) < 1e-12


def test_forced_iterations_are_honoured():
    g = inputs.grid(20, 14, "uniform", seed=8)
    r = oracle.solve(g)
    forced = [3] * r.num_levels
    r2 = oracle.solve(g, forced_pi=forced)
    assert r2.pi_iters == forced
    r3 = oracle.solve(g, forced_pi=r.pi_iters)
    assert np.array_equal(r3.x(g.n), r.x(g.n))


# --------------------------------------------------------------------------
# edge cases of the input

def test_two_vertices():
    g = inputs.csr_from_edges(2, [0], [1], [0.75])
    r = oracle.solve(g)
    assert r.status == 0
    assert abs(r.lam - 1.5) < 1e-15
    assert np.allclose(r.x(2), [2 ** -0.5, -(2 ** -0.5)], atol=1e-15)


def test_disconnected_and_invalid_inputs():
    g = inputs.disjoint_union(inputs.grid(10, 8), inputs.path(40))
    assert oracle.solve(g).status == oracle.EDISCONNECTED
    good = inputs.grid(6, 5, "uniform", seed=1)
    bad = inputs.CSR(good.n, good.rowptr, good.col.copy(), good.w.copy())
    bad.w[3] *= 2  # asymmetric
    r = oracle.solve(bad)
    assert r.status == oracle.EINVAL and r.bad_index >= 0
    bad = inputs.CSR(good.n, good.rowptr, good.col.copy(), good.w.copy())
    bad.col[0], bad.col[1] = bad.col[1], bad.col[0]  # unsorted row
    assert oracle.solve(bad).status == oracle.EINVAL
    bad = inputs.CSR(good.n, good.rowptr, good.col.copy(), -good.w)
    assert oracle.solve(bad).status == oracle.EINVAL
    single = inputs.CSR(1, np.array([0, 0]), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert oracle.solve(single).status == oracle.EINVAL


def test_self_loops_are_dropped():
    g = inputs.grid(12, 9, "uniform", seed=2)
    gl = inputs.with_self_loops(g, [0, 5, 50], weight=3.0)
    r1, r2 = oracle.solve(g), oracle.solve(gl)
    assert r1.lam == r2.lam
    assert np.array_equal(r1.x(g.n), r2.x(g.n))


def test_star_graph():
    """Star: lambda_2 = 1 (multiplicity n-2); Gauss-Seidel may annihilate the
    iterate, which the guard must survive."""
    g = inputs.star(40)
    r = oracle.solve(g, **TIGHT)
    assert r.status == 0 and abs(r.lam - 1.0) < 1e-9


# --------------------------------------------------------------------------
# Alg. 1's random order (reading R11) and the finest-level Krylov refinement
# (reading R12: Sec. 4's Krylov smoother)

def test_paper_hec_order_is_sorted_splitmix_keys():
    """Without an explicit order, hec_paper visits the vertices in ascending
    order of splitmix64(seed, v) (ties by v): the same aggregates as the order
    computed here from the published generator; the hierarchy's level l uses
    seed + l."""
    g = inputs.random_connected(120, 4.0, seed=5)
    for seed in (3, 20160214):
        keys = inputs.splitmix64(seed, np.arange(g.n))
        perm = np.lexsort((np.arange(g.n), keys))
        a1, n1 = oracle.hec_paper(g, seed=seed)
        a2, n2 = oracle.hec_paper(g, perm=perm)
        assert n1 == n2 and np.array_equal(a1, a2)
    run = oracle.build_hierarchy(g, hec_mode=oracle.HEC_PAPER, seed=77)
    lv = run.levels
    for l in range(len(lv) - 1):
        h = inputs.CSR(lv[l].n, lv[l].rowptr, lv[l].col, lv[l].w)
        agg, nc = oracle.hec_paper(h, seed=77 + l)
        assert np.array_equal(lv[l].agg, agg) and lv[l].nc == nc


REFINES = [oracle.REFINE_LOBPCG, oracle.REFINE_LANCZOS]
# the LOBPCG preconditioners (reading R13); the Lanczos runs ignore it
PRECONDS = [oracle.PRECOND_DEGREE, oracle.PRECOND_VCYCLE]
RTIGHT = dict(refine_tol=1e-9, refine_max_iters=200000)


@pytest.mark.parametrize("refine", REFINES)
def test_refine_path_and_grid_closed_forms(refine):
    """Refined to a tight residual, lambda_2 and phi_2 of a path and of a
    non-square unit grid match their closed forms."""
    n = 60
    r = oracle.solve(inputs.path(n), refine=refine, **RTIGHT)
    assert r.status == 0 and r.level(0).pi_iters == 0 and r.refine_iters > 0
    lam = 2 - 2 * np.cos(np.pi / n)
    assert abs(r.lam - lam) <= 1e-11 * lam
    v = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    assert angle(r.x(n), v) <= 1e-10
    m, k = 40, 27
    g = inputs.grid(m, k, "unit")
    r = oracle.solve(g, refine=refine, **RTIGHT)
    lam = 2 - 2 * np.cos(np.pi / m)
    assert r.status == 0 and abs(r.lam - lam) <= 1e-11 * lam
    v = np.cos(np.pi * (np.arange(g.n) // k + 0.5) / m)
    assert angle(r.x(g.n), v) <= 1e-10


@pytest.mark.parametrize("refine", REFINES)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_refine_against_dense_jacobi(refine, seed):
    """Random weighted graphs (n <= 200): the refined pair equals the dense
    Jacobi eigenpair; the returned vector's residual, recomputed here, meets
    the stop rule ||L x - theta x|| <= refine_tol theta ||x||."""
    g = inputs.random_connected(170, 4.0, seed=seed)
    ev, V, _ = oracle.jacobi_eig(laplacian_dense(g))
    r = oracle.solve(g, refine=refine, refine_tol=1e-6, refine_max_iters=200000)
    assert r.status == 0 and not r.capped
    x = r.x(g.n)
    Ld = laplacian_dense(g)
    th = x @ Ld @ x
    assert np.linalg.norm(Ld @ x - th * x) <= 1.001e-6 * th
    assert abs(r.lam - ev[1]) <= 1e-10 * ev[1]
    if ev[2] - ev[1] > 1e-3 * ev[1]:
        assert 1 - abs(x @ V[:, 1]) <= 1e-9
    r2 = oracle.solve(g, refine=refine, **RTIGHT)
    assert abs(r2.lam - ev[1]) <= 1e-13 * ev[1]


def test_refine_skewed_degrees():
    """On a skewed-degree R-MAT graph the paper's stop rule leaves lambda_2 far
    off, while both refinements reach the dense eigenvalue."""
    g = inputs.rmat(8, seed=5)
    ev = np.linalg.eigvalsh(laplacian_dense(g))
    paper = oracle.solve(g)
    assert paper.lam > 1.5 * ev[1]
    its = {}
    for refine, pre in ((oracle.REFINE_LOBPCG, oracle.PRECOND_DEGREE), (oracle.REFINE_LOBPCG, oracle.PRECOND_VCYCLE),
                        (oracle.REFINE_LANCZOS, oracle.PRECOND_DEGREE)):
        r = oracle.solve(g, refine=refine, refine_precond=pre, refine_tol=1e-7, refine_max_iters=200000)
        assert r.status == 0 and abs(r.lam - ev[1]) <= 1e-10 * ev[1], refine
        its[(refine, pre)] = r.refine_iters
    # the D^-1 preconditioner evens out the spread of degrees: LOBPCG needs
    # far fewer matvecs than the unpreconditioned Krylov method
    assert its[(oracle.REFINE_LOBPCG, oracle.PRECOND_DEGREE)] * 5 < its[(oracle.REFINE_LANCZOS, 0)]


@pytest.mark.parametrize("refine", REFINES)
def test_refine_forced_count_replays(refine):
    """refine_forced = k runs exactly k matvecs; k = the free run's count gives
    the free run's result bit for bit; one fewer gives a larger Rayleigh
    quotient (the methods lower it monotonically)."""
    g = inputs.grid(33, 19, "uniform", seed=12)
    tol = 1e-5  # reached before the Rayleigh quotient hits its rounding floor
    free = oracle.solve(g, refine=refine, refine_tol=tol, refine_max_iters=200000)
    k = free.refine_iters
    same = oracle.solve(g, refine=refine, refine_tol=tol, refine_forced=k)
    assert same.refine_iters == k and same.lam == free.lam
    assert np.array_equal(same.x(g.n), free.x(g.n))
    Ld = laplacian_dense(g)
    if refine == oracle.REFINE_LOBPCG:
        # the stop rule is tested before every step: the iterate one step
        # earlier does not meet it (its residual, recomputed here, is too big)
        less = oracle.solve(g, refine=refine, refine_tol=tol, refine_forced=k - 1)
        assert less.refine_iters == k - 1 and less.lam > free.lam
    else:
        # the Ritz estimate is tested at the end of each cycle: the cycle
        # before the last one ends above the tolerance, the last one below
        m = 24
        assert k % m == 0 and k > m
        less = oracle.solve(g, refine=refine, refine_tol=tol, refine_forced=k - m)
    for run, ok in ((free, True), (less, False)):
        x = run.x(g.n)
        th = x @ Ld @ x
        assert (np.linalg.norm(Ld @ x - th * x) <= 1.001 * tol * th) == ok


@pytest.mark.parametrize("pre", [0, 1])
def test_lobpcg_stops_at_the_rounding_floor(pre):
    """With a tolerance below reach, LOBPCG ends at the rounding floor (a step
    without p that does not lower the Rayleigh quotient), long before its cap,
    with lambda_2 exact to rounding; replaying its count gives the same bits
    (the restarts without p are part of the step sequence)."""
    g = inputs.grid(33, 19, "uniform", seed=12)
    free = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_precond=pre, refine_tol=1e-15,
                        refine_max_iters=100000)
    assert not free.capped and free.refine_iters < 2000
    ev = np.linalg.eigvalsh(laplacian_dense(g))
    assert abs(free.lam - ev[1]) <= 1e-13 * ev[1]
    again = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_precond=pre, refine_forced=free.refine_iters)
    assert again.lam == free.lam


def test_refine_cap_and_degenerate_start():
    """A cap below the needed count reports capped; on K_n (every vector of
    1-perp an eigenvector) the refinement stops at once with lambda_2 = n."""
    g = inputs.grid(30, 20, "uniform", seed=2)
    r = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_tol=1e-12, refine_max_iters=3)
    assert r.status == 0 and r.capped and r.refine_iters == 3
    for refine in REFINES:
        r = oracle.solve(inputs.complete(12), refine=refine)
        assert r.status == 0 and abs(r.lam - 12) <= 1e-12 * 12
        assert r.refine_iters <= 1


# --------------------------------------------------------------------------
# the V-cycle preconditioner (reading R13)

def _dense_gs(A, d, b, e, order):
    for i in order:
        e[i] = (b[i] + A[i] @ e) / d[i]
    return e


def test_vcycle_two_levels_written_out():
    """On a two-level hierarchy the V-cycle equals its definition written out
    with dense matrices: forward colour sweep, aggregate sums of the residual,
    20 forward sweeps and the mean removed on the coarse level, the correction
    added to the members, backward colour sweep."""
    g = inputs.random_connected(40, 3.0, seed=8)
    run = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_forced=0)
    assert run.num_levels == 2
    f, c = run.level(0), run.level(1)
    A0 = inputs.CSR(f.n, f.rowptr, f.col, f.w).dense()
    A1 = inputs.CSR(c.n, c.rowptr, c.col, c.w).dense()
    o0 = np.lexsort((np.arange(f.n), f.color))
    o1 = np.lexsort((np.arange(c.n), c.color))
    rng = np.random.default_rng(3)
    b = rng.standard_normal(f.n)
    b -= b.mean()
    e = _dense_gs(A0, f.d, b, np.zeros(f.n), o0)
    res = b - (np.diag(f.d) - A0) @ e
    bc = np.zeros(c.n)
    np.add.at(bc, f.agg, res)
    ec = np.zeros(c.n)
    for _ in range(20):
        _dense_gs(A1, c.d, bc, ec, o1)
    ec -= ec.mean()
    e = e + ec[f.agg]
    e = _dense_gs(A0, f.d, b, e, o0[::-1])
    got = run.vcycle(b)
    assert np.allclose(got, e, rtol=1e-12, atol=1e-14)


def test_vcycle_is_a_contracting_approximate_inverse():
    """On a weighted grid one V-cycle removes most of the error of L e = b for
    b orthogonal to 1 (measured against the dense pseudo-inverse solution)."""
    g = inputs.grid(30, 22, "uniform", seed=5)
    run = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_forced=0)
    assert run.num_levels >= 3
    L = laplacian_dense(g)
    rng = np.random.default_rng(1)
    for _ in range(3):
        b = rng.standard_normal(g.n)
        b -= b.mean()
        exact = np.linalg.pinv(L) @ b
        e = run.vcycle(b)
        e -= e.mean()
        assert np.linalg.norm(L @ (e - exact)) < 0.6 * np.linalg.norm(b)


def test_vcycle_preconditioning_cuts_lobpcg_steps_on_grids():
    g = inputs.grid(90, 61, "uniform", seed=4)
    its = {}
    for pre in PRECONDS:
        r = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_precond=pre, refine_tol=1e-6,
                         refine_max_iters=100000)
        assert r.status == 0 and not r.capped
        its[pre] = r.refine_iters
    assert its[oracle.PRECOND_VCYCLE] * 5 < its[oracle.PRECOND_DEGREE]


@pytest.mark.parametrize("pre", PRECONDS)
def test_lobpcg_both_preconditioners_reach_dense_jacobi(pre):
    g = inputs.random_connected(190, 5.0, seed=11)
    ev, V, _ = oracle.jacobi_eig(laplacian_dense(g))
    r = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_precond=pre, refine_tol=1e-8, refine_max_iters=100000)
    assert r.status == 0 and abs(r.lam - ev[1]) <= 1e-12 * ev[1]


@pytest.mark.parametrize("pre", [0, 1])
def test_lobpcg_first_step_written_out(pre):
    """One LOBPCG step from the cascade's start, written out: w = M r with its
    mean removed (M = D^-1 or one V-cycle), r = L x - theta x, then the
    smallest Rayleigh-Ritz pair of span{x, w} (dense generalized eigenproblem),
    the Ritz vector deflated, normalised and sign-normalised."""
    import scipy.linalg as sla
    g = inputs.grid(24, 17, "uniform", seed=6)
    Ld = laplacian_dense(g)
    d = np.diag(Ld)
    r0 = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_precond=pre, refine_forced=0)
    x = r0.x(g.n)
    th = x @ Ld @ x / (x @ x)
    r = Ld @ x - th * x
    w = r / d if pre == 0 else r0.vcycle(r)
    w -= w.mean()
    S = np.stack([x, w], axis=1)
    ev, V = sla.eigh(S.T @ Ld @ S, S.T @ S)
    x1 = S @ V[:, 0]
    x1 -= x1.mean()
    x1 /= np.linalg.norm(x1)
    if x1[np.argmax(np.abs(x1))] < 0:
        x1 = -x1
    r1 = oracle.solve(g, refine=oracle.REFINE_LOBPCG, refine_precond=pre, refine_forced=1)
    assert np.allclose(r1.x(g.n), x1, rtol=0, atol=1e-10)
