"""The oracle's pins must catch plausible mistakes anywhere in it.

Each mutant below plants one mistake in a copy of fiedler_oracle.c, made at
test time in a temporary folder: a dropped term, a wrong sign, a wrong index, a
transposed operand or reversed order, a wrong constant.  The copy is compiled
with the oracle's own flags and the pins (test_oracle_pins.py) are run against
it in a child process.  Every mutant must make at least one pin fail.  The
oracle source itself is only read.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fiedler_oracle.c")

# (name, text in the oracle, planted replacement): each text occurs once
MUTANTS = [
    # Def 2.1: the degree is the weighted degree
    ("degree_counts_edges", "      di += w[e];\n", "      di += 1.0;\n"),
    ("ingest_skips_weight_symmetry", "if (found < 0 || w[found] != w[e])", "if (found < 0)"),
    # Alg. 1 (heavy edge coarsening) under the order K
    ("matching_prefers_light_edges", "if (w1 != w2) return w1 > w2;", "if (w1 != w2) return w1 < w2;"),
    ("tie_hash_wrong_endpoint", "h2 = orc_edge_hash(lo2, hi2);", "h2 = orc_edge_hash(lo1, hi2);"),
    ("tie_order_reversed", "if (lo1 != lo2) return lo1 < lo2;", "if (lo1 != lo2) return lo1 > lo2;"),
    ("handshake_not_mutual", "if (v >= 0 && cand[v] == u) mate[u] = v;", "if (v >= 0) mate[u] = v;"),
    ("unmatched_join_first_neighbour", "int v = best_neighbour(L, u, mate, 0, tie_rule);",
     "int v = L->col[L->rowptr[u]];"),
    ("aggregate_leader_is_max", "agg[u] = id[u < mate[u] ? u : mate[u]];", "agg[u] = id[u < mate[u] ? mate[u] : u];"),
    ("paper_hec_takes_lightest", "if (m < 0 || val < best) { best = val; m = L->col[e]; }",
     "if (m < 0 || val > best) { best = val; m = L->col[e]; }"),
    # Alg. 3 setup: L^{i+1} = I L^i I^T
    ("galerkin_drops_duplicate_terms", "      C->w[g] += T[t].w;\n", "      C->w[g] = T[t].w;\n"),
    ("galerkin_column_not_mapped", "int I = agg[i], J = agg[F->col[e]];", "int I = agg[i], J = F->col[e] % nc;"),
    ("coarse_diagonal_halved", "    C->d[I] = s;\n", "    C->d[I] = 0.5 * s;\n"),
    ("coarsening_stops_early", "if (n <= o->coarse_max_n ||", "if (n < 2 * o->coarse_max_n ||"),
    # colouring priority
    ("greedy_colour_order_reversed", "if (x->h != y->h) return x->h > y->h ? -1 : 1;",
     "if (x->h != y->h) return x->h > y->h ? 1 : -1;"),
    ("colour_reuses_neighbour_colour", "while (c < lim && used[c]) c++;", "while (c < lim && used[c] && c < 1) c++;"),
    # Alg. 2 (Gauss-Seidel)
    ("gs_wrong_sign", "s += w[e] * x[col[e]];", "s -= w[e] * x[col[e]];"),
    ("gs_drops_division", "    x[i] = s / d[i];\n", "    x[i] = s;\n"),
    ("gs_ignores_colour_classes", "      if (lv->color[i] == c) order[t++] = i;",
     "      if (c == 0) order[t++] = n - 1 - i;"),
    # Sec. 2: power iteration on sigma I - L, deflation, Rayleigh quotient
    ("laplacian_signless", "s += L->w[e] * (x[i] - x[L->col[e]]);", "s += L->w[e] * (x[i] + x[L->col[e]]);"),
    ("rayleigh_drops_half", "return 0.5 * num / vdot(L->n, x, x);", "return num / vdot(L->n, x, x);"),
    ("no_deflation", "double mu = vsum(n, x) / (double)n;", "double mu = 0.0 * vsum(n, x);"),
    ("shift_too_small", "  return 2.0 * m;\n", "  return 0.5 * m;\n"),
    ("residual_wrong_sign", "double t = tmp[i] - rho * x[i];", "double t = tmp[i] + rho * x[i];"),
    # Alg. 3 refinement and the stop rule of Sec. 3
    ("prolongation_wrong_index", "xf[i] = xc[lv->agg[i]];", "xf[i] = xc[i % r->lv[j + 1].L.n];"),
    ("stop_rule_looser", "if (c > 1.0 - o->pi_cos_tol &&", "if (c > 1.0 - 100.0 * o->pi_cos_tol &&"),
    ("sign_rule_reversed", "if (r->x[imax] < 0.0)", "if (r->x[imax] > 0.0)"),
    # Alg. 1's random order (reading R11)
    ("paper_order_descending", "if (a->key != b->key) return a->key < b->key ? -1 : 1;",
     "if (a->key != b->key) return a->key < b->key ? 1 : -1;"),
    ("paper_order_level_seed", "o->seed + (uint64_t)(r->nlevels - 1)", "o->seed + (uint64_t)r->nlevels"),
    # finest-level Krylov refinement (reading R12)
    ("lobpcg_preconditioner_inverted", "for (int i = 0; i < n; i++) w[i] /= L->d[i];",
     "for (int i = 0; i < n; i++) w[i] *= L->d[i];"),
    ("lobpcg_keeps_constant_in_w", "for (int i = 0; i < n; i++) w[i] -= mw;",
     "for (int i = 0; i < n; i++) w[i] -= 0.0 * mw;"),
    ("lobpcg_largest_ritz_vector", "for (int i = 0; i < m; i++) y += Rinv[i][a] * V[i * m + 0];",
     "for (int i = 0; i < m; i++) y += Rinv[i][a] * V[i * m + (m - 1)];"),
    ("lobpcg_stop_rule_absolute", "sqrt(rr) <= o->refine_tol * theta * sqrt(vdot(n, x, x))",
     "sqrt(rr) <= o->refine_tol * sqrt(vdot(n, x, x))"),
    ("lobpcg_stall_rule_loose", "if (k == 0 || theta < theta_best) {",
     "if (k == 0 || theta < theta_best * (1.0 - 1e-3)) {"),
    ("vcycle_restricts_rhs_not_residual", "bc[lv->agg[i]] += b[i] - t[i];", "bc[lv->agg[i]] += b[i];"),
    ("vcycle_post_sweep_forward", "for (int a = 0, z = n - 1; a < z; a++, z--)",
     "for (int a = 0, z = n - 1; a < 0; a++, z--)"),
    ("vcycle_coarse_mean_kept", "    for (int i = 0; i < n; i++) e[i] -= mu;\n", "    for (int i = 0; i < n; i++) e[i] -= 0.0 * mu;\n"),
    ("vcycle_prolongation_wrong_level", "for (int i = 0; i < n; i++) e[i] += ec[lv->agg[i]];",
     "for (int i = 0; i < n; i++) e[i] += ec[i % nc];"),
    ("lanczos_alpha_halved", "      al[j] = vdot(n, q, u);\n", "      al[j] = 0.5 * vdot(n, q, u);\n"),
    ("lanczos_largest_ritz_vector", "y += V[t * kk + 0] * Q[(size_t)t * n + i];",
     "y += V[t * kk + (kk - 1)] * Q[(size_t)t * n + i];"),
    ("lanczos_estimate_wrong_entry", "fabs(V[(kk - 1) * kk + 0])", "fabs(V[0 * kk + 0])"),
    # truth references and generators used by the pins themselves
    ("jacobi_rotation_sign", "A[k * n + p] = c * akp - s * akq;", "A[k * n + p] = c * akp + s * akq;"),
    ("splitmix_constant", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 27)) * 0x94D049BB133111EFULL;"),
    ("uniform_wrong_bits", "(oracle_splitmix64(s, k) >> 11)", "(oracle_splitmix64(s, k) >> 12)"),
]


def _run_mutant(tmp, idx, name, find, repl, src):
    d = os.path.join(tmp, f"m{idx:02d}")
    os.makedirs(d)
    c = os.path.join(d, "fiedler_oracle.c")
    with open(c, "w") as f:
        f.write(src.replace(find, repl))
    so = os.path.join(d, "liboracle.so")
    cc = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, c, "-lm"],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        return name, "does not compile: " + cc.stderr[-300:]
    env = dict(os.environ, ORACLE_LIB=so, PYTHONDONTWRITEBYTECODE="1")
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                            "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return name, "killed (pins time out)"
    if r.returncode == 0:
        return name, "survived"
    return name, "killed"


def test_every_mutant_text_occurs_once():
    src = open(SRC).read()
    for name, find, repl in MUTANTS:
        assert src.count(find) == 1, name
        assert find != repl, name


def test_pins_kill_every_planted_mistake():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    src = open(SRC).read()
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")
    try:
        workers = max(1, min(8, (os.cpu_count() or 2) // 2))
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            futs = [ex.submit(_run_mutant, tmp, i, name, find, repl, src)
                    for i, (name, find, repl) in enumerate(MUTANTS)]
            results = [f.result() for f in futs]
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    bad = [(n, v) for n, v in results if not v.startswith("killed")]
    assert not bad, bad
