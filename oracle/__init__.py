"""CPU oracle of the Gauss-Seidel cascadic multigrid Fiedler solver.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It is a plain,
sequential FP64 C implementation (``fiedler_oracle.c``) of the paper's method
(Def 2.1, Alg. 1-3, the shifted power iteration and Rayleigh quotient of
Sec. 2, the tolerance of Sec. 3), built with gcc and loaded through ctypes.
It shares no code with the CUDA library.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, a dense Jacobi eigensolver checked against LAPACK,
brute force, the literal Galerkin product and hand-worked fixtures.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fiedler_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EDISCONNECTED, EDEGENERATE = 0, -1, -2, -3, -8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Opts(C.Structure):
    _fields_ = [
        ("coarse_max_n", C.c_int),
        ("max_levels", C.c_int),
        ("stall_ratio", C.c_double),
        ("hec_mode", C.c_int),
        ("tie_rule", C.c_int),
        ("gs_order", C.c_int),
        ("gs_sweeps", C.c_int),
        ("pi_max_iters", C.c_int),
        ("pi_max_iters_coarsest", C.c_int),
        ("pi_cos_tol", C.c_double),
        ("resid_tol", C.c_double),
        ("guard", C.c_double),
        ("seed", C.c_uint64),
        ("coarsest_dense", C.c_int),
        ("refine", C.c_int),
        ("refine_max_iters", C.c_int),
        ("refine_tol", C.c_double),
        ("lanczos_basis", C.c_int),
        ("refine_forced", C.c_int),
        ("refine_precond", C.c_int),
    ]


HEC_HANDSHAKE, HEC_GREEDY, HEC_PAPER = 0, 1, 2
TIE_HASHED, TIE_INDEX = 0, 1
GS_LEX, GS_COLORED = 0, 1
REFINE_NONE, REFINE_LOBPCG, REFINE_LANCZOS = 0, 1, 2
PRECOND_DEGREE, PRECOND_VCYCLE = 0, 1


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB names another build of fiedler_oracle.c (the mutation
            # tests load copies with planted mistakes that way)
            path = os.environ.get("ORACLE_LIB") or build()
            L = C.CDLL(path)
            ip, dp, lp = C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_longlong)
            L.oracle_run_create.restype = C.c_void_p
            L.oracle_run_destroy.argtypes = [C.c_void_p]
            L.oracle_default_opts.argtypes = [C.POINTER(Opts)]
            L.oracle_build.argtypes = [C.c_void_p, C.c_int, C.c_longlong, ip, ip, dp, C.POINTER(Opts)]
            L.oracle_solve.argtypes = [C.c_void_p, C.c_int, C.c_longlong, ip, ip, dp, C.POINTER(Opts), ip]
            for f in ("oracle_run_status", "oracle_run_num_levels"):
                getattr(L, f).argtypes = [C.c_void_p]
            L.oracle_run_bad_index.argtypes = [C.c_void_p]
            L.oracle_run_bad_index.restype = C.c_longlong
            for f in ("oracle_run_lambda", "oracle_run_residual", "oracle_run_ortho"):
                getattr(L, f).argtypes = [C.c_void_p]
                getattr(L, f).restype = C.c_double
            L.oracle_run_copy_x.argtypes = [C.c_void_p, dp]
            L.oracle_run_level_info.argtypes = [C.c_void_p, C.c_int, lp, dp]
            L.oracle_run_copy_level.argtypes = [C.c_void_p, C.c_int, ip, ip, dp, dp, ip, ip, ip, dp]
            L.oracle_match.argtypes = [C.c_int, C.c_longlong, ip, ip, dp, C.c_int, C.c_int, ip, ip]
            L.oracle_aggregate.argtypes = [C.c_int, C.c_longlong, ip, ip, dp, ip, C.c_int, ip]
            L.oracle_hec_paper.argtypes = [C.c_int, C.c_longlong, ip, ip, dp, C.c_uint64, ip, ip]
            L.oracle_color.argtypes = [C.c_int, C.c_longlong, ip, ip, dp, C.c_int, ip, ip]
            L.oracle_galerkin.argtypes = [C.c_int, C.c_longlong, ip, ip, dp, ip, C.c_int, C.c_longlong,
                                          ip, ip, dp, dp, lp]
            L.oracle_gauss_seidel.argtypes = [C.c_int, ip, ip, dp, dp, dp, dp, C.c_int, ip]
            L.oracle_jacobi_eig.argtypes = [C.c_int, dp, dp, dp, C.c_int, C.c_double]
            L.oracle_jacobi_eig.restype = C.c_int
            L.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            L.oracle_splitmix64.restype = C.c_uint64
            L.oracle_vcycle.argtypes = [C.c_void_p, dp, dp]
            L.oracle_uniform01.argtypes = [C.c_uint64, C.c_uint64]
            L.oracle_uniform01.restype = C.c_double
            _lib = L
    return _lib


def _ip(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int))


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _csr(g):
    rowptr = np.ascontiguousarray(g.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.float64)
    return rowptr, col, w


def opts(**kw) -> Opts:
    o = Opts()
    lib().oracle_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Level:
    def __init__(self, **kw):
        self.__dict__.update(kw)


class Run:
    """Result of an oracle build or solve: hierarchy, per-level stats, vector."""

    def __init__(self):
        self._h = lib().oracle_run_create()
        self.status = None

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_run_destroy(self._h)
            self._h = None

    @property
    def num_levels(self):
        return lib().oracle_run_num_levels(self._h)

    def level(self, l) -> Level:
        info = np.zeros(12, dtype=np.int64)
        dinfo = np.zeros(2, dtype=np.float64)
        lib().oracle_run_level_info(self._h, l, info.ctypes.data_as(C.POINTER(C.c_longlong)), _dp(dinfo))
        n, nnz = int(info[0]), int(info[1])
        rowptr = np.zeros(n + 1, np.int32)
        col = np.zeros(max(nnz, 1), np.int32)
        w = np.zeros(max(nnz, 1), np.float64)
        d = np.zeros(n, np.float64)
        agg = np.full(n, -1, np.int32) if info[7] else None
        mate = np.full(n, -1, np.int32)
        color = np.full(n, -1, np.int32)
        x = np.zeros(n, np.float64) if info[8] else None
        lib().oracle_run_copy_level(self._h, l, _ip(rowptr), _ip(col), _dp(w), _dp(d), _ip(agg), _ip(mate),
                                    _ip(color), _dp(x))
        return Level(n=n, nnz=nnz, nc=int(info[2]), ncolors=int(info[3]), match_rounds=int(info[4]),
                     gs_sweeps=int(info[5]), pi_iters=int(info[6]), color_rounds=int(info[9]),
                     refine_iters=int(info[10]), capped=int(info[11]),
                     sigma=float(dinfo[0]), last_cos=float(dinfo[1]), rowptr=rowptr, col=col[:nnz], w=w[:nnz],
                     d=d, agg=agg, mate=mate, color=color, x=x)

    @property
    def levels(self):
        return [self.level(l) for l in range(self.num_levels)]

    @property
    def lam(self):
        return lib().oracle_run_lambda(self._h)

    @property
    def residual(self):
        return lib().oracle_run_residual(self._h)

    @property
    def ortho(self):
        return lib().oracle_run_ortho(self._h)

    @property
    def bad_index(self):
        return lib().oracle_run_bad_index(self._h)

    def x(self, n):
        out = np.zeros(n, np.float64)
        lib().oracle_run_copy_x(self._h, _dp(out))
        return out

    @property
    def pi_iters(self):
        return [self.level(l).pi_iters for l in range(self.num_levels)]

    def vcycle(self, b):
        """One V-cycle of the run's hierarchy applied to b (level-0 numbering)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        e = np.zeros_like(b)
        st = lib().oracle_vcycle(self._h, _dp(b), _dp(e))
        if st != OK:
            raise RuntimeError(f"oracle_vcycle status {st}")
        return e

    @property
    def refine_iters(self):
        return self.level(0).refine_iters if self.num_levels else 0

    @property
    def capped(self):
        return any(self.level(l).capped for l in range(self.num_levels))


def build_hierarchy(g, **kw) -> Run:
    """Setup phase of Alg. 3 on graph g (inputs.CSR)."""
    r = Run()
    rowptr, col, w = _csr(g)
    o = opts(**kw)
    r.status = lib().oracle_build(r._h, g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), C.byref(o))
    return r


def solve(g, forced_pi=None, **kw) -> Run:
    """Whole method on graph g; returns a Run (check .status)."""
    r = Run()
    rowptr, col, w = _csr(g)
    o = opts(**kw)
    fp = None
    if forced_pi is not None:
        fp = np.full(64, -1, np.int32)
        fp[:len(forced_pi)] = np.asarray(forced_pi, dtype=np.int32)
    r.status = lib().oracle_solve(r._h, g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), C.byref(o), _ip(fp))
    r.n = g.n
    return r


def match(g, mode=HEC_HANDSHAKE, tie_rule=TIE_HASHED):
    rowptr, col, w = _csr(g)
    mate = np.zeros(g.n, np.int32)
    rounds = C.c_int(0)
    st = lib().oracle_match(g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), mode, tie_rule, _ip(mate), C.byref(rounds))
    if st != OK:
        raise RuntimeError(f"oracle_match status {st}")
    return mate, rounds.value


def aggregate(g, mate, tie_rule=TIE_HASHED):
    rowptr, col, w = _csr(g)
    mate = np.ascontiguousarray(mate, dtype=np.int32)
    agg = np.zeros(g.n, np.int32)
    nc = lib().oracle_aggregate(g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), _ip(mate), tie_rule, _ip(agg))
    if nc < 0:
        raise RuntimeError(f"oracle_aggregate status {nc}")
    return agg, nc


def hec_paper(g, seed=0, perm=None):
    rowptr, col, w = _csr(g)
    agg = np.zeros(g.n, np.int32)
    p = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    nc = lib().oracle_hec_paper(g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), seed, _ip(p), _ip(agg))
    if nc < 0:
        raise RuntimeError(f"oracle_hec_paper status {nc}")
    return agg, nc


def color(g, jp=False):
    rowptr, col, w = _csr(g)
    c = np.zeros(g.n, np.int32)
    rounds = C.c_int(0)
    nc = lib().oracle_color(g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), int(jp), _ip(c), C.byref(rounds))
    if nc < 0:
        raise RuntimeError(f"oracle_color status {nc}")
    return c, nc, rounds.value


def galerkin(g, agg, nc):
    rowptr, col, w = _csr(g)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    sizes = np.zeros(2, np.int64)
    cap = g.nnz
    crow = np.zeros(nc + 1, np.int32)
    ccol = np.zeros(max(cap, 1), np.int32)
    cw = np.zeros(max(cap, 1), np.float64)
    cd = np.zeros(max(nc, 1), np.float64)
    st = lib().oracle_galerkin(g.n, g.nnz, _ip(rowptr), _ip(col), _dp(w), _ip(agg), nc, cap, _ip(crow), _ip(ccol),
                               _dp(cw), _dp(cd), sizes.ctypes.data_as(C.POINTER(C.c_longlong)))
    if st != OK:
        raise RuntimeError(f"oracle_galerkin status {st}")
    m = int(sizes[1])
    return crow, ccol[:m], cw[:m], cd[:nc]


def gauss_seidel(rowptr, col, w, d, b, x, sweeps, order=None):
    """Alg. 2 (N sweeps) for (diag(d) - W) x = b; x updated in place and returned."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    b = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    lib().oracle_gauss_seidel(len(d), _ip(rowptr), _ip(col), _dp(w), _dp(d), _dp(b), _dp(x), sweeps, _ip(o))
    return x


def jacobi_eig(A, max_sweeps=100, tol=1e-15):
    """Dense cyclic Jacobi: (eigenvalues ascending, eigenvectors as columns, sweeps)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    ev = np.zeros(n)
    V = np.zeros((n, n))
    sw = lib().oracle_jacobi_eig(n, _dp(A), _dp(ev), _dp(V), max_sweeps, tol)
    return ev, V, sw


def splitmix64(seed, k):
    return lib().oracle_splitmix64(seed, k)


def uniform01(seed, k):
    return lib().oracle_uniform01(seed, k)
