"""ctypes binding of the C-ABI in include/fiedler.h (argument marshalling only).

Every step of the solve runs in the CUDA library ``_build/libfiedler.so``; this
module only lays out the C structs, passes pointers (numpy arrays for host
memory, torch CUDA tensors for device memory) and converts status codes.  It
raises if the library has not been built: there is no CPU fallback.

The functions ``fiedler_*`` mirror the C entry points one to one; ``Plan`` is
a small convenience wrapper used by the tests and the benchmark.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- constants
FIEDLER_OK = 0
FIEDLER_EAGAIN = 1
FIEDLER_EINVAL = -1
FIEDLER_ENOMEM = -2
FIEDLER_EDISCONNECTED = -3
FIEDLER_ENOTCONVERGED = -4
FIEDLER_ETIMEOUT = -5
FIEDLER_ECUDA = -6
FIEDLER_ECANCELED = -7
FIEDLER_EDEGENERATE = -8
FIEDLER_ENOTSUP = -9

FIEDLER_FP64 = 0
FIEDLER_FP32_FP64RED = 1
FIEDLER_TIE_HASHED = 0
FIEDLER_TIE_INDEX = 1
FIEDLER_W_F32 = 0
FIEDLER_W_F64 = 1
FIEDLER_REFINE_NONE = 0
FIEDLER_REFINE_LOBPCG = 1
FIEDLER_REFINE_LANCZOS = 2
FIEDLER_HEC_DOMINANT = 0
FIEDLER_HEC_PAPER = 1
FIEDLER_PRECOND_DEGREE = 0
FIEDLER_PRECOND_VCYCLE = 1

#: exported symbols declared in include/fiedler.h
SYMBOLS = (
    "fiedler_options_default", "fiedler_plan_create", "fiedler_solve", "fiedler_batch_submit",
    "fiedler_poll", "fiedler_cancel", "fiedler_plan_destroy", "fiedler_status_str",
    "fiedler_plan_num_levels", "fiedler_plan_level_info", "fiedler_plan_copy_level",
    "fiedler_plan_set_profiling", "fiedler_plan_get_profile", "fiedler_solve_noalloc",
    "fiedler_solve_batch", "fiedler_plan_serving_stats", "fiedler_plan_autotune", "fiedler_poll_any",
    "fiedler_partition",
)


class fiedler_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("coarse_max_n", C.c_int),
        ("max_levels", C.c_int),
        ("stall_ratio", C.c_double),
        ("gs_sweeps", C.c_int),
        ("pi_max_iters", C.c_int),
        ("pi_max_iters_coarsest", C.c_int),
        ("pi_cos_tol", C.c_double),
        ("resid_tol", C.c_double),
        ("tie_rule", C.c_int),
        ("seed", C.c_uint64),
        ("validate", C.c_int),
        ("tail_max_n", C.c_int),
        ("tail_max_nnz", C.c_int),
        ("barrier_timeout_ms", C.c_int),
        ("fault_inject", C.c_int),
        ("hbm_budget_bytes", C.c_size_t),
        ("max_batch", C.c_int),
        ("queue_budget_bytes", C.c_size_t),
        ("batch_threads", C.c_int),
        ("refine", C.c_int),
        ("refine_max_iters", C.c_int),
        ("refine_tol", C.c_double),
        ("lanczos_basis", C.c_int),
        ("hec_mode", C.c_int),
        ("refine_precond", C.c_int),
        ("lane_sms", C.c_int),
        ("lane_min_n", C.c_int),
        ("lane_slots", C.c_int),
    ]


class fiedler_graph(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("rowptr", C.c_void_p),
        ("col", C.c_void_p),
        ("w", C.c_void_p),
        ("w_dtype", C.c_int),
        ("on_device", C.c_int),
    ]


class fiedler_result(C.Structure):
    _fields_ = [
        ("lambda2", C.c_double),
        ("residual", C.c_double),
        ("ortho", C.c_double),
        ("levels", C.c_int),
        ("coarsest_n", C.c_int),
        ("pi_iters_total", C.c_int),
        ("gs_sweeps_total", C.c_int),
        ("x", C.c_void_p),
        ("x_on_device", C.c_int),
        ("ms", C.c_float),
        ("bad_index", C.c_longlong),
        ("status", C.c_int),
        ("refine_iters", C.c_int),
    ]


class fiedler_level_info(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("nc", C.c_int),
        ("ncolors", C.c_int),
        ("match_rounds", C.c_int),
        ("color_rounds", C.c_int),
        ("gs_sweeps", C.c_int),
        ("pi_iters", C.c_int),
        ("sigma", C.c_double),
        ("last_cos", C.c_double),
        ("phase_ms", C.c_float * 16),
        ("refine_iters", C.c_int),
    ]


class fiedler_partition_info(C.Structure):
    _fields_ = [
        ("parts", C.c_int),
        ("solves", C.c_int),
        ("component_splits", C.c_int),
        ("ms", C.c_float),
    ]


class fiedler_serving_stats(C.Structure):
    _fields_ = [
        ("submitted", C.c_uint64),
        ("completed", C.c_uint64),
        ("batches", C.c_uint64),
        ("p50_ms", C.c_double),
        ("p99_ms", C.c_double),
        ("mean_ms", C.c_double),
        ("mean_batch", C.c_double),
        ("peak_inflight_bytes", C.c_size_t),
        ("launches", C.c_uint64),
        ("block_seconds", C.c_double),
        ("mean_inflight", C.c_double),
        ("mean_blocks", C.c_double),
    ]


class fiedler_tuning(C.Structure):
    _fields_ = [
        ("batch_threads", C.c_int),
        ("batch_ms", C.c_float * 3),
    ]


class fiedler_profile(C.Structure):
    _fields_ = [
        ("kernel_launches", C.c_uint64),
        ("n_kernels", C.c_int),
        ("kernel_name", C.c_char_p * 4),
        ("kernel_launches_by", C.c_int * 4),
        ("kernel_ms", C.c_float * 4),
        ("kernel_bytes", C.c_double * 4),
        ("n_phases", C.c_int),
        ("phase_name", C.c_char_p * 16),
        ("phase_ms", (C.c_double * 16) * 2),
        ("phase_bytes", (C.c_double * 16) * 2),
    ]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libfiedler.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run paper_1602_04386_gb300.build.build() "
                               "(or __graft_entry__.build()) first; there is no CPU fallback")
        L = C.CDLL(path)
        vp = C.c_void_p
        L.fiedler_options_default.argtypes = [C.POINTER(fiedler_options)]
        L.fiedler_options_default.restype = None
        L.fiedler_plan_create.argtypes = [C.POINTER(fiedler_options), vp, C.POINTER(vp)]
        L.fiedler_solve.argtypes = [vp, C.POINTER(fiedler_graph), C.POINTER(fiedler_result)]
        L.fiedler_batch_submit.argtypes = [vp, C.POINTER(fiedler_graph), C.POINTER(C.c_uint64)]
        L.fiedler_poll.argtypes = [vp, C.c_uint64, C.c_int, C.POINTER(fiedler_result)]
        L.fiedler_cancel.argtypes = [vp, C.c_uint64]
        L.fiedler_plan_destroy.argtypes = [vp]
        L.fiedler_plan_destroy.restype = None
        L.fiedler_status_str.argtypes = [C.c_int]
        L.fiedler_status_str.restype = C.c_char_p
        L.fiedler_plan_num_levels.argtypes = [vp]
        L.fiedler_plan_level_info.argtypes = [vp, C.c_int, C.POINTER(fiedler_level_info)]
        L.fiedler_plan_copy_level.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, vp]
        L.fiedler_plan_set_profiling.argtypes = [vp, C.c_int]
        L.fiedler_plan_get_profile.argtypes = [vp, C.POINTER(fiedler_profile)]
        L.fiedler_solve_noalloc.argtypes = [C.POINTER(fiedler_options), C.POINTER(fiedler_graph), vp, vp,
                                            C.POINTER(fiedler_result)]
        L.fiedler_solve_batch.argtypes = [vp, C.POINTER(fiedler_graph), C.c_int, C.POINTER(fiedler_result)]
        L.fiedler_plan_serving_stats.argtypes = [vp, C.POINTER(fiedler_serving_stats)]
        L.fiedler_plan_autotune.argtypes = [vp, C.POINTER(fiedler_graph), C.c_int, C.POINTER(fiedler_tuning)]
        L.fiedler_poll_any.argtypes = [vp, C.POINTER(C.c_uint64), C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.fiedler_partition.argtypes = [vp, C.POINTER(fiedler_graph), C.c_int, C.c_void_p, C.c_int,
                                        C.POINTER(fiedler_partition_info)]
        for f in ("fiedler_plan_create", "fiedler_solve", "fiedler_batch_submit", "fiedler_poll", "fiedler_cancel",
                  "fiedler_plan_num_levels", "fiedler_plan_level_info", "fiedler_plan_copy_level",
                  "fiedler_plan_set_profiling", "fiedler_plan_get_profile", "fiedler_solve_noalloc",
                  "fiedler_solve_batch", "fiedler_plan_serving_stats", "fiedler_plan_autotune", "fiedler_poll_any"):
            getattr(L, f).restype = C.c_int
        _lib = L
        return L


# ------------------------------------------------------ same-name wrappers
def fiedler_options_default() -> fiedler_options:
    o = fiedler_options()
    load().fiedler_options_default(C.byref(o))
    return o


def fiedler_plan_create(opts: fiedler_options | None, cuda_stream: int | None):
    h = C.c_void_p()
    st = load().fiedler_plan_create(C.byref(opts) if opts is not None else None, cuda_stream, C.byref(h))
    return st, h


def fiedler_solve(plan, graph: fiedler_graph, result: fiedler_result) -> int:
    return load().fiedler_solve(plan, C.byref(graph), C.byref(result))


def fiedler_batch_submit(plan, graph: fiedler_graph):
    t = C.c_uint64(0)
    st = load().fiedler_batch_submit(plan, C.byref(graph), C.byref(t))
    return st, t.value


def fiedler_poll(plan, ticket: int, timeout_ms: int, result: fiedler_result) -> int:
    return load().fiedler_poll(plan, ticket, timeout_ms, C.byref(result))


def fiedler_partition(plan, graph: fiedler_graph, parts: int, labels_ptr, labels_on_device: int):
    info = fiedler_partition_info()
    st = load().fiedler_partition(plan, C.byref(graph), parts, labels_ptr, labels_on_device, C.byref(info))
    return st, info


def fiedler_poll_any(plan, max_count: int, timeout_ms: int):
    """(status, [ticket ids]) of tickets finished since the last call."""
    buf = (C.c_uint64 * max_count)()
    cnt = C.c_int(0)
    st = load().fiedler_poll_any(plan, buf, max_count, timeout_ms, C.byref(cnt))
    return st, [buf[i] for i in range(cnt.value)]


def fiedler_cancel(plan, ticket: int) -> int:
    return load().fiedler_cancel(plan, ticket)


def fiedler_plan_destroy(plan) -> None:
    load().fiedler_plan_destroy(plan)


def fiedler_status_str(st: int) -> str:
    return load().fiedler_status_str(st).decode()


def fiedler_plan_num_levels(plan) -> int:
    return load().fiedler_plan_num_levels(plan)


def fiedler_plan_level_info(plan, level: int):
    info = fiedler_level_info()
    st = load().fiedler_plan_level_info(plan, level, C.byref(info))
    return st, info


def fiedler_plan_copy_level(plan, level, rowptr, col, w, d, agg, mate, color) -> int:
    def p(a):
        return None if a is None else a.ctypes.data
    return load().fiedler_plan_copy_level(plan, level, p(rowptr), p(col), p(w), p(d), p(agg), p(mate), p(color))


def fiedler_plan_set_profiling(plan, on: int) -> int:
    return load().fiedler_plan_set_profiling(plan, on)


def fiedler_plan_get_profile(plan):
    pr = fiedler_profile()
    st = load().fiedler_plan_get_profile(plan, C.byref(pr))
    return st, pr


def fiedler_solve_batch(plan, graphs, results) -> int:
    """graphs: ctypes array of fiedler_graph; results: ctypes array of fiedler_result."""
    return load().fiedler_solve_batch(plan, graphs, len(graphs), results)


def fiedler_plan_autotune(plan, graphs) -> tuple[int, fiedler_tuning]:
    """graphs: ctypes array of fiedler_graph (the sample)."""
    out = fiedler_tuning()
    st = load().fiedler_plan_autotune(plan, graphs, len(graphs), C.byref(out))
    return st, out


def fiedler_plan_serving_stats(plan):
    out = fiedler_serving_stats()
    st = load().fiedler_plan_serving_stats(plan, C.byref(out))
    return st, out


def fiedler_solve_noalloc(opts: fiedler_options | None, graph: fiedler_graph, x_dev_ptr, cuda_stream,
                          result: fiedler_result) -> int:
    return load().fiedler_solve_noalloc(C.byref(opts) if opts is not None else None, C.byref(graph), x_dev_ptr,
                                        cuda_stream, C.byref(result))


# ------------------------------------------------------------ convenience
class FiedlerError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {fiedler_status_str(status)} ({status})")


class Result:
    """Result of one solve: scalars, the vector (numpy float64 or a torch tensor)."""

    def __init__(self, r: fiedler_result, x):
        self.status = r.status
        self.lambda2 = r.lambda2
        self.residual = r.residual
        self.ortho = r.ortho
        self.levels = r.levels
        self.coarsest_n = r.coarsest_n
        self.pi_iters_total = r.pi_iters_total
        self.gs_sweeps_total = r.gs_sweeps_total
        self.ms = r.ms
        self.bad_index = r.bad_index
        self.refine_iters = r.refine_iters
        self.x = x

    def __repr__(self):
        return (f"Result(status={self.status}, lambda2={self.lambda2!r}, residual={self.residual:.3e}, "
                f"levels={self.levels}, ms={self.ms:.3f})")


def device_graph(g, torch_device="cuda"):
    """Copies an inputs.CSR to torch CUDA tensors; returns (graph struct, tensors kept alive)."""
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(g.rowptr, dtype=np.int32)).to(torch_device)
    ci = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(torch_device)
    w = torch.from_numpy(np.ascontiguousarray(g.w)).to(torch_device)
    if w.numel() == 0:
        w = torch.zeros(1, dtype=w.dtype, device=torch_device)
        ci = torch.zeros(1, dtype=torch.int32, device=torch_device)
    wd = FIEDLER_W_F64 if g.w.dtype == np.float64 else FIEDLER_W_F32
    gs = fiedler_graph(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), w.data_ptr(), wd, 1)
    return gs, (rp, ci, w)


def host_graph(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w)
    wd = FIEDLER_W_F64 if w.dtype == np.float64 else FIEDLER_W_F32
    gs = fiedler_graph(g.n, g.nnz, rp.ctypes.data, ci.ctypes.data if ci.size else None,
                       w.ctypes.data if w.size else None, wd, 0)
    return gs, (rp, ci, w)


class Plan:
    """Owns a fiedler_plan; options are fiedler_options field names."""

    def __init__(self, stream: int | None = None, **opts):
        self.opts = fiedler_options_default()
        for k, v in opts.items():
            if not hasattr(self.opts, k):
                raise KeyError(k)
            setattr(self.opts, k, v)
        st, self.h = fiedler_plan_create(self.opts, stream)
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_plan_create")

    def close(self):
        if getattr(self, "h", None):
            fiedler_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve_struct(self, graph: fiedler_graph, x=None, x_on_device=False) -> fiedler_result:
        r = fiedler_result()
        if x is not None:
            r.x = x.data_ptr() if x_on_device else x.ctypes.data
            r.x_on_device = 1 if x_on_device else 0
        fiedler_solve(self.h, graph, r)
        return r

    def solve(self, g, on_device=True, want_x=True, x_on_device=False) -> Result:
        """Solve inputs.CSR g.  on_device: inputs copied to the GPU first (not timed
        by the library); x returned as numpy (or as a torch tensor if x_on_device)."""
        keep = None
        if on_device:
            gs, keep = device_graph(g)
        else:
            gs, keep = host_graph(g)
        x = None
        if want_x:
            if x_on_device:
                import torch
                x = torch.empty(g.n, dtype=torch.float64, device="cuda")
            else:
                x = np.zeros(g.n, dtype=np.float64)
        r = self.solve_struct(gs, x, x_on_device)
        del keep
        return Result(r, x)

    @property
    def num_levels(self) -> int:
        return fiedler_plan_num_levels(self.h)

    def level_info(self, l):
        st, info = fiedler_plan_level_info(self.h, l)
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_plan_level_info")
        return info

    def copy_level(self, l):
        info = self.level_info(l)
        n, m = int(info.n), int(info.nnz)
        out = dict(rowptr=np.zeros(n + 1, np.int32), col=np.zeros(max(m, 1), np.int32),
                   w=np.zeros(max(m, 1), np.float64), d=np.zeros(n, np.float64), agg=np.full(n, -1, np.int32),
                   mate=np.full(n, -1, np.int32), color=np.full(n, -1, np.int32))
        st = fiedler_plan_copy_level(self.h, l, out["rowptr"], out["col"], out["w"], out["d"], out["agg"],
                                     out["mate"], out["color"])
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_plan_copy_level")
        out["col"] = out["col"][:m]
        out["w"] = out["w"][:m]
        out["info"] = info
        return out

    def partition(self, g, parts, on_device=True):
        """Recursive spectral bisection of inputs.CSR g into `parts` parts;
        returns (labels as numpy int32, fiedler_partition_info)."""
        gs, keep = device_graph(g) if on_device else host_graph(g)
        labels = np.zeros(g.n, np.int32)
        st, info = fiedler_partition(self.h, gs, parts, labels.ctypes.data, 0)
        del keep
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_partition")
        return labels, info

    def set_profiling(self, on=True):
        fiedler_plan_set_profiling(self.h, 1 if on else 0)

    def profile(self) -> fiedler_profile:
        st, pr = fiedler_plan_get_profile(self.h)
        return pr

    def submit(self, g, on_device=False) -> int:
        gs, keep = (device_graph(g) if on_device else host_graph(g))
        st, t = fiedler_batch_submit(self.h, gs)
        del keep
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_batch_submit")
        return t

    def poll(self, ticket, timeout_ms=-1, n=None):
        r = fiedler_result()
        x = None
        if n is not None:
            x = np.zeros(n, np.float64)
            r.x = x.ctypes.data
        st = fiedler_poll(self.h, ticket, timeout_ms, r)
        return st, Result(r, x)

    def finished(self, max_count=256, timeout_ms=-1):
        """Ids of tickets that finished since the last call (empty on timeout)."""
        st, ids = fiedler_poll_any(self.h, max_count, timeout_ms)
        if st not in (FIEDLER_OK, FIEDLER_EAGAIN):
            raise FiedlerError(st, "fiedler_poll_any")
        return ids

    def cancel(self, ticket) -> int:
        return fiedler_cancel(self.h, ticket)

    def serving_stats(self) -> fiedler_serving_stats:
        st, out = fiedler_plan_serving_stats(self.h)
        return out

    def autotune(self, graphs, on_device=True) -> fiedler_tuning:
        """Autotunes the batched form's block size on a sample of inputs.CSR graphs."""
        keep = []
        garr = (fiedler_graph * len(graphs))()
        for i, g in enumerate(graphs):
            gs, k = device_graph(g) if on_device else host_graph(g)
            keep.append(k)
            garr[i] = gs
        st, out = fiedler_plan_autotune(self.h, garr)
        del keep
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_plan_autotune")
        return out

    def solve_batch_struct(self, garr, rarr) -> int:
        """Batched solve of prepared arrays of fiedler_graph and fiedler_result
        (same length); returns the fiedler_status of the call."""
        return fiedler_solve_batch(self.h, garr, rarr)

    def solve_batch(self, graphs, on_device=True, want_x=True):
        """Batched solve of a list of inputs.CSR; returns a list of Result (x as numpy)."""
        keep = []
        garr = (fiedler_graph * len(graphs))()
        rarr = (fiedler_result * len(graphs))()
        xs = []
        for i, g in enumerate(graphs):
            gs, k = device_graph(g) if on_device else host_graph(g)
            keep.append(k)
            garr[i] = gs
            x = np.zeros(g.n, np.float64) if want_x else None
            xs.append(x)
            if x is not None:
                rarr[i].x = x.ctypes.data
                rarr[i].x_on_device = 0
        st = fiedler_solve_batch(self.h, garr, rarr)
        if st != FIEDLER_OK:
            raise FiedlerError(st, "fiedler_solve_batch")
        del keep
        return [Result(rarr[i], xs[i]) for i in range(len(graphs))]
