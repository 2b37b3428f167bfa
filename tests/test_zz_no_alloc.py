"""fiedler_solve_noalloc: the entry point for callers that cannot allocate
device memory (code inside someone else's memory pool or cap, plug-ins that
must not grow the device footprint, allocation-free latency paths).  It must
give the same answer as the ordinary plan-based fiedler_solve, call after
call, while working only in its fixed device array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1602_04386_gb300 import inputs

pytestmark = pytest.mark.gpu

fiedler = pytest.importorskip("paper_1602_04386_gb300.fiedler")
torch = pytest.importorskip("torch")

# the tolerances of the parity suite: FP64 form 1e-10 relative in lambda_2
# (vector 1e-8), FP32 form 1e-5
TOL = {fiedler.FIEDLER_FP64: (1e-10, 1e-8), fiedler.FIEDLER_FP32_FP64RED: (1e-5, 1e-4)}


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    fiedler.load()


def _noalloc(g, precision, stream):
    gs, keep = fiedler.device_graph(g)
    x = torch.empty(g.n, dtype=torch.float64, device="cuda")
    opts = fiedler.fiedler_options_default()
    opts.precision = precision
    r = fiedler.fiedler_result()
    st = fiedler.fiedler_solve_noalloc(opts, gs, x.data_ptr(), stream, r)
    torch.cuda.synchronize()
    return st, r, x.cpu().numpy(), keep


GRAPHS = {
    "grid64x48": lambda: inputs.grid(64, 48, "unit"),
    "grid150x101w": lambda: inputs.grid(150, 101, "uniform", seed=7),
    "grid15x11w": lambda: inputs.grid(15, 11, "uniform", seed=2),  # n <= 256: the tiny-level path
    "knn6000": lambda: inputs.knn_mixture(6000, seed=4),
    "rmat13": lambda: inputs.rmat(13, seed=6),  # skewed degrees, near the array's size limit
}


@pytest.mark.parametrize("precision", [fiedler.FIEDLER_FP64, fiedler.FIEDLER_FP32_FP64RED])
@pytest.mark.parametrize("graph", list(GRAPHS))
def test_noalloc_matches_plan_solve_twice(precision, graph):
    g = GRAPHS[graph]()
    lam_tol, x_tol = TOL[precision]
    with fiedler.Plan(precision=precision, tail_max_n=1 << 30, tail_max_nnz=1 << 30) as p:
        ref = p.solve(g)
    assert ref.status == fiedler.FIEDLER_OK
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the shared array keeps the previous call's contents
        st, r, x, _keep = _noalloc(g, precision, stream)
        assert st == fiedler.FIEDLER_OK and r.status == st
        assert abs(r.lambda2 - ref.lambda2) <= lam_tol * abs(ref.lambda2)
        assert np.abs(x - ref.x).max() <= x_tol
        assert r.levels == ref.levels


def test_noalloc_allocates_no_device_memory():
    """After a first call (which looks up the array's address), further calls
    leave the device's free memory unchanged."""
    g = inputs.grid(90, 70, "uniform", seed=5)
    stream = torch.cuda.current_stream().cuda_stream
    gs, keep = fiedler.device_graph(g)
    x = torch.empty(g.n, dtype=torch.float64, device="cuda")
    r = fiedler.fiedler_result()
    assert fiedler.fiedler_solve_noalloc(None, gs, x.data_ptr(), stream, r) == fiedler.FIEDLER_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert fiedler.fiedler_solve_noalloc(None, gs, x.data_ptr(), stream, r) == fiedler.FIEDLER_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_too_large_and_host_inputs():
    big = inputs.grid(1024, 768, "uniform", seed=1)
    gs, keep = fiedler.device_graph(big)
    r = fiedler.fiedler_result()
    r.status = 12345
    st = fiedler.fiedler_solve_noalloc(None, gs, None, None, r)
    assert st == fiedler.FIEDLER_ENOTSUP and r.status == st and r.bad_index == -1
    small = inputs.grid(20, 10)
    hs, hkeep = fiedler.host_graph(small)
    r.status = 12345
    assert fiedler.fiedler_solve_noalloc(None, hs, None, None, r) == fiedler.FIEDLER_EINVAL
    assert r.status == fiedler.FIEDLER_EINVAL
    # the options are checked as fiedler_plan_create checks them
    sg, skeep = fiedler.device_graph(small)
    for field, bad in (("tie_rule", 7), ("pi_cos_tol", float("nan")), ("resid_tol", -1.0), ("refine", 9)):
        o = fiedler.fiedler_options_default()
        setattr(o, field, bad)
        r.status = 12345
        assert fiedler.fiedler_solve_noalloc(o, sg, None, None, r) == fiedler.FIEDLER_EINVAL, field
        assert r.status == fiedler.FIEDLER_EINVAL
