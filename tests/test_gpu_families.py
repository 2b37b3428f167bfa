"""Parity on the batched / spectral-clustering workload families: R-MAT
(skewed degrees: hub rows, large aggregates and segments take the block-level
sort paths) and the Gaussian-mixture kNN graph (weights exp(-d^2/0.25) span
many binades, so the FP64 Galerkin sums depend on their order).  Hierarchy
bit for bit, lambda_2 within 1e-10 (FP64) / 1e-5 (FP32) of the oracle run
with the GPU's per-level iteration counts; batched results equal single
solves bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1602_04386_gb300 import inputs

pytestmark = pytest.mark.gpu

fiedler = pytest.importorskip("paper_1602_04386_gb300.fiedler")
torch = pytest.importorskip("torch")

FP64, FP32 = 0, 1


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    fiedler.load()


def check_against_oracle(g, precision, lam_tol, tail=4096, tail_nnz=32768):
    with fiedler.Plan(precision=precision, tail_max_n=tail, tail_max_nnz=tail_nnz) as p:
        r = p.solve(g)
        assert r.status in (fiedler.FIEDLER_OK, fiedler.FIEDLER_ENOTCONVERGED), r
        counts = [p.level_info(l).pi_iters for l in range(p.num_levels)]
        ref = oracle.solve(g, forced_pi=counts)
        assert ref.status == 0 and p.num_levels == ref.num_levels
        for l in range(p.num_levels):
            a, b = p.copy_level(l), ref.level(l)
            assert np.array_equal(a["rowptr"], b.rowptr) and np.array_equal(a["col"], b.col), l
            assert np.array_equal(a["w"], b.w), l
            assert np.array_equal(a["color"], b.color), l
            if l + 1 < p.num_levels:
                assert np.array_equal(a["agg"], b.agg), l
    assert abs(r.lambda2 - ref.lam) <= lam_tol * abs(ref.lam), (r.lambda2, ref.lam)
    # reported residual and orthogonality against the oracle's (same counts)
    rt, at = (1e-6, 1e-12) if precision == FP64 else (1e-2, 1e-6)
    sigma = ref.level(0).sigma
    assert abs(r.residual - ref.residual) <= rt * ref.residual + at * sigma, (r.residual, ref.residual)
    assert abs(r.ortho - ref.ortho) <= (1e-12 if precision == FP64 else 1e-9)
    return r


@pytest.mark.parametrize("scale,seed", [(9, 1), (10, 2), (12, 3)])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (FP32, 1e-5)])
def test_rmat(scale, seed, precision, tol):
    g = inputs.rmat(scale, seed=seed)
    check_against_oracle(g, precision, tol)


@pytest.mark.parametrize("npts", [2000, 20000])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (FP32, 1e-5)])
def test_knn_mixture(npts, precision, tol):
    g = inputs.knn_mixture(npts, seed=7)
    check_against_oracle(g, precision, tol)


def test_batch_mix_equals_single_solves():
    gs = inputs.batch_mix(16, scale_range=(9, 12), side_range=(20, 120))
    with fiedler.Plan() as p:
        res = p.solve_batch(gs)
    for g, r in zip(gs, res):
        with fiedler.Plan(tail_max_n=1 << 30, tail_max_nnz=1 << 30) as q:
            a = q.solve(g)
        assert r.status == a.status == fiedler.FIEDLER_OK
        assert r.lambda2 == a.lambda2 and np.array_equal(r.x, a.x)


def test_knn_full_size_fp32():
    """The spectral-clustering workload at its full size (200,000 points, FP32
    form as the benchmark runs it): hierarchy bit for bit on every level, lambda_2
    within 1e-5 of the oracle run with the GPU's per-level iteration counts."""
    g = inputs.knn_mixture(200000)
    r = check_against_oracle(g, FP32, 1e-5)
    assert abs(np.linalg.norm(r.x) - 1) < 1e-9 and r.ortho < 1e-9


def test_batch_workload_sample():
    """Graphs of the 4096-graph batched workload solved in a batch with 29
    others (among them scale-16 R-MAT graphs, the largest): each equals its
    own one-block solve bit for bit, and that solve matches the oracle."""
    sample = [0, 1, 2, 15, 17, 37]  # grids and R-MAT graphs; 15, 17 and 37 are scale 16
    others = list(range(100, 124))
    gs = inputs.batch_mix(indices=sample + others)
    with fiedler.Plan() as p:
        res = p.solve_batch(gs)
    for g, r in zip(gs[:len(sample)], res[:len(sample)]):
        assert r.status == fiedler.FIEDLER_OK
        a = check_against_oracle(g, FP32, 1e-5, tail=1 << 30, tail_nnz=1 << 30)
        assert r.lambda2 == a.lambda2
