"""Spectral bisection with the Fiedler vector (the application the method
serves, Sec. 1): on a two-component Gaussian-mixture kNN graph whose
components touch (one connected graph), the sign cut of the GPU's Fiedler
vector recovers the mixture labels, in both forms, as the oracle's does."""
import numpy as np
import pytest

import oracle
from paper_1602_04386_gb300 import inputs

SEED = inputs.BASE_SEED + 33  # means 3.9 apart at sigma 0.5: one connected graph


def cut_accuracy(x, labels):
    cut = x > 0
    return max((cut == (labels == 1)).mean(), (cut == (labels == 0)).mean())


def test_oracle_sign_cut_recovers_the_mixture():
    g, labels = inputs.knn_mixture(20000, clusters=2, seed=SEED, return_labels=True)
    assert g.n == 20000  # connected: nothing dropped
    r = oracle.solve(g)
    assert cut_accuracy(r.x(g.n), labels) >= 0.99


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_sign_cut_recovers_the_mixture(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_04386_gb300 import fiedler
    g, labels = inputs.knn_mixture(20000, clusters=2, seed=SEED, return_labels=True)
    with fiedler.Plan(precision=precision) as p:
        r = p.solve(g)
    assert r.status == fiedler.FIEDLER_OK
    assert cut_accuracy(r.x, labels) >= 0.99
    ref = oracle.solve(g).x(g.n)
    assert ((r.x > 0) == (ref > 0)).mean() >= 0.99  # same cut as the oracle (signs are normalised)
