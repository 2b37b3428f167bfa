"""The large-graph lane of the batched and serving forms (lane_sms > 0):
graphs with n >= lane_min_n are solved one at a time by the cooperative
grid-wide kernels on lane_sms SMs while the one-block kernels run the rest.

Bars: a graph's result is the same, bit for bit, alone and in a mix (batched
call or ticket stream) under the same plan options; lane results match the
oracle (hierarchy bit for bit, lambda_2 within 1e-10 FP64 / 1e-5 FP32 of the
run replayed with the lane's per-level counts)."""
import numpy as np
import pytest

import oracle
from paper_1602_04386_gb300 import inputs

pytestmark = pytest.mark.gpu

fiedler = pytest.importorskip("paper_1602_04386_gb300.fiedler")
torch = pytest.importorskip("torch")

LANE = dict(lane_sms=8, lane_min_n=5000)


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    fiedler.load()


def mix():
    big = [inputs.grid(120, 90, "uniform", seed=1), inputs.knn_mixture(9000, seed=2), inputs.rmat(13, seed=3)]
    small = [inputs.grid(30 + 5 * i, 20 + 3 * i, "uniform", seed=10 + i) for i in range(6)]
    return big + small


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_with_lane_alone_equals_mix(precision):
    gs = mix()
    assert sum(g.n >= LANE["lane_min_n"] for g in gs) == 3
    with fiedler.Plan(precision=precision, **LANE) as p:
        res = p.solve_batch(gs)
        alone = [p.solve_batch([g])[0] for g in gs]
    for g, r, a in zip(gs, res, alone):
        assert r.status == a.status == fiedler.FIEDLER_OK, g.name
        assert r.lambda2 == a.lambda2 and np.array_equal(r.x, a.x), g.name


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_lane_results_match_oracle(precision, tol):
    g = inputs.grid(150, 101, "uniform", seed=6)
    with fiedler.Plan(precision=precision, **LANE) as p:
        r = p.solve_batch([g])[0]
    assert r.status == fiedler.FIEDLER_OK
    # the lane runs the single-graph engine: its per-level counts are those of
    # fiedler_solve with the same options on the grid-wide engine
    with fiedler.Plan(precision=precision) as q:
        s = q.solve(g)
        counts = [q.level_info(l).pi_iters for l in range(q.num_levels)]
    ref = oracle.solve(g, forced_pi=counts)
    assert abs(r.lambda2 - ref.lam) <= tol * ref.lam
    assert abs(s.lambda2 - ref.lam) <= tol * ref.lam
    if precision == 0:
        assert np.abs(r.x - ref.x(g.n)).max() <= 1e-8


@pytest.mark.parametrize("slots", [1, 2])
def test_serving_with_lane_alone_equals_mix(slots):
    """Large tickets run lane_slots at a time, each slot on its own stream and
    reduction partials: results are the same bits alone and in the mix."""
    gs = mix()
    with fiedler.Plan(lane_slots=slots, **LANE) as p:
        alone = []
        for g in gs:
            t = p.submit(g)
            st, r = p.poll(t, -1, n=g.n)
            assert st == fiedler.FIEDLER_OK
            alone.append(r)
        tickets = [p.submit(g) for g in gs]
        for g, t, a in zip(gs, tickets, alone):
            st, r = p.poll(t, -1, n=g.n)
            assert st == fiedler.FIEDLER_OK, g.name
            assert r.lambda2 == a.lambda2 and np.array_equal(r.x, a.x), g.name


def test_lane_slot_options_checked():
    with pytest.raises(fiedler.FiedlerError):
        fiedler.Plan(lane_sms=8, lane_slots=9)
    with pytest.raises(fiedler.FiedlerError):
        fiedler.Plan(lane_sms=8, lane_slots=0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with pytest.raises(fiedler.FiedlerError):  # the one-block kernels keep 16 SMs
        fiedler.Plan(lane_sms=sms - 15)
    with fiedler.Plan(lane_sms=sms - 16, lane_slots=4):
        pass


def test_lane_refined_batch_matches_fp64():
    """With the finest-level refinement, lane and block results of the FP32
    form agree with the FP64 form within 1e-5."""
    gs = mix()
    lam = {}
    for prec in (0, 1):
        with fiedler.Plan(precision=prec, refine=1, **LANE) as p:
            lam[prec] = [r.lambda2 for r in p.solve_batch(gs)]
    for a, b, g in zip(lam[1], lam[0], gs):
        assert abs(a - b) <= 1e-5 * b, g.name
