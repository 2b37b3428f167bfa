"""Batched and serving forms through the C-ABI.

A graph's result must not depend on the batch it runs in: batched results
are compared bit for bit with the same graph solved alone (one-block engine:
tail_max_n >= n and tail_max_nnz >= nnz), alone and in mixes, through fiedler_solve_batch and the
ticket queue, including tickets admitted while others are on the GPU.  A
sample is also checked against the oracle (hierarchy bit for bit, lambda_2
to 1e-10 in FP64, 1e-5 in FP32)."""
import time

import numpy as np
import pytest

import oracle
from paper_1602_04386_gb300 import inputs

pytestmark = pytest.mark.gpu

fiedler = pytest.importorskip("paper_1602_04386_gb300.fiedler")
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    fiedler.load()


def mixed_grids(k, seed=0):
    rng = inputs.uniform01(seed, np.arange(2 * k))
    out = []
    for i in range(k):
        m = 20 + int(rng[2 * i] * 100)
        q = 20 + int(rng[2 * i + 1] * 100)
        out.append(inputs.grid(m, q, "uniform" if i % 2 else "unit", seed=seed + i))
    return out


def alone(g, precision):
    with fiedler.Plan(precision=precision, tail_max_n=1 << 30, tail_max_nnz=1 << 30) as p:
        return p.solve(g)


@pytest.mark.parametrize("precision", [fiedler.FIEDLER_FP64, fiedler.FIEDLER_FP32_FP64RED])
def test_batch_equals_alone_bitwise(precision):
    gs = mixed_grids(12, seed=3)
    with fiedler.Plan(precision=precision) as p:
        res = p.solve_batch(gs)
        res_host = p.solve_batch(gs, on_device=False)
        sub = p.solve_batch([gs[5]])  # the same graph alone in a batch of one
    for g, r, rh in zip(gs, res, res_host):
        a = alone(g, precision)
        assert r.status == a.status == fiedler.FIEDLER_OK
        assert r.lambda2 == a.lambda2 and np.array_equal(r.x, a.x)
        assert rh.lambda2 == r.lambda2 and np.array_equal(rh.x, r.x)
    assert sub[0].lambda2 == res[5].lambda2 and np.array_equal(sub[0].x, res[5].x)


def test_batch_against_oracle_sample():
    gs = mixed_grids(6, seed=11)
    with fiedler.Plan(precision=fiedler.FIEDLER_FP64) as p:
        res = p.solve_batch(gs)
    for g, r in zip(gs[:3], res[:3]):
        with fiedler.Plan(precision=fiedler.FIEDLER_FP64, tail_max_n=1 << 30, tail_max_nnz=1 << 30) as q:
            a = q.solve(g)
            counts = [q.level_info(l).pi_iters for l in range(q.num_levels)]
        ref = oracle.solve(g, forced_pi=counts)
        assert abs(r.lambda2 - ref.lam) <= 1e-10 * ref.lam
        assert np.abs(r.x - ref.x(g.n)).max() <= 1e-8


def test_batch_invalid_members_do_not_stop_the_batch():
    good = inputs.grid(30, 20, "uniform", seed=1)
    bad = inputs.CSR(good.n, good.rowptr, good.col.copy(), good.w.copy())
    bad.w[3] *= 2
    disc = inputs.disjoint_union(inputs.grid(10, 8), inputs.path(12))
    with fiedler.Plan() as p:
        res = p.solve_batch([good, bad, disc, good])
    assert res[0].status == res[3].status == fiedler.FIEDLER_OK
    assert res[1].status == fiedler.FIEDLER_EINVAL
    assert res[2].status == fiedler.FIEDLER_EDISCONNECTED
    assert res[0].lambda2 == res[3].lambda2


def test_serving_tickets_alone_and_in_the_mix():
    """Tickets submitted in waves while earlier ones are on the GPU (admitted
    as memory and blocks free up) give the same result as alone."""
    gs = mixed_grids(24, seed=5)
    want = [alone(g, fiedler.FIEDLER_FP32_FP64RED) for g in gs]
    with fiedler.Plan(max_batch=5) as p:
        tickets = []
        for i, g in enumerate(gs):
            tickets.append(p.submit(g))
            if i % 6 == 5:
                time.sleep(0.002)
        for g, t, a in zip(gs, tickets, want):
            st, r = p.poll(t, -1, n=g.n)
            assert st == fiedler.FIEDLER_OK
            assert r.lambda2 == a.lambda2 and np.array_equal(r.x, a.x)
        stats = p.serving_stats()
    assert stats.submitted == stats.completed == len(gs)
    assert stats.batches >= 2 and stats.p99_ms >= stats.p50_ms > 0


def test_serving_memory_budget_admits_one_at_a_time():
    gs = mixed_grids(5, seed=9)
    want = [alone(g, fiedler.FIEDLER_FP32_FP64RED) for g in gs]
    with fiedler.Plan(hbm_budget_bytes=1) as p:
        tickets = [p.submit(g) for g in gs]
        for g, t, a in zip(gs, tickets, want):
            st, r = p.poll(t, -1, n=g.n)
            assert st == fiedler.FIEDLER_OK and r.lambda2 == a.lambda2
        stats = p.serving_stats()
    assert stats.batches == len(gs) and stats.mean_batch == 1.0


def test_serving_cancel_and_poll_timeout():
    with fiedler.Plan(max_batch=1) as p:
        big = inputs.grid(200, 150, "uniform", seed=2)
        ts = [p.submit(big) for _ in range(3)]
        p.cancel(ts[2])
        st, _ = p.poll(ts[0], 0)
        assert st in (fiedler.FIEDLER_EAGAIN, fiedler.FIEDLER_OK)
        for t in ts[:2]:
            st, r = p.poll(t, -1, n=big.n)
            assert st == fiedler.FIEDLER_OK
        st, _ = p.poll(ts[2], -1)
        assert st in (fiedler.FIEDLER_ECANCELED, fiedler.FIEDLER_OK)


def test_submit_back_pressure():
    """With the queue budget used up, submit returns EAGAIN without queueing;
    once the earlier ticket is polled, the same submit succeeds."""
    g = inputs.grid(40, 30, "unit")
    gs, keep = fiedler.host_graph(g)
    with fiedler.Plan(queue_budget_bytes=1) as p:
        st, t1 = fiedler.fiedler_batch_submit(p.h, gs)  # an empty queue always takes one
        assert st == fiedler.FIEDLER_OK
        st, _ = fiedler.fiedler_batch_submit(p.h, gs)
        assert st == fiedler.FIEDLER_EAGAIN
        assert fiedler.fiedler_poll(p.h, t1, -1, fiedler.fiedler_result()) == fiedler.FIEDLER_OK
        st, t2 = fiedler.fiedler_batch_submit(p.h, gs)
        assert st == fiedler.FIEDLER_OK
        r = fiedler.fiedler_result()
        assert fiedler.fiedler_poll(p.h, t2, -1, r) == fiedler.FIEDLER_OK
        with fiedler.Plan() as q:
            a = q.solve(g)
        assert abs(r.lambda2 - a.lambda2) <= 1e-5 * a.lambda2
    del keep


@pytest.mark.parametrize("threads", [256, 128])
def test_block_size_variants(threads):
    """Every block size of the batched kernel: a graph's result is the same
    alone and in a mixed batch (bit for bit), and grids agree with the
    512-thread kernel to the FP32-form tolerance."""
    gs = inputs.batch_mix(8, scale_range=(8, 10), side_range=(20, 60))
    with fiedler.Plan(batch_threads=threads) as p:
        mix = p.solve_batch(gs)
        alone = [p.solve_batch([g])[0] for g in gs]
    with fiedler.Plan(batch_threads=512) as q:
        ref = q.solve_batch(gs)
    for g, a, b, c in zip(gs, mix, alone, ref):
        assert a.status == b.status == fiedler.FIEDLER_OK
        assert a.lambda2 == b.lambda2 and np.array_equal(a.x, b.x)
        if g.name.startswith("grid"):
            assert abs(a.lambda2 - c.lambda2) <= 1e-5 * c.lambda2


def test_autotune_picks_a_block_size():
    gs = inputs.batch_mix(12, scale_range=(8, 10), side_range=(20, 80))
    with fiedler.Plan() as p:
        t = p.autotune(gs)
        assert t.batch_threads in (512, 256, 128)
        assert all(ms > 0 for ms in t.batch_ms)
        res = p.solve_batch(gs)
        assert all(r.status == fiedler.FIEDLER_OK for r in res)
    with fiedler.Plan(batch_threads=256) as q:
        st, _ = fiedler.fiedler_plan_autotune(q.h, (fiedler.fiedler_graph * 1)())
        assert st == fiedler.FIEDLER_EINVAL  # a fixed block size is not tuned


def test_poll_any_lists_each_finished_ticket_once():
    """fiedler_poll_any lists every ticket once, as it finishes; collecting
    them in that order gives the same results as alone; an empty list times
    out (EAGAIN)."""
    gs = mixed_grids(10, seed=21)
    want = [alone(g, fiedler.FIEDLER_FP32_FP64RED) for g in gs]
    with fiedler.Plan(max_batch=3) as p:
        st, ids = fiedler.fiedler_poll_any(p.h, 4, 0)
        assert st == fiedler.FIEDLER_EAGAIN and ids == []
        tickets = [p.submit(g) for g in gs]
        index = {t: i for i, t in enumerate(tickets)}
        seen = []
        deadline = time.time() + 120
        while len(seen) < len(gs) and time.time() < deadline:
            for t in p.finished(4, 1000):
                i = index[t]
                st, r = p.poll(t, 0, n=gs[i].n)
                assert st == fiedler.FIEDLER_OK
                assert r.lambda2 == want[i].lambda2 and np.array_equal(r.x, want[i].x)
                seen.append(t)
        assert sorted(seen) == sorted(tickets)
        assert p.finished(4, 50) == []
        # a ticket collected by fiedler_poll before it is listed is not listed
        t = p.submit(gs[0])
        assert p.poll(t, -1)[0] == fiedler.FIEDLER_OK
        assert p.finished(4, 50) == []
