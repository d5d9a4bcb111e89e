"""The serving loop: results match the oracle, a field's result is the same alone and in a
mix of concurrent requests (bitwise: same kernels, fixed-order reductions), admission by HBM
footprint, error statuses."""
import math
import time

import numpy as np
import pytest
import torch

import oracle
from fieldgen import voronoi_stress_field, log_uniform_int
import paper_2105_01612_gb300 as eq

pytestmark = pytest.mark.gpu
W = np.array([1.0, 1, 1, 2, 2, 2]).reshape(6, 1, 1, 1)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def rel(a, b):
    return math.sqrt(float((W * (a - b) ** 2).sum() / (W * b ** 2).sum()))


def host_field(shape, seed, dtype=torch.float32):
    f = voronoi_stress_field(shape, 20, 150.0, 5.0, seed, dtype=dtype)
    return f.contiguous().pin_memory()


def test_alone_equals_in_the_mix_and_matches_oracle():
    srv = eq.Server(8 << 30, max_inflight=6)
    probe = host_field((40, 33, 48), 77)
    alone_out = torch.empty_like(probe).pin_memory()
    t = srv.submit(probe, alone_out)
    n_alone, _ = srv.wait(t)
    ref = oracle.project(probe.double().numpy(), "ddo")
    assert rel(alone_out.double().numpy(), ref) <= 2e-6
    rng = np.random.Generator(np.random.PCG64(210501612 + 4))
    jobs = []
    for i in range(24):
        shape = tuple(log_uniform_int(rng, 16, 96) for _ in range(3))
        x = host_field(shape, 1000 + i)
        o = torch.empty_like(x).pin_memory()
        jobs.append((srv.submit(x, o), x, o))
        if i == 11:
            mix_out = torch.empty_like(probe).pin_memory()
            tp = srv.submit(probe, mix_out)
    n_mix, _ = srv.wait(tp)
    for tk, x, o in jobs:
        nrm, lat = srv.wait(tk)
        assert lat > 0
        assert rel(o.double().numpy(), oracle.project(x.double().numpy(), "ddo")) <= 2e-6
    assert torch.equal(alone_out, mix_out)
    assert n_alone == n_mix
    srv.close()


def test_admission_budget_and_errors():
    x = host_field((32, 32, 32), 5)
    o = torch.empty_like(x).pin_memory()
    small = eq.Server(2 * x.numel() * 4 + 1024, max_inflight=4)   # room for one request at a time
    tickets = [small.submit(x, o.clone().pin_memory()) for _ in range(5)]
    for t in tickets:
        small.wait(t)
    big = host_field((64, 64, 64), 6)
    with pytest.raises(eq.EqError) as ei:
        small.submit(big, torch.empty_like(big))
    assert ei.value.status == 2                      # EQ_ERR_OOM
    with pytest.raises(eq.EqError) as ei:
        small.poll(123456789)
    assert ei.value.status == 7                      # EQ_ERR_NOT_FOUND
    small.close()


def test_destroy_cancels_queued_requests():
    srv = eq.Server(1 << 30, max_inflight=1)
    x = host_field((48, 48, 48), 9)
    outs = [torch.empty_like(x).pin_memory() for _ in range(8)]
    for o in outs:
        srv.submit(x, o)
    srv.close()                                      # returns: running work completes, rest cancelled


def test_requests_overlap_on_the_device_and_results_are_unchanged():
    """Several large requests submitted back to back run concurrently (the server's in-flight
    high-water mark is at least 2) and a field's result in that mix equals its result alone,
    bit for bit."""
    srv = eq.Server(32 << 30, max_inflight=4)
    probe = host_field((96, 80, 112), 31)
    alone = torch.empty_like(probe).pin_memory()
    n_alone, _ = srv.wait(srv.submit(probe, alone))
    big = [host_field((160, 144, 192), 40 + i) for i in range(5)]
    outs = [torch.empty_like(b).pin_memory() for b in big]
    mixed = torch.empty_like(probe).pin_memory()
    tickets = []
    for i, (b, o) in enumerate(zip(big, outs)):
        tickets.append(srv.submit(b, o))
        if i == 2:
            tp = srv.submit(probe, mixed)
    n_mix, _ = srv.wait(tp)
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    srv.close()
    assert st["inflight_peak"] >= 2, st
    assert st["completed"] == 7 and st["failed"] == 0 and st["queued"] == 0 and st["inflight"] == 0
    assert torch.equal(alone, mixed)
    assert n_alone == n_mix
    assert rel(outs[0].double().numpy(), oracle.project(big[0].double().numpy(), "ddo")) <= 2e-6


def test_cancel_a_queued_request_and_counters():
    srv = eq.Server(16 << 30, max_inflight=1)
    x = host_field((256, 256, 256), 12)                 # a few ms per request on one slot
    outs = [torch.empty_like(x).pin_memory() for _ in range(6)]
    tickets = [srv.submit(x, o) for o in outs]
    # the last request waits behind five others; its plan may be in the making for a moment
    # (EQ_ERR_BUSY), so ask again until it is withdrawn
    t0 = time.monotonic()
    while not srv.cancel(tickets[-1]):
        assert time.monotonic() - t0 < 5.0
        time.sleep(2e-4)
    with pytest.raises(eq.EqError) as ei:
        srv.poll(tickets[-1])
    assert ei.value.status == 7                      # the ticket is consumed
    for t in tickets[:-1]:
        srv.wait(t)
    with pytest.raises(eq.EqError) as ei:
        srv.cancel(tickets[0])                       # consumed by wait
    assert ei.value.status == 7
    st = srv.stats()
    srv.close()
    assert st["submitted"] == 6 and st["cancelled"] == 1 and st["completed"] == 5
    assert st["inflight_peak"] == 1 and st["plans_created"] >= 1 and st["plans_cached"] >= 1
    assert st["hbm_in_use"] <= st["hbm_budget"]
    for o in outs[1:5]:
        assert torch.equal(o, outs[0])


def test_fresh_shapes_build_plans_off_the_scheduler_and_the_cache_stays_bounded():
    """Every request a new grid: each gets its own plan (built by the plan thread), the idle-plan
    cache keeps at most 64, and the results still match the oracle."""
    srv = eq.Server(8 << 30, max_inflight=8)
    rng = np.random.Generator(np.random.PCG64(2105))
    shapes = set()
    while len(shapes) < 80:
        shapes.add(tuple(int(v) for v in rng.integers(8, 40, size=3)))
    shapes = sorted(shapes)
    jobs = []
    for i, sh in enumerate(shapes):
        x = host_field(sh, 500 + i)
        o = torch.empty_like(x).pin_memory()
        jobs.append((srv.submit(x, o), x, o))
    for k, (t, x, o) in enumerate(jobs):
        srv.wait(t)
        if k % 16 == 0:
            assert rel(o.double().numpy(), oracle.project(x.double().numpy(), "ddo")) <= 2e-6
    st = srv.stats()
    srv.close()
    assert st["plans_created"] == 80 and st["plans_reused"] == 0
    assert st["plans_cached"] <= 64 and st["plans_evicted"] >= 16
    assert st["completed"] == 80 and st["plan_create_seconds"] > 0
