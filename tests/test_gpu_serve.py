"""The serving loop: results match the oracle, a field's result is the same alone and in a
mix of concurrent requests (bitwise: same kernels, fixed-order reductions), admission by HBM
footprint, error statuses."""
import math

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
