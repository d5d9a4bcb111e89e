"""Failure detection of the bounded waits, without a GPU fault: the self-test kernel runs the same
bounded mbarrier wait as the TMA passes on a barrier nothing completes, with a short limit; the
host must see EQ_ERR_TIMEOUT at eq_norms, the flag must clear, and the plan must keep working."""
import time

import numpy as np
import pytest
import torch

import oracle
from fieldgen import voronoi_stress_field
import paper_2105_01612_gb300 as eq
from paper_2105_01612_gb300._lib import EQ_ERR_TIMEOUT, EqError

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_wait_runs_out_is_reported_and_cleared(dtype):
    shape = (32, 32, 32)
    s = voronoi_stress_field(shape, 9, 100.0, 5.0, 2105, dtype=torch.float64).numpy()
    if dtype == torch.float32:
        s = s.astype(np.float32).astype(np.float64)
    x = torch.as_tensor(s).to(dtype).cuda().unsqueeze(0)
    plan = eq.Plan(32, 32, 32, dtype, 1, "ddo")
    try:
        plan.project(x)
        before = plan.norms()[0]

        t0 = time.perf_counter()
        plan.selftest_wait_timeout(polls=4096)
        with pytest.raises(EqError) as info:
            plan.norms()
        assert info.value.status == EQ_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5.0          # the wait ended by itself

        # the flag is cleared and the context is intact: the next projection is the oracle's
        out = plan.project(x)
        after = plan.norms()[0]
        assert after["resid_l2"] == before["resid_l2"]
        ref = oracle.project(s, "ddo")
        assert rel(out[0].double().cpu().numpy(), ref) <= (2e-6 if dtype == torch.float32 else 1e-12)
    finally:
        plan.close()


def test_runtime_length_plans_have_no_waits_to_test():
    plan = eq.Plan(12, 10, 9, torch.float32, 1, "ddo")
    try:
        with pytest.raises(EqError):
            plan.selftest_wait_timeout()
    finally:
        plan.close()
