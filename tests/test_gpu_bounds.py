"""The bounds-checked build (libeq_check.so, device-side index checks on the global loads and
stores of the plain, warp-per-row and runtime-length passes and on the runtime-length shared
work buffers): projections of odd, prime and uneven grids raise no out-of-range flag and still
match the oracle.  Run in a child process, since the library choice is made when it is first
loaded (EQ_BOUNDS_CHECK=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import math, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle
from fieldgen import voronoi_stress_field
import paper_2105_01612_gb300 as eq
from paper_2105_01612_gb300 import _lib
assert _lib.lib_path().endswith("libeq_check.so"), _lib.lib_path()
W = np.array([1.0, 1, 1, 2, 2, 2]).reshape(6, 1, 1, 1)
def rel(a, b):
    return math.sqrt(float((W * (a - b) ** 2).sum() / (W * b ** 2).sum()))
# (nz, ny, nx): primes, odd sizes, the warp-row Bluestein lengths, powers of two (fixed path)
shapes = [(7, 11, 13), (5, 31, 97), (3, 2, 131), (13, 17, 200), (1, 1, 1), (2, 3, 5),
          (16, 8, 256), (8, 4, 512), (32, 32, 32)]
for i, sh in enumerate(shapes):
    s = voronoi_stress_field(sh, 5, 100.0, 10.0, 70 + i).numpy()
    for dt, tol in ((torch.float32, 2e-6), (torch.float64, 1e-12)):
        x = torch.as_tensor(s).to(dt).cuda()
        out, nrm = eq.project(x, op="ddo")
        torch.cuda.synchronize()
        ref = oracle.project(x.double().cpu().numpy(), "ddo")
        err = rel(out.double().cpu().numpy(), ref)
        assert err <= tol, (sh, dt, err)
# an uneven batch in one plan (runtime-length path, one launch per pass)
dims = [(13, 11, 7), (200, 9, 5), (64, 3, 17), (131, 2, 2)]
fields = [voronoi_stress_field((nz, ny, nx), 4, 80.0, 5.0, 90 + k).float().cuda()
          for k, (nx, ny, nz) in enumerate(dims)]
plan = eq.VarlenPlan(dims, torch.float32, "ddo")
flat = plan.pack(fields)
out = plan.unpack(plan.project(flat))
plan.norms()
for f, o in zip(fields, out):
    ref = oracle.project(f.double().cpu().numpy(), "ddo")
    assert rel(o.double().cpu().numpy(), ref) <= 2e-6
print("bounds-checked projections ok")
'''


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def test_bounds_checked_build_raises_no_flag_on_odd_prime_and_uneven_grids():
    env = dict(os.environ, EQ_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds-checked projections ok" in r.stdout
