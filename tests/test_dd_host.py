"""Double-float arithmetic of the FP64 path (csrc/eq_dd.cuh), checked on the host: compiled with
nvcc as host code (no GPU) and run against long-double references.  The format carries about 48
significant bits, so conversions are exact to 2^-48 relative, sums to a few units of 2^-48 of
|a| + |b|, products to a few units of 2^-48; values that came from a double round-trip exactly."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2105_01612_gb300", "csrc")
U48 = 2.0 ** -48


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("dd") / "dd_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "native", "dd_check.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.splitlines():
        k, *v = line.split()
        rows.setdefault(k, []).append(v)
    return rows


def test_conversions_and_round_trip(report):
    assert float(report["conv"][0][0]) <= 1.01 * U48
    assert float(report["trip"][0][0]) == 0.0


def test_sum_and_product_error_bounds(report):
    assert float(report["add"][0][0]) <= 4 * U48
    assert float(report["mul"][0][0]) <= 8 * U48


def test_special_values(report):
    for v, back in report["special"]:
        v, back = float(v), float(back)
        if v in (float("inf"), float("-inf")) or v == 0.0:
            assert back == v
        else:
            assert abs(back - v) <= U48 * abs(v)
    assert report["nan"][0][0] == "1"


def test_fp64_instruction_conversions(report):
    """The FP64-unit forms (used for the last pass's stores and re-read input): round to nearest
    for hi, the exact remainder rounded for lo (error below 2^-48 relative), the way back exact
    to one FP64 rounding (agreeing with the bit form); out of FP32's range they give infinities
    or zero."""
    assert float(report["conv2"][0][0]) <= U48
    assert float(report["agree"][0][0]) <= 2.0 ** -52
    got = {float(v): float(b) for v, b in report["special2"]}
    assert got[float("inf")] == float("inf")
    assert got[-1e300] == float("-inf")
    assert got[1e-300] == 0.0

