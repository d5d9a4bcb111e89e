"""The C-ABI library builds, loads and exports every entry point declared in include/*.h; host
logic that needs no GPU (argument validation, defaults, struct layout)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared_symbols():
    names = set()
    for f in os.listdir(INCLUDE):
        if f.endswith(".h"):
            src = open(os.path.join(INCLUDE, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(eq_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2105_01612_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2105_01612_gb300 import _lib
    declared = _declared_symbols()
    assert "eq_project" in declared and "eq_plan_create" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(eq_[a-z0-9_]+)$", out, flags=re.M))
    assert declared <= exported, declared - exported
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert declared == bound, declared ^ bound
    for name in declared:
        getattr(lib, name)


def test_struct_layout_matches_the_header(tmp_path):
    from paper_2105_01612_gb300._lib import EqNorms, EqPlanOpts
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "eq.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(eq_plan_opts),"
        " offsetof(eq_plan_opts, nyq), offsetof(eq_plan_opts, target), sizeof(eq_norms_t),"
        " offsetof(eq_norms_t, resid_linf), offsetof(eq_norms_t, flags),"
        " offsetof(eq_norms_t, div_out_l2)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(EqPlanOpts), EqPlanOpts.nyq.offset, EqPlanOpts.target.offset,
            ctypes.sizeof(EqNorms), EqNorms.resid_linf.offset, EqNorms.flags.offset,
            EqNorms.div_out_l2.offset]
    assert got == want


def test_defaults_and_argument_validation_without_a_gpu(lib):
    from paper_2105_01612_gb300._lib import (EqPlanOpts, EQ_ERR_INVALID, EQ_OP_DDO, EQ_NYQ_KEEP,
                                            EQ_TARGET_EQUILIBRIUM)
    o = EqPlanOpts()
    lib.eq_plan_opts_default(ctypes.byref(o))
    assert (o.op, o.hx, o.hy, o.hz, o.nyq, o.want_linf, o.graph, o.target) == \
        (EQ_OP_DDO, 1.0, 1.0, 1.0, EQ_NYQ_KEEP, 1, 1, EQ_TARGET_EQUILIBRIUM)
    bad = EqPlanOpts()
    lib.eq_plan_opts_default(ctypes.byref(bad))
    bad.target = 5
    assert lib.eq_plan_create(64, 64, 64, 0, 1, ctypes.byref(bad), ctypes.byref(ctypes.c_void_p())) \
        == EQ_ERR_INVALID
    assert b"target" in lib.eq_last_error()
    h = ctypes.c_void_p()
    # unsupported length, bad batch, bad spacing, NULL out: rejected before any CUDA call
    assert lib.eq_plan_create(2048, 64, 64, 0, 1, None, ctypes.byref(h)) == EQ_ERR_INVALID
    assert b"unsupported" in lib.eq_last_error()
    assert lib.eq_plan_create(64, 64, 601, 0, 1, None, ctypes.byref(h)) == EQ_ERR_INVALID
    dims = (ctypes.c_int * 6)(16, 16, 16, 8, 0, 8)
    assert lib.eq_plan_create_varlen(dims, 2, 0, None, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_plan_create_varlen(None, 2, 0, None, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_plan_create(64, 64, 64, 0, 0, None, ctypes.byref(h)) == EQ_ERR_INVALID
    o.hx = -1.0
    assert lib.eq_plan_create(64, 64, 64, 0, 1, ctypes.byref(o), ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_plan_create(64, 64, 64, 0, 1, None, None) == EQ_ERR_INVALID
    assert lib.eq_plan_create(64, 64, 64, 7, 1, None, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_project(None, None, None, None) == EQ_ERR_INVALID
    assert lib.eq_norms(None, None) == EQ_ERR_INVALID
    assert lib.eq_plan_workspace_bytes(None) == 0
    lib.eq_plan_destroy(None)
    # serving: argument checks that precede any CUDA call
    assert lib.eq_server_create(0, 4, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_server_create(1 << 30, 0, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_serve_submit(None, 8, 8, 8, 0, None, None, None, None) == EQ_ERR_INVALID
    assert lib.eq_serve_poll(None, 1, 0, None, None) == EQ_ERR_INVALID
    lib.eq_server_destroy(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2105_01612_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
                assert "oracle/" not in txt, f


def test_grain_map_validation_without_a_gpu(lib):
    from paper_2105_01612_gb300._lib import EQ_ERR_INVALID
    h = ctypes.c_void_p()
    ids = (ctypes.c_int * 8)(0, 1, 2, 3, 0, 1, 2, 9)
    assert lib.eq_grains_create(ids, 2, 2, 2, 4, ctypes.byref(h)) == EQ_ERR_INVALID
    assert b"outside" in lib.eq_last_error()
    assert lib.eq_grains_create(None, 2, 2, 2, 4, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_grains_create(ids, 2, 2, 2, 0, ctypes.byref(h)) == EQ_ERR_INVALID
    assert lib.eq_grain_average(None, 0, 1, None, None, None, None) == EQ_ERR_INVALID
    lib.eq_grains_destroy(None)


def test_new_entry_points_reject_bad_arguments_without_a_gpu(lib):
    from paper_2105_01612_gb300._lib import EQ_ERR_INVALID
    assert lib.eq_project_hodge(None, None, None, None, None) == EQ_ERR_INVALID
    assert lib.eq_project_padded(None, 8, 8, 8, None, None, None) == EQ_ERR_INVALID
    assert lib.eq_project_host_async(None, None, None, None) == EQ_ERR_INVALID
    assert b"NULL" in lib.eq_last_error()


def test_wait_selftest_rejects_bad_arguments_without_a_gpu(lib):
    from paper_2105_01612_gb300._lib import EQ_ERR_INVALID
    assert lib.eq_selftest_wait_timeout(None, 1024, None) == EQ_ERR_INVALID
    assert b"NULL plan" in lib.eq_last_error()


def test_server_stats_layout_matches_the_header(tmp_path):
    from paper_2105_01612_gb300._lib import EqServerStats
    src = tmp_path / "stats.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "eq.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(eq_server_stats_t),"
        " offsetof(eq_server_stats_t, plan_create_seconds), offsetof(eq_server_stats_t, queued),"
        " offsetof(eq_server_stats_t, hbm_in_use_peak), offsetof(eq_server_stats_t, plans_cached));"
        " return 0;}\n")
    exe = tmp_path / "stats"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(EqServerStats), EqServerStats.plan_create_seconds.offset,
            EqServerStats.queued.offset, EqServerStats.hbm_in_use_peak.offset,
            EqServerStats.plans_cached.offset]
    assert got == want
