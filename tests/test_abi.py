"""The C-ABI library builds, loads and exports every declared symbol (CPU only).

No compute call is made: only the host-side argument checks, which return
before any CUDA call, are exercised.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2102_12739_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "degrid.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for want in ("degrid_plan_create", "degrid_plan_destroy", "degrid_execute",
                 "grid_adjoint_execute", "degrid_get_status", "degrid_plan_set_tuning",
                 "degrid_status_string", "degrid_coords_execute", "degrid_pack_subgrids"):
        assert want in names
    # the Python binding binds exactly what the header declares
    assert set(names) == set(_native.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(build.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), f"{name} not exported by libdegrid.so"


def test_status_strings(lib):
    assert lib.degrid_status_string(0) == b"ok"
    assert b"offsets" in lib.degrid_status_string(_native.DG_ERR_OFFSETS)
    assert b"sm_103a" in lib.degrid_version()


def test_host_argument_checks_need_no_gpu(lib):
    P = ctypes.c_void_p
    g_uv = np.zeros((16384, 8))
    g_w = np.zeros((128, 4))
    h = P()
    a, b = g_uv.ctypes.data_as(P), g_w.ctypes.data_as(P)
    assert lib.degrid_plan_create(None, 512, 512, 4, a, 8, 16384, b, 4, 128, 0, 0) == _native.DG_ERR_ARG
    assert lib.degrid_plan_create(ctypes.byref(h), 512, 512, 4, None, 8, 16384, b, 4, 128, 0, 0) == _native.DG_ERR_ARG
    assert lib.degrid_plan_create(ctypes.byref(h), 512, 512, 4, a, 6, 16384, b, 4, 128, 0, 0) == _native.DG_ERR_UNSUPPORTED
    assert lib.degrid_plan_create(ctypes.byref(h), 512, 512, 4, a, 8, 10000, b, 4, 128, 0, 0) == _native.DG_ERR_ARG
    assert lib.degrid_plan_create(ctypes.byref(h), 512, 512, 2, a, 8, 16384, b, 4, 128, 0, 0) == _native.DG_ERR_UNSUPPORTED
    assert lib.degrid_plan_create(ctypes.byref(h), 512, 512, 4, a, 8, 16384, b, 4, 128, 7, 0) == _native.DG_ERR_DTYPE
    # an oversampled coordinate n * O beyond 2^31 does not fit the exact 32-bit snap
    assert lib.degrid_plan_create(ctypes.byref(h), 1 << 18, 8, 4, a, 8, 16384, b, 4, 128, 0, 0) == _native.DG_ERR_UNSUPPORTED
    assert lib.degrid_plan_create(ctypes.byref(h), 8, 1 << 18, 4, a, 8, 16384, b, 4, 128, 0, 0) == _native.DG_ERR_UNSUPPORTED
    assert h.value is None
    assert lib.degrid_execute(None, None, 1, None, None, None, None, 0, None) == _native.DG_ERR_ARG
    assert lib.grid_adjoint_execute(None, None, 1, None, None, 0, None, None, 0) == _native.DG_ERR_ARG
    assert lib.degrid_coords_execute(None, None, None, 0, None) == _native.DG_ERR_ARG
    assert lib.degrid_plan_set_compensated(None, 1) == _native.DG_ERR_ARG
    assert lib.degrid_plan_get_compensated(None, None) == _native.DG_ERR_ARG
    assert lib.degrid_plan_set_direct_runs(None, 9) == _native.DG_ERR_ARG
    assert lib.degrid_execute_host(None, 1, None, None, None, None, 0, None) == _native.DG_ERR_ARG
    # 2D G_uv plans: a table is required and its oversampling is bounded
    t2 = np.zeros((4, 4, 8, 8))
    c2 = t2.ctypes.data_as(P)
    assert lib.degrid_plan_create_2d(ctypes.byref(h), 64, 64, 4, None, 4, b, 4, 128, 0, 0) == _native.DG_ERR_ARG
    assert lib.degrid_plan_create_2d(ctypes.byref(h), 64, 64, 4, c2, 512, b, 4, 128, 0, 0) == _native.DG_ERR_ARG
    assert lib.degrid_plan_create_2d(ctypes.byref(h), 64, 64, 4, c2, 6, b, 4, 128, 0, 0) == _native.DG_ERR_ARG
    assert h.value is None
    assert lib.degrid_plan_get_direct_runs(None, None) == _native.DG_ERR_ARG
    assert lib.degrid_plan_set_tuning(None, 256, 8, 0) == _native.DG_ERR_ARG
    assert lib.degrid_get_status(None, None, None) == _native.DG_ERR_ARG
    assert lib.degrid_pack_subgrids(None, 0, 1, 4, None, None, None) == _native.DG_ERR_DTYPE
    assert lib.degrid_pack_subgrids(None, 1, -1, 4, None, None, None) == _native.DG_ERR_ARG


def test_header_constants_match_the_binding():
    text = open(HEADER).read()
    for name in ("DG_DIRECT_RUNS_NEVER", "DG_DIRECT_RUNS_SHORT", "DG_TABLE2D_MAX_OVERSAMPLE"):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(_native, name)
    assert re.search(r"#define\s+DG_DIRECT_RUNS_DEFAULT\s+DG_DIRECT_RUNS_NEVER", text)
    assert _native.DG_DIRECT_RUNS_DEFAULT == _native.DG_DIRECT_RUNS_NEVER


def test_library_variant_selection():
    # DEGRID_LIBRARY_VARIANT picks a variant build (the bounds-checking one);
    # an unknown name is refused; the product library is the default
    import subprocess
    import sys
    code = ("import paper_2102_12739_gb300._native as n; print(n.lib_path())")
    env = dict(os.environ, DEGRID_LIBRARY_VARIANT="bounds")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         cwd=ROOT, check=True).stdout.strip()
    assert out == build.variant_path("bounds") and "/bounds/" in out
    env["DEGRID_LIBRARY_VARIANT"] = "nonsense"
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    assert r.returncode != 0 and "unknown DEGRID_LIBRARY_VARIANT" in r.stderr
    env.pop("DEGRID_LIBRARY_VARIANT")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         cwd=ROOT, check=True).stdout.strip()
    assert out == build.LIB_PATH
