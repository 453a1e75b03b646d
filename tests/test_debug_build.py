"""The SVR_DEBUG build (libsvr_debug.so): device-side index checks that count
a failed check, keep the first one's site, index and bound, skip the access
and never trap; svr_debug_report() reads and clears the report.

CPU: both libraries build and export the same C ABI, each reports which build
it is, and the release report is all zeros.  GPU (with SVR_DEBUG=1, which
loads the debug library): a tile range whose end lies one past the pair
capacity is caught by the render's check and reported; every other GPU test
then runs with an empty report asserted after it (tests/conftest.py)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "svr.h")
SITE_RANGE = 2


def _exports(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    return set(re.findall(r"\bT\s+(svr_\w+)", out))


@pytest.fixture(scope="module")
def libs():
    from paper_2412_04459_gb300 import build
    rel = ctypes.CDLL(build.build())
    dbg = ctypes.CDLL(build.build(debug=True))
    for L in (rel, dbg):
        L.svr_debug_build.restype = ctypes.c_int
        L.svr_debug_report.restype = ctypes.c_int
        L.svr_debug_report.argtypes = [ctypes.c_void_p]
    return rel, dbg


def test_both_builds_export_the_same_abi(libs):
    from paper_2412_04459_gb300 import build
    rel, dbg = libs
    declared = set(re.findall(r"SVR_API\s+[^;{(]*?\b(svr_\w+)\s*\(", open(HEADER).read()))
    assert "svr_debug_report" in declared and "svr_debug_build" in declared
    assert _exports(build.LIB) == declared
    assert _exports(build.LIB_DEBUG) == declared


def test_each_build_says_which_it_is(libs):
    rel, dbg = libs
    assert rel.svr_debug_build() == 0
    assert dbg.svr_debug_build() == 1


def test_release_report_is_empty_and_checks_its_argument(libs):
    rel, _ = libs
    out = (ctypes.c_uint64 * 4)(7, 7, 7, 7)
    assert rel.svr_debug_report(out) == 0
    assert list(out) == [0, 0, 0, 0]
    assert rel.svr_debug_report(None) == 1          # SVR_ERR_INVALID


def test_binding_selects_the_library_from_the_environment():
    code = ("import paper_2412_04459_gb300._native as N, os; "
            "print(os.path.basename(N.LIB_PATH), N.DEBUG)")
    env = dict(os.environ, PYTHONPATH=ROOT)
    for val, want in (("1", "libsvr_debug.so True"), ("0", "libsvr.so False"), ("", "libsvr.so False")):
        env["SVR_DEBUG"] = val
        out = subprocess.run(["python", "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                             check=True).stdout.strip()
        assert out == want, (val, out)


@pytest.mark.gpu
def test_out_of_range_tile_range_is_reported_not_faulted():
    """Planted in the debug build only: after the sort, one tile's range end
    is set to capacity + 1 (past the pairs the workspace holds, still inside
    the workspace for every read it could cause).  The render's range check
    rejects it, the tile renders empty, and the report names the check."""
    from paper_2412_04459_gb300 import _native as N
    if not N.DEBUG:
        pytest.skip("needs the SVR_DEBUG build (SVR_DEBUG=1)")
    import torch
    import synth
    from paper_2412_04459_gb300 import DeviceScene, Frame
    from paper_2412_04459_gb300.raster import _device_copy
    sc = synth.dense_scene(4, seed=1)
    cam = synth.dense_view_camera(64, 64)
    fr = Frame(DeviceScene.from_host(sc), cam, K=1, t_stop=1e-4)
    fr.render()
    assert N.debug_report()[0] == 0
    ins = fr.inspect()
    lens = ins["ranges"][:, 1].astype(np.int64) - ins["ranges"][:, 0]
    g = int(np.argmax((lens > 0) & (lens <= 1024)))
    assert 0 < lens[g] <= 1024
    cap = int(fr.pair_capacity)
    bad = torch.tensor([int(ins["ranges"][g, 0]), cap + 1], dtype=torch.int32, device="cuda")
    _device_copy(int(fr.buffers().ranges) + 8 * g, bad.data_ptr(), 8)
    out = fr.forward()
    torch.cuda.synchronize()
    count, site, index, bound = N.debug_report()
    assert count >= 1 and site == SITE_RANGE and index == cap + 1 and bound == cap + 1, (count, site, index, bound)
    assert N.debug_report() == (0, 0, 0, 0)          # read and cleared
    assert torch.isfinite(out["rgb"]).all()
