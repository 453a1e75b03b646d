"""The C ABI library loads and exports every symbol include/svr.h declares;
host-side argument checks answer without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "svr.h")


def _declared():
    text = open(HEADER).read()
    return re.findall(r"SVR_API\s+[^;{(]*?\b(svr_\w+)\s*\(", text)


@pytest.fixture(scope="module")
def lib():
    from paper_2412_04459_gb300 import build
    build.build()
    from paper_2412_04459_gb300 import _native
    return _native.lib()


def test_header_declares_the_four_path_calls():
    names = set(_declared())
    for n in ("svr_preprocess", "svr_bin_sort", "svr_render_fwd", "svr_render_bwd",
              "svr_workspace_size", "svr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2412_04459_gb300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(svr_\w+)", out))
    declared = set(_declared())
    assert declared, "no declarations parsed"
    assert declared <= exported, declared - exported
    # nothing but the declared C ABI is exported under the svr_ prefix
    assert exported <= declared, exported - declared
    for name in declared:
        assert hasattr(lib, name)


def test_bindings_cover_the_header(lib):
    from paper_2412_04459_gb300 import _native
    assert set(_native.SIGNATURES) == set(_declared())


def test_struct_sizes_match_c(lib, tmp_path):
    """ctypes struct layouts equal the C compiler's (sizeof of each struct)."""
    from paper_2412_04459_gb300 import _native as N
    src = tmp_path / "sz.c"
    src.write_text('#include "svr.h"\n#include <stdio.h>\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(svr_camera),sizeof(svr_params),sizeof(svr_scene),sizeof(svr_frame),'
                   'sizeof(svr_buffers),__builtin_offsetof(svr_frame, offsets),sizeof(svr_render_extras));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(N.SvrCamera), ctypes.sizeof(N.SvrParams), ctypes.sizeof(N.SvrScene),
                     ctypes.sizeof(N.SvrFrame), ctypes.sizeof(N.SvrBuffers), N.SvrFrame.offsets.offset,
                     ctypes.sizeof(N.SvrRenderExtras)]


def test_workspace_size_host_checks(lib):
    import synth
    from paper_2412_04459_gb300 import _native as N
    from paper_2412_04459_gb300.raster import camera_struct, params_struct
    cam = camera_struct(synth.dense_view_camera())
    p = params_struct(K=3)
    n1 = lib.svr_workspace_size(1000, 5000, N.ref(cam), N.ref(p))
    n2 = lib.svr_workspace_size(2000, 5000, N.ref(cam), N.ref(p))
    n3 = lib.svr_workspace_size(1000, 50000, N.ref(cam), N.ref(p))
    assert 0 < n1 < n2 and n1 < n3 and n1 % 256 == 0
    assert lib.svr_workspace_size(-1, 10, N.ref(cam), N.ref(p)) == 0
    assert lib.svr_workspace_size((1 << 29) + 1, 10, N.ref(cam), N.ref(p)) == 0
    assert lib.svr_workspace_size(10, 10, None, N.ref(p)) == 0
    bad = params_struct(K=4)
    assert lib.svr_workspace_size(10, 10, N.ref(cam), N.ref(bad)) == 0
    bad = params_struct(K=1, tile=12)
    assert lib.svr_workspace_size(10, 10, N.ref(cam), N.ref(bad)) == 0
    big = camera_struct(synth.look_at((0, 0, -2), (0, 0, 0), (0, 1, 0), 50, 4112, 4112))
    assert lib.svr_workspace_size(10, 10, N.ref(big), N.ref(p)) == 0   # > 2^16 tiles


def test_argument_errors_are_reported_before_any_launch(lib):
    """Null pointers and out-of-range sizes come back as status codes with a
    message; nothing reaches the device (no GPU needed)."""
    import synth
    from paper_2412_04459_gb300 import _native as N
    from paper_2412_04459_gb300.raster import camera_struct, params_struct
    cam = camera_struct(synth.dense_view_camera())
    p = params_struct(K=1)
    fr = N.SvrFrame()
    sc = N.SvrScene()
    sc.world_size = 1.0
    sc.max_level = 5
    sc.n_vox = 10
    assert lib.svr_preprocess(None, N.ref(sc), N.ref(cam), N.ref(p), None, 0, 0, None) == N.SVR_ERR_INVALID
    assert lib.svr_preprocess(N.ref(fr), N.ref(sc), N.ref(cam), N.ref(p), None, 0, 0, None) == N.SVR_ERR_INVALID
    assert b"null scene array" in lib.svr_last_error()
    sc.n_vox = (1 << 29) + 1
    assert lib.svr_preprocess(N.ref(fr), N.ref(sc), N.ref(cam), N.ref(p), None, 0, 0, None) == N.SVR_ERR_LIMIT
    sc.n_vox = 0
    sc.max_level = 17
    assert lib.svr_preprocess(N.ref(fr), N.ref(sc), N.ref(cam), N.ref(p), None, 0, 0, None) == N.SVR_ERR_INVALID
    sc.max_level = 5
    ws = ctypes.c_void_p(0x1001)   # misaligned, never dereferenced
    assert lib.svr_preprocess(N.ref(fr), N.ref(sc), N.ref(cam), N.ref(p), ws, 1 << 20, 0, None) == N.SVR_ERR_INVALID
    assert b"256-byte" in lib.svr_last_error()
    ws = ctypes.c_void_p(0x100000)  # aligned but too small, never dereferenced
    assert lib.svr_preprocess(N.ref(fr), N.ref(sc), N.ref(cam), N.ref(p), ws, 16, 0, None) == N.SVR_ERR_INVALID
    assert b"workspace" in lib.svr_last_error()
    # calls that need an earlier stage refuse an empty frame
    fr = N.SvrFrame()
    assert lib.svr_bin_sort(N.ref(fr), None, None) == N.SVR_ERR_INVALID
    assert lib.svr_render_fwd(N.ref(fr), None, None, None, None, None, None) == N.SVR_ERR_INVALID
    assert lib.svr_render_bwd(N.ref(fr), None, None, None, None, None, None, None, None) == N.SVR_ERR_INVALID
    assert lib.svr_frame_buffers(N.ref(fr), None) == N.SVR_ERR_INVALID


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libsvr.so the binding raises: there is no CPU fallback."""
    from paper_2412_04459_gb300 import _native
    monkeypatch.setattr(_native, "_LIB", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "libsvr.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native.lib()
