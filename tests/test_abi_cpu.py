"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol the header
declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gabsplat.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:gs_status|size_t|const char\*|void)\s+(gabsplat_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def B():
    from paper_2508_05343_b300 import build
    build.build()
    from paper_2508_05343_b300 import binding
    return binding


def test_header_declares_the_four_stages():
    names = declared_functions()
    for stage in ("gabsplat_preprocess", "gabsplat_bin_sort", "gabsplat_render_fwd", "gabsplat_render_bwd"):
        assert stage in names


def test_every_declared_symbol_is_exported(B):
    for name in declared_functions():
        assert hasattr(B.lib, name), name
        assert name in B.SIGNATURES, name


def test_version_and_status_strings(B):
    assert "sm_103a" in B.gabsplat_version()
    assert B.gabsplat_status_string(B.GS_ERR_CAPACITY) == "pair capacity exceeded"
    assert B.gabsplat_status_string(99) == "unknown status"


def test_workspace_size_arithmetic(B):
    s1 = B.gabsplat_workspace_size(1000, 4, 3, 128, 128, 10000)
    s2 = B.gabsplat_workspace_size(1000, 4, 3, 128, 128, 20000)
    assert s1 > 0 and s2 > s1
    assert s2 - s1 >= 10000 * 16           # two 8-byte pair buffers (emission / sort ping-pong) per pair
    assert B.gabsplat_workspace_size(-1, 4, 3, 128, 128, 10) == 0
    assert B.gabsplat_workspace_size(10, 9, 3, 128, 128, 10) == 0       # K > GS_MAX_K
    assert B.gabsplat_workspace_size(10, 4, 4, 128, 128, 10) == 0       # SH degree > 3
    assert B.gabsplat_workspace_size(10, 4, 3, 0, 128, 10) == 0
    assert B.gabsplat_workspace_size(10, 4, 3, 128, 128, 1 << 32) == 0


def test_invalid_arguments_rejected_on_host(B):
    lib = B.lib
    f = B.gs_frame()
    f.n, f.K, f.sh_degree, f.width, f.height, f.pair_capacity = 10, 2, 0, 64, 64, 1000
    f.ws, f.ws_bytes = None, 0
    assert lib.gabsplat_bin_sort(C.byref(f), None) == B.GS_ERR_INVALID_ARG
    assert lib.gabsplat_render_fwd(C.byref(f), None, None, None) == B.GS_ERR_INVALID_ARG
    assert lib.gabsplat_render_bwd(None, None, None, None) == B.GS_ERR_INVALID_ARG
    assert lib.gabsplat_render_bwd_2d_zero(C.byref(f), None, None, None) == B.GS_ERR_INVALID_ARG
    assert lib.gabsplat_preprocess_bwd_prezeroed(None, None, None) == B.GS_ERR_INVALID_ARG
    f.ws = 0x1000 + 8                       # misaligned (never dereferenced)
    assert lib.gabsplat_bin_sort(C.byref(f), None) == B.GS_ERR_WORKSPACE
    f.ws, f.ws_bytes = 0x100000, 16         # too small (never dereferenced)
    assert lib.gabsplat_bin_sort(C.byref(f), None) == B.GS_ERR_WORKSPACE
    f.ws_bytes = B.gabsplat_workspace_size(10, 2, 0, 64, 64, 1000)
    f.storage = 7                           # unknown storage type
    assert lib.gabsplat_bin_sort(C.byref(f), None) == B.GS_ERR_INVALID_ARG
    f.storage = B.GS_F32
    cam, cfg, pr = B.gs_camera(), B.make_config(), B.gs_prims()
    pr.n, pr.K, pr.sh_degree = 11, 2, 0     # n does not match the frame
    assert lib.gabsplat_preprocess(C.byref(f), C.byref(pr), C.byref(cam), C.byref(cfg), None) == B.GS_ERR_INVALID_ARG
    pr.n = 10
    pr.storage = B.GS_BF16                  # storage differs from the frame's
    assert lib.gabsplat_preprocess(C.byref(f), C.byref(pr), C.byref(cam), C.byref(cfg), None) == B.GS_ERR_INVALID_ARG
    pr.storage = B.GS_F32
    cam.width, cam.height = 64, 64          # fx = 0: invalid camera (checked before any launch)
    pr.means = pr.scales = pr.quats = pr.opacity = pr.sh = pr.freqs = pr.weights = 0x100000
    assert lib.gabsplat_preprocess(C.byref(f), C.byref(pr), C.byref(cam), C.byref(cfg), None) == B.GS_ERR_INVALID_ARG
    cam.fx = cam.fy = 50.0
    cam.znear, cam.zfar = 0.2, 100.0
    cfg.flags = 2                           # unknown flag (bit 0 is the z-attenuation variant)
    assert lib.gabsplat_preprocess(C.byref(f), C.byref(pr), C.byref(cam), C.byref(cfg), None) == B.GS_ERR_INVALID_ARG
    img = C.c_void_p(0x100000)
    assert lib.gabsplat_loss(img, img, 0, 0, img, img, img, None) == B.GS_ERR_INVALID_ARG
    assert lib.gabsplat_loss(img, img, 10, 7, img, img, img, None) == B.GS_ERR_INVALID_ARG
