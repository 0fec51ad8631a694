"""The C ABI library builds, loads and exports every symbol include/lgs.h
declares; host-side argument checks reject bad calls before touching a GPU
(no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2511_16144_gb300 import build
    return build.build()


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^(?:lgs_status|size_t|int64_t|void|const char\*)\s+(\w+)\s*\(",
                                text, re.M)
    return names


def test_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert len(names) >= 8
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2511_16144_gb300 import lgs
    assert set(names) == set(lgs.exported_symbols())


def test_version_and_error_string(lib_path):
    from paper_2511_16144_gb300 import lgs
    lib = lgs.load()
    assert b"sm_103a" in lib.lgs_version()
    st = lib.gs_project(None, None, None, None, 10, None, 1, None, None, None)
    assert st == 1
    assert b"cams_host" in lib.lgs_last_error()


def test_host_argument_checks(lib_path):
    from paper_2511_16144_gb300 import lgs
    lib = lgs.load()
    cam = lgs.cameras([type("C", (), dict(fx=100.0, fy=100.0, cx=32.0, cy=24.0, width=64,
                                          height=48, viewmat=[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0],
                                          znear=0.2))()])
    fake = ctypes.c_void_p(0x1000)
    odd = ctypes.c_void_p(0x1004)
    # too many cameras
    assert lib.gs_project(fake, fake, fake, fake, 10, cam, 17, fake, fake, None) == 1
    # misaligned quaternion array
    assert lib.gs_project(fake, odd, fake, fake, 10, cam, 1, fake, fake, None) == 1
    assert b"misaligned" in lib.lgs_last_error()
    # feature width not a multiple of 8
    bg = (ctypes.c_float * 3)(0, 0, 0)
    assert lib.gs_render_fwd(fake, fake, fake, 10, cam, 1, fake, fake, 12, 0, bg, fake, fake,
                             fake, fake, fake, None, None) == 1
    assert b"feat_dim" in lib.lgs_last_error()
    # bin sort workspace too small
    assert lib.gs_bin_sort(fake, fake, 10, 1, 4, 3, 100, fake, fake, None, fake, fake, 16,
                           None) == 1
    assert b"workspace" in lib.lgs_last_error()
    assert lib.gs_bin_sort_workspace(1000, 2, 40, 30, 100000) > 0
    # an empty call is a no-op that succeeds
    assert lib.lgs_l1_loss(None, None, 0, 0, 1.0, None, None, None) == 0
    # a camera with a NaN or an infinite value is refused on the host
    for field, bad in (("cx", float("nan")), ("viewmat", [1, 0, 0, 0, 0, 1, 0, float("inf"),
                                                           0, 0, 1, 0])):
        kw = dict(fx=100.0, fy=100.0, cx=32.0, cy=24.0, width=64, height=48,
                  viewmat=[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], znear=0.2)
        kw[field] = bad
        badcam = lgs.cameras([type("C", (), kw)()])
        assert lib.gs_project(fake, fake, fake, fake, 10, badcam, 1, fake, fake, None) == 3
        assert b"non-finite" in lib.lgs_last_error()


def test_prune_host_argument_checks(lib_path):
    from paper_2511_16144_gb300 import lgs
    lib = lgs.load()
    fake = ctypes.c_void_p(0x1000)
    odd2 = ctypes.c_void_p(0x1002)
    ws = lib.gs_prune_workspace(1000)
    assert ws > 0 and lib.gs_compact_workspace(1000) > 0

    def call(n=1000, d=16, dtype=0, ws_bytes=ws, **kw):
        p = lgs.prune_params((0, 0, 0), (6, 6, 3), **kw)
        return lib.gs_prune(fake, fake, fake, fake, d, dtype, n, ctypes.byref(p), fake, fake, fake,
                            ws_bytes, None)

    assert call(k=0) == 1 and b"k must" in lib.lgs_last_error()
    assert call(k=17) == 1
    assert call(tau_dist=0.0) == 1 and b"tau_dist" in lib.lgs_last_error()
    assert call(min_opacity=1.0) == 1
    assert call(max_scale=0.0) == 1
    assert call(d=65) == 1 and b"feat_dim" in lib.lgs_last_error()
    assert call(dtype=2) == 1
    assert call(ws_bytes=16) == 1 and b"workspace" in lib.lgs_last_error()
    # a 1 mm grid over a 100 m box has too many cells
    p = lgs.prune_params((0, 0, 0), (100, 100, 100), tau_dist=0.001)
    assert lib.gs_prune(fake, fake, fake, fake, 16, 0, 1000, ctypes.byref(p), fake, fake, fake,
                        ws, None) == 1
    assert b"grid" in lib.lgs_last_error()
    assert lib.gs_gather_rows(fake, 10, 7, fake, fake, None) == 1
    assert lib.gs_gather_rows(odd2, 10, 8, fake, fake, None) == 1
    assert lib.gs_gather_rows(None, 0, 12, None, None, None) == 0
    assert lib.gs_compact_index(fake, 10, fake, fake, fake, 8, None) == 1


def test_status_codes_without_a_device(lib_path):
    """lgs_sync_status reports a failed synchronisation as LGS_ERR_CUDA (here:
    no device) with detail 0; the wait-limit hook takes any value."""
    from paper_2511_16144_gb300 import lgs
    lib = lgs.load()
    d = ctypes.c_int64(-7)
    assert lib.lgs_sync_status(None, ctypes.byref(d)) == 5
    assert d.value == 0
    assert lib.lgs_sync_status(None, None) == 5
    lib.lgs_set_sort_wait_limit(3)
    lib.lgs_set_sort_wait_limit(0)
    assert (lgs.OK, lgs.ERR_INVALID, lgs.ERR_CAPACITY, lgs.ERR_NONFINITE, lgs.ERR_TIMEOUT,
            lgs.ERR_CUDA) == (0, 1, 2, 3, 4, 5)
    text = open(os.path.join(ROOT, "include", "lgs.h")).read()
    for name, v in (("LGS_OK", 0), ("LGS_ERR_INVALID", 1), ("LGS_ERR_CAPACITY", 2),
                    ("LGS_ERR_NONFINITE", 3), ("LGS_ERR_TIMEOUT", 4), ("LGS_ERR_CUDA", 5)):
        assert re.search(rf"{name}\s*=\s*{v}\b", text), name


def test_decode_pack_argument_checks(lib_path):
    """The split distillation calls check their arguments on the host."""
    from paper_2511_16144_gb300 import lgs
    lib = lgs.load()
    w = lgs.AeWeights()
    for l in range(lgs.AE_LAYERS):
        w.W[l] = w.Wt[l] = w.b[l] = 0x1000
    fake = ctypes.c_void_p(0x1000)
    small = lib.ae_workspace_bytes(0, lgs.AE_DECODE)
    assert small > 0 and lib.ae_workspace_bytes(1000, lgs.AE_DECODE) > small
    assert lib.ae_decode_pack(ctypes.byref(w), fake, small // 2, None) == 1
    assert b"workspace" in lib.lgs_last_error()
    assert lib.ae_decode_pack(ctypes.byref(w), ctypes.c_void_p(0x1010), small, None) == 1
    # a target is required, and the workspace must hold P pixels' buffers
    assert lib.ae_decode_packed(ctypes.byref(w), fake, 1000, None, ctypes.c_float(1.0), fake, fake,
                                fake, lib.ae_workspace_bytes(1000, lgs.AE_DECODE), None) == 1
    assert lib.ae_decode_packed(ctypes.byref(w), fake, 1000, fake, ctypes.c_float(1.0), fake, fake,
                                fake, small, None) == 1
    assert b"workspace" in lib.lgs_last_error()
    # nothing to do for P = 0
    assert lib.ae_decode_packed(ctypes.byref(w), None, 0, None, ctypes.c_float(1.0), None, None,
                                None, 0, None) == 0
    # F_gt is read 32 bytes a lane: a target on a 16-byte (not 32-byte) boundary is refused
    big = lib.ae_workspace_bytes(1000, lgs.AE_DECODE)
    odd = ctypes.c_void_p(0x1010)
    assert lib.ae_decode(ctypes.byref(w), fake, 1000, odd, ctypes.c_float(1.0), fake, fake, None,
                         fake, big, None) == 1
    assert b"misaligned" in lib.lgs_last_error()
    assert lib.ae_decode_packed(ctypes.byref(w), fake, 1000, odd, ctypes.c_float(1.0), fake, fake,
                                fake, big, None) == 1
