"""The C ABI without a GPU: libsdgr.so loads, exports every function that
include/sdgr.h declares, and rejects bad arguments on the host (no compute
call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sdgr.h")).read()
    return sorted(set(re.findall(r"^(?:sdgr_status|const char \*|int64_t|int32_t|size_t)\s*(sdgr_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def L():
    from paper_2506_21633_b300 import build
    build.build()
    from paper_2506_21633_b300 import _lib
    return _lib


def test_exports_match_header(L):
    names = _declared()
    assert len(names) >= 12
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r"\bT %s$" % n, out, re.M), n


def test_status_strings(L):
    for code in range(6):
        assert L.status_string(code)
    assert L.status_string(99) == "unknown status"


def test_host_validation(L):
    import sdgr_scenes as sc
    lib = L.lib()
    good = [sc.make_view(0.0, 45.0, 0.1, 0.1, 64, 48)]
    offs = L.make_offsets([0, 100])
    caps = L.sdgr_caps_for(L.make_views(good), 1, offs, 1, 1000)
    assert caps.max_view_gauss == 100 and caps.max_pixels == 64 * 48 and caps.max_tiles == 4 * 3
    assert L.sdgr_workspace_size(L.make_cfg(), caps) > 0
    for bad in [dict(theta=0.0), dict(theta=1.5708), dict(NA=0), dict(dR=-1.0), dict(dA=0.0), dict(scene=1)]:
        v = dict(good[0], **bad)
        with pytest.raises(L.SdgrError) as e:
            L.sdgr_caps_for(L.make_views([v]), 1, offs, 1, 1000)
        assert e.value.code == L.SDGR_ERR_INVALID
    with pytest.raises(L.SdgrError):
        L.sdgr_caps_for(L.make_views(good), 1, L.make_offsets([0, 10, 5]), 2, 0)
    with pytest.raises(L.SdgrError):
        L.sdgr_workspace_size(L.make_cfg(cutoff_K=-1.0), caps)
    with pytest.raises(L.SdgrError):
        L.sdgr_workspace_size(L.make_cfg(norm_mode=3), caps)
    # NULL / misaligned buffers are refused before any CUDA call
    assert lib.sdgr_ws_create(ctypes.byref(ctypes.c_void_p()), None, 1 << 30, ctypes.byref(L.make_cfg()),
                              ctypes.byref(caps)) == L.SDGR_ERR_INVALID
    assert lib.sdgr_ws_create(ctypes.byref(ctypes.c_void_p()), ctypes.c_void_p(4096 + 8), 1 << 30,
                              ctypes.byref(L.make_cfg()), ctypes.byref(caps)) == L.SDGR_ERR_INVALID
    assert lib.sdgr_ws_create(ctypes.byref(ctypes.c_void_p()), ctypes.c_void_p(4096), 16,
                              ctypes.byref(L.make_cfg()), ctypes.byref(caps)) == L.SDGR_ERR_INVALID
    assert lib.sdgr_preprocess(None, None, offs, 1, L.make_views(good), 1, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_bin_sort(None, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_render_fwd(None, None, None, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_render_bwd(None, None, None, 0, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_count_pairs(None, None, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_launch_count() == 0
    assert lib.sdgr_read_status(None, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_ws_destroy(None) == L.SDGR_ERR_INVALID
    lr = (ctypes.c_float * 5)(1, 1, 1, 1, 1)
    assert lib.sdgr_adam_step(None, None, None, None, -1, lr, 0.9, 0.999, 1e-8, 1, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_adam_step(None, None, None, None, 10, lr, 0.9, 0.999, 1e-8, 0, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_adam_step(ctypes.c_void_p(8), ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(48), 10,
                              lr, 0.9, 0.999, 1e-8, 1, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_l1_loss(None, None, 10, None, None, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_set_stage_batch(None, 0, 256) == L.SDGR_ERR_INVALID
    assert lib.sdgr_device_selfcheck(None, None) == L.SDGR_ERR_INVALID
    assert lib.sdgr_device_selfcheck(ctypes.c_void_p(4096 + 2), None) == L.SDGR_ERR_INVALID


def test_stage_batch_options(L):
    """Every raster kernel lists its staging batch sizes, the default first:
    multiples of the threads of a CTA (each thread stages whole records);
    an unknown kernel has none."""
    for k, name in enumerate(L.RASTER_KERNELS):
        opts = L.sdgr_stage_batch_options(name)
        assert opts and opts == L.sdgr_stage_batch_options(k)
        assert len(set(opts)) == len(opts)
        assert all(nb % 128 == 0 and 128 <= nb <= 1024 for nb in opts)
    assert L.sdgr_stage_batch_options(1) == (512, 256)
    assert L.lib().sdgr_stage_batch_options(4, None, 0) == 0
    assert L.lib().sdgr_stage_batch_options(-1, None, 0) == 0


def test_product_does_not_import_oracle():
    """The package never imports, links or calls the oracle."""
    pkg = os.path.join(ROOT, "paper_2506_21633_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "liboracle" not in text, f
