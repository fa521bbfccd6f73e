"""The allocation-free forward entry point, called through the C ABI.

Some callers cannot allocate device memory themselves (a plugin whose host
application owns every device allocation, a real-time loop that must not
allocate once running); sdgr_render_fwd_noalloc serves them from a fixed
scratch array inside the library.  Its images and intensities must match
the workspace-based entry points (sdgr_preprocess + sdgr_bin_sort +
sdgr_render_fwd) within the forward tolerance, on two calls in a row with
different scenes and views (the second call reuses the scratch the first
one left behind).  Collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

import sdgr_scenes as sc
from gpu_helpers import IMG_TOL

pytestmark = pytest.mark.gpu


def _noalloc(params32, views, cfg):
    import torch
    from paper_2506_21633_b300 import _lib as L
    p = torch.from_numpy(params32).cuda().contiguous()
    npix = sum(v["NA"] * v["NR"] for v in views)
    images = torch.full((npix,), -1.0, dtype=torch.float32, device="cuda")
    inten = torch.full((max(1, len(views) * params32.shape[0]),), -1.0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = L.lib().sdgr_render_fwd_noalloc(ctypes.c_void_p(p.data_ptr() if params32.shape[0] else None),
                                           params32.shape[0], L.make_views(views), len(views), ctypes.byref(cfg),
                                           ctypes.c_void_p(images.data_ptr()), ctypes.c_void_p(inten.data_ptr()),
                                           ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return code, images.cpu().numpy(), inten.cpu().numpy()[:len(views) * params32.shape[0]]


def _workspace_path(params32, views):
    import torch
    from paper_2506_21633_b300.render import Renderer
    r = Renderer()
    p = torch.from_numpy(params32).cuda().contiguous()
    r.prepare(p, views)
    inten = torch.zeros(max(1, len(views) * params32.shape[0]), dtype=torch.float32, device="cuda")
    img = r.forward(intensity=inten)
    torch.cuda.synchronize()
    return img.cpu().numpy(), inten.cpu().numpy()[:len(views) * params32.shape[0]]


def test_noalloc_matches_workspace_path_twice():
    from paper_2506_21633_b300 import _lib as L
    cfg = L.make_cfg()
    cases = [
        (sc.vehicle_box_scene(6000, seed=61, extent=(3.0, 2.0, 1.5), log_s_mean=math.log(0.06),
                              center=(0.0, 0.0, 0.5)),
         sc.random_views(3, seed=62, size=160, res=0.03, center=(0.0, 0.0, 0.5))),
        (sc.random_cube_scene(2000, half=2.0, s_lo=0.03, s_hi=0.2, seed=63),
         [sc.make_view(40.0, 35.0, 0.03, 0.035, 200, 150), sc.make_view(250.0, 55.0, 0.04, 0.03, 97, 131)]),
    ]
    for params, views in cases:
        p32 = np.ascontiguousarray(params, dtype=np.float32)
        code, img, inten = _noalloc(p32, views, cfg)
        assert code == L.SDGR_OK, L.status_string(code)
        ref_img, ref_inten = _workspace_path(p32, views)
        off = 0
        for v in views:
            n = v["NA"] * v["NR"]
            a, b = img[off:off + n], ref_img[off:off + n]
            assert np.abs(a - b).max() <= IMG_TOL * np.abs(b).max()
            off += n
        assert np.abs(inten - ref_inten).max() <= IMG_TOL * np.abs(ref_inten).max()


def test_noalloc_rejects_oversize():
    from paper_2506_21633_b300 import _lib as L
    cfg = L.make_cfg()
    too_many = np.zeros((16385, 12), dtype=np.float32)
    too_many[:, 8] = 1.0
    code, _, _ = _noalloc(too_many, [sc.make_view(0.0, 45.0, 0.1, 0.1, 32, 32)], cfg)
    assert code == L.SDGR_ERR_INVALID
    small = sc.random_cube_scene(10, seed=64).astype(np.float32)
    code, _, _ = _noalloc(small, [sc.make_view(0.0, 45.0, 0.1, 0.1, 1024, 1024)], cfg)
    assert code == L.SDGR_ERR_INVALID
