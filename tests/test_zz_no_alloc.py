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


def _workspace_path(params32, views, **cfg):
    import torch
    from paper_2506_21633_b300.render import Renderer
    r = Renderer(**cfg)
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


def test_noalloc_capacity_exceeded_gives_zeros():
    """A dense scene inside the N, V and pixel limits whose tile instances do
    not fit the scratch: SDGR_ERR_CAPACITY and all-zero images."""
    from paper_2506_21633_b300 import _lib as L
    cfg = L.make_cfg()
    dense = sc.random_cube_scene(16384, half=1.0, s_lo=0.2, s_hi=0.4, seed=65)
    views = [sc.make_view(45.0 + 80.0 * k, 40.0 + 5.0 * k, 0.02, 0.02, 256, 256) for k in range(4)]
    code, img, _ = _noalloc(np.ascontiguousarray(dense, dtype=np.float32), views, cfg)
    assert code == L.SDGR_ERR_CAPACITY, L.status_string(code)
    assert np.all(img == 0.0)


@pytest.mark.parametrize("opts", [dict(norm_mode=1), dict(alpha_mode=1)])
def test_noalloc_other_options(opts):
    """A call with other renderer options rebuilds the scratch's workspace
    binding; the result still matches the workspace-based path."""
    from paper_2506_21633_b300 import _lib as L
    cfg = L.make_cfg(norm_mode=opts.get("norm_mode", 0), alpha_mode=opts.get("alpha_mode", 0))
    params = sc.vehicle_box_scene(3000, seed=66, extent=(2.0, 1.5, 1.0), log_s_mean=math.log(0.06),
                                  center=(0.0, 0.0, 0.5))
    views = sc.random_views(2, seed=67, size=128, res=0.03, center=(0.0, 0.0, 0.5))
    p32 = np.ascontiguousarray(params, dtype=np.float32)
    code, img, inten = _noalloc(p32, views, cfg)
    assert code == L.SDGR_OK, L.status_string(code)
    ref_img, ref_inten = _workspace_path(p32, views, **opts)
    assert np.abs(img - ref_img).max() <= IMG_TOL * np.abs(ref_img).max()
    assert np.abs(inten - ref_inten).max() <= IMG_TOL * np.abs(ref_inten).max()
