"""Parity at the full headline size, in the launch configuration the bench
times: the 300 000-Gaussian config-3 scene, all 64 views of 1024^2 in one
batch with the default (persistent, longest-first) schedule.

- images and per-(view, Gaussian) intensities of two sampled views against
  the FP64 oracle (bounding-box culled mode: the same arithmetic), pixel by
  pixel, 1e-4 of the maximum;
- the gradient of the whole 64-view launch with a non-zero upstream image on
  one view only equals the oracle's gradient of that view (the other 63 views
  must contribute nothing), 1e-3 per parameter group;
- one 2048^2 view (the largest image size the server accepts) of a 40 000-
  Gaussian scene, against the oracle;
- the Beer-Lambert opacity (alpha_mode 1), whose intensity adjoint walks each
  hit list one hit at a time: the full scene, eight of its views in one
  batch, the gradient with a non-zero upstream image on one view against the
  oracle's gradient of that view."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import IMG_TOL, assert_grads, assert_images, f32

pytestmark = pytest.mark.gpu

SAMPLED = (0, 37)
GRAD_VIEW = 5


@pytest.fixture(scope="module")
def full():
    import torch
    from paper_2506_21633_b300.render import Renderer, split_images
    params, views = sc.config3()
    p32, p64 = f32(params)
    r = Renderer()
    assert r.schedule == "persistent"
    p = torch.from_numpy(p32).cuda()
    r.prepare(p, views)
    inten = torch.zeros(r.view_gauss(), dtype=torch.float32, device="cuda")
    img = r.forward(intensity=inten)
    torch.cuda.synchronize()
    ims = [x.cpu().numpy().astype(np.float64) for x in split_images(img, views)]
    return params, views, p32, p64, r, ims, inten.cpu().numpy().astype(np.float64)


def test_config3_full_forward_sampled_views(full):
    params, views, p32, p64, r, ims, inten = full
    N = p64.shape[0]
    for k in SAMPLED:
        ref, A, _ = oracle.render(p64, [views[k]], oracle.cfg(), culled=True)
        assert_images([ims[k]], ref, tol=IMG_TOL)
        refI = p64[:, 7] * A[0]
        gpuI = inten[k * N:(k + 1) * N]
        assert np.abs(gpuI - refI).max() <= IMG_TOL * np.abs(refI).max()


def test_config3_full_gradient_one_view(full):
    import torch
    params, views, p32, p64, r, ims, inten = full
    rng = np.random.default_rng(11)
    G = [np.zeros((v["NR"], v["NA"])) for v in views]
    G[GRAD_VIEW] = rng.normal(size=G[GRAD_VIEW].shape)
    g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
    grads = r.backward(g)
    torch.cuda.synchronize()
    ref = oracle.grad(p64, [views[GRAD_VIEW]], [G[GRAD_VIEW]], oracle.cfg(), culled=True)[0]
    assert_grads(grads.cpu().numpy().astype(np.float64), ref)


def test_largest_image_2048():
    from gpu_helpers import gpu_forward
    params = sc.vehicle_box_scene(40000, seed=44, extent=(6.0, 3.0, 2.0), log_s_mean=math.log(0.03))
    view = sc.make_view(123.0, 41.0, 0.005, 0.005, 2048, 2048, center=(0.0, 0.0, 1.0))
    p32, p64 = f32(params)
    ims, inten, _, _ = gpu_forward(p32, [view])
    ref, A, _ = oracle.render(p64, [view], oracle.cfg(), culled=True)
    assert_images(ims, ref)
    refI = p64[:, 7] * A[0]
    assert np.abs(inten - refI).max() <= IMG_TOL * np.abs(refI).max()


def test_config3_beer_lambert_gradient_one_view():
    import torch
    from paper_2506_21633_b300.render import Renderer
    params, views = sc.config3()
    views = views[:8]
    p32, p64 = f32(params)
    r = Renderer(alpha_mode=1)
    r.prepare(torch.from_numpy(p32).cuda(), views)
    ims = r.forward()
    rng = np.random.default_rng(12)
    k = 3
    G = [np.zeros((v["NR"], v["NA"])) for v in views]
    G[k] = rng.normal(size=G[k].shape)
    g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
    grads = r.backward(g)
    torch.cuda.synchronize()
    cfg = oracle.cfg(alpha_mode=1)
    ref_img = oracle.render(p64, [views[k]], cfg, culled=True)[0]
    n0 = sum(v["NR"] * v["NA"] for v in views[:k])
    img_k = ims[n0:n0 + views[k]["NR"] * views[k]["NA"]].cpu().numpy().astype(np.float64)
    assert_images([img_k.reshape(views[k]["NR"], views[k]["NA"])], ref_img, tol=IMG_TOL)
    ref = oracle.grad(p64, [views[k]], [G[k]], cfg, culled=True)[0]
    assert_grads(grads.cpu().numpy().astype(np.float64), ref)
