"""View-dependent scattering (spherical harmonics of the direction toward the
radar, degrees 1..3): GPU images, parameter gradients and dL/dsh against the
FP64 oracle on the same float32 inputs."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import GRAD_TOL, assert_grads, assert_images, f32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_sh_forward_and_gradients(degree):
    import torch
    from paper_2506_21633_b300.render import Renderer, split_images
    params = sc.vehicle_box_scene(800, seed=90 + degree, extent=(2.0, 1.5, 1.0), log_s_mean=math.log(0.1),
                                  center=(0, 0, 0))
    views = sc.random_views(3, seed=91, size=56, res=0.07, center=(0, 0, 0))
    rng = np.random.default_rng(degree)
    sh32 = rng.normal(scale=0.3, size=(800, 16)).astype(np.float32)
    sh32[:, 15] = 0.0
    p32, p64 = f32(params)
    r = Renderer()
    p = torch.from_numpy(p32).cuda()
    sh = torch.from_numpy(sh32).cuda()
    dsh = torch.zeros_like(sh)
    r.set_sh(sh, dsh, degree)
    r.prepare(p, views)
    img = r.forward()
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
    grads = r.backward(g)
    torch.cuda.synchronize()
    c = oracle.cfg(sh=sh32.astype(np.float64), sh_degree=degree)
    ref_imgs, _, _ = oracle.render(p64, views, c, culled=True)
    assert_images([x.cpu().numpy().astype(np.float64) for x in split_images(img, views)], ref_imgs)
    ref_g, ref_dsh = oracle.grad_sh(p64, views, G, c, culled=True)
    assert_grads(grads.cpu().numpy().astype(np.float64), ref_g)
    got = dsh.cpu().numpy().astype(np.float64)
    nk = {1: 3, 2: 8, 3: 15}[degree]
    scale = np.abs(ref_dsh[:, :nk]).max()
    assert scale > 0
    assert np.abs(got[:, :nk] - ref_dsh[:, :nk]).max() <= GRAD_TOL * scale
    assert np.all(got[:, nk:] == 0)
