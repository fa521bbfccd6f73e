"""Degenerate inputs on the GPU, against the FP64 oracle (images 1e-4 of the
maximum, gradients 1e-3 per parameter group):

- saturated opacities stacked along one line of sight, so that rays fall
  below the 2^-100 transmittance floor and stop (the pass records where, the
  adjoint starts there; the oracle runs without a floor: what is cut is below
  float32 resolution);
- a Gaussian much larger than the image (every tile of the view in its list);
- thin Gaussians whose 2D covariance is mostly the dilation;
- grazing angles of 5 and 85 degrees;
- one-row and one-column images;
- an empty scene inside a multi-scene batch;
- a Gaussian with NaN parameters: the call completes, the status stays OK and
  the other Gaussians' images and gradients are those without it;
- image sizes that cut the tiles' 4 x 8 half-blocks (the intensity adjoint's
  culling unit) and small Gaussians that reach only one half of a warp's
  block, so that the two halves' hit lists differ in length and the shorter
  one is padded."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import assert_grads, assert_images, f32, gpu_forward, gpu_grad

pytestmark = pytest.mark.gpu


def _one(mu, s, o, P=0.8):
    p = np.zeros((1, 12))
    p[0, 0:3] = mu
    p[0, 3] = 40.0 if o >= 1.0 else math.log(o) - math.log1p(-o)
    p[0, 4:7] = math.log(s)
    p[0, 7] = P
    p[0, 8] = 1.0
    return p


def _parity(params, views, seed, **cfg):
    p32, p64 = f32(params)
    rng = np.random.default_rng(seed)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    g_gpu, ims, _ = gpu_grad(p32, views, G, **cfg)
    ref_img = oracle.render(p64, views, oracle.cfg(), culled=True)[0]
    assert_images(ims, ref_img)
    ref_g = oracle.grad(p64, views, G, oracle.cfg(), culled=True)[0]
    assert_grads(g_gpu, ref_g)
    return g_gpu, ims


def test_saturated_stack_stops_rays():
    v = sc.make_view(40.0, 50.0, 0.04, 0.04, 48, 48)
    th, ph = v["theta"], v["phi"]
    los = np.array([-math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    side = np.array([-math.sin(ph), -math.cos(ph), 0.0])
    # 24 near-opaque Gaussians one behind another, slightly staggered sideways
    stack = [_one(0.15 * k * los + 0.01 * k * side, 0.25, 1.0 if k % 3 == 0 else 0.999, P=0.3 + 0.02 * k)
             for k in range(24)]
    params = np.concatenate(stack)[::-1].copy()  # storage order differs from depth order
    _parity(params, [v], 1)


def test_gaussian_larger_than_the_image():
    params = np.concatenate([_one((0.0, 0.0, 0.0), 3.0, 0.3),
                             sc.vehicle_box_scene(200, seed=5, extent=(1.0, 1.0, 0.5), log_s_mean=math.log(0.05),
                                                  center=(0.0, 0.0, 0.0))])
    views = [sc.make_view(10.0, 35.0, 0.03, 0.03, 70, 50), sc.make_view(100.0, 60.0, 0.025, 0.03, 64, 64)]
    _parity(params, views, 2)


def test_thin_gaussians():
    params = sc.vehicle_box_scene(400, seed=6, extent=(1.0, 1.0, 0.6), log_s_mean=math.log(0.0005), log_s_sd=0.3,
                                  center=(0.0, 0.0, 0.0))
    views = [sc.make_view(25.0, 45.0, 0.02, 0.02, 56, 56)]
    _parity(params, views, 3)


@pytest.mark.parametrize("theta", [5.0, 85.0])
def test_extreme_grazing_angles(theta):
    params = sc.vehicle_box_scene(500, seed=7, extent=(1.2, 1.0, 0.8), log_s_mean=math.log(0.06), center=(0, 0, 0))
    views = [sc.make_view(70.0, theta, 0.04, 0.04, 60, 44)]
    _parity(params, views, 4)


def test_single_row_and_column_images():
    params = sc.vehicle_box_scene(300, seed=8, extent=(1.0, 1.0, 0.5), log_s_mean=math.log(0.08), center=(0, 0, 0))
    views = [sc.make_view(15.0, 40.0, 0.05, 0.05, 64, 1), sc.make_view(200.0, 55.0, 0.05, 0.05, 1, 64),
             sc.make_view(300.0, 45.0, 0.05, 0.05, 1, 1)]
    _parity(params, views, 5)


def test_empty_scene_in_a_batch():
    a = sc.vehicle_box_scene(300, seed=9, extent=(1.0, 1.0, 0.5), log_s_mean=math.log(0.08), center=(0, 0, 0))
    b = sc.vehicle_box_scene(200, seed=10, extent=(1.0, 1.0, 0.5), log_s_mean=math.log(0.08), center=(0, 0, 0))
    params = np.concatenate([a, b])
    offs = [0, 300, 300, 500]  # scene 1 is empty
    views = [sc.make_view(30.0, 40.0, 0.05, 0.05, 40, 40, scene=0), sc.make_view(90.0, 40.0, 0.05, 0.05, 40, 40, scene=1),
             sc.make_view(150.0, 50.0, 0.05, 0.05, 36, 44, scene=2)]
    p32, p64 = f32(params)
    ims, _, r, _ = gpu_forward(p32, views, offs)
    assert np.all(ims[1] == 0)
    for k, s in ((0, 0), (2, 2)):
        ref = oracle.render(p64[offs[s]:offs[s + 1]], [views[k]], oracle.cfg(), culled=True)[0]
        assert_images([ims[k]], ref)


def test_nan_gaussian_stays_local():
    params = sc.vehicle_box_scene(400, seed=11, extent=(1.0, 1.0, 0.5), log_s_mean=math.log(0.08), center=(0, 0, 0))
    views = [sc.make_view(30.0, 40.0, 0.05, 0.05, 48, 40), sc.make_view(200.0, 55.0, 0.05, 0.05, 40, 48)]
    bad = params.copy()
    bad[123, 0:3] = np.nan
    p32, p64 = f32(params)
    b32, _ = f32(bad)
    rng = np.random.default_rng(12)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    g_ok, ims_ok, _ = gpu_grad(np.delete(p32, 123, axis=0), views, G)
    g_bad, ims_bad, _ = gpu_grad(b32, views, G)
    for a, b in zip(ims_bad, ims_ok):
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    keep = np.delete(g_bad, 123, axis=0)
    assert np.all(np.isfinite(keep))
    assert_grads(keep, g_ok, tol=1e-4)


def test_ragged_half_blocks_and_one_sided_hits():
    # small Gaussians (a few pixels) scattered over a view whose sides are not
    # multiples of 4, 8 or 16: most reach one 4-column half of a warp's block
    params = sc.vehicle_box_scene(600, seed=13, extent=(1.2, 1.2, 0.4), log_s_mean=math.log(0.02),
                                  center=(0, 0, 0))
    views = [sc.make_view(25.0, 45.0, 0.03, 0.03, 37, 29), sc.make_view(160.0, 35.0, 0.03, 0.03, 45, 51)]
    _parity(params, views, 14)
