"""Transmittance floor on the GPU: rays that stop part-way through their tile
lists (Section III-A's early termination).

With a high floor (T_min = 0.3) most rays stop after a few Gaussians, at every
position of the 32-Gaussian slices the intensity pass walks (first, middle or
last hit of a slice; both rays of a lane in one slice, or in different ones),
so its per-slice search for the stopping pair runs in nearly every warp; with
T_min = 1e-4 fewer rays stop, deep in their lists.  In the opaque variants a
third of the Gaussians have opacity logit 30: o = 1 in float32 (alpha = the
profile) and, in the Beer-Lambert mode, alpha = 1 exactly near their centres,
so the transmittance behind a stopping pair is exactly 0.  Images,
per-Gaussian intensities and gradients of every parameter group against the
FP64 oracle, in both opacity modes; the scene is checked to make most rays
stop where the case says so."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import IMG_TOL, assert_grads, assert_images, f32, gpu_grad

pytestmark = pytest.mark.gpu


def _scene(opaque):
    params = sc.vehicle_box_scene(900, seed=61, extent=(1.5, 1.2, 0.8), log_s_mean=math.log(0.08),
                                  center=(0, 0, 0))
    if opaque:
        params = params.copy()
        params[::3, 3] = 30.0
    # 52 x 44: ragged last tile row and column
    views = [sc.make_view(35.0, 40.0, 0.035, 0.035, 52, 44), sc.make_view(215.0, 50.0, 0.035, 0.035, 52, 44)]
    return params, views


@pytest.mark.parametrize("alpha_mode", [0, 1])
@pytest.mark.parametrize("T_min,opaque", [(0.3, False), (0.3, True), (1e-4, False), (1e-4, True), (0.0, True)])
def test_floor_matches_oracle(alpha_mode, T_min, opaque):
    params, views = _scene(opaque)
    p32, p64 = f32(params)
    rng = np.random.default_rng(62)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    cfg = dict(T_min=T_min, alpha_mode=alpha_mode)
    g_gpu, ims, inten = gpu_grad(p32, views, G, **cfg)
    ocfg = oracle.cfg(T_min=T_min, alpha_mode=alpha_mode)
    ref_ims, A, Tf = oracle.render(p64, views, ocfg, culled=True)
    stopped = np.mean(np.concatenate([(t < T_min).ravel() for t in Tf]))
    if T_min >= 0.3:
        assert stopped > 0.7, stopped  # most rays stop
    elif T_min > 0:
        assert 0.2 < stopped < 0.95, stopped  # rays that stop and rays that run to the end
    assert_images(ims, ref_ims)
    refI = np.concatenate([p64[:, 7] * A[k] for k in range(len(views))])
    assert np.abs(inten - refI).max() <= IMG_TOL * np.abs(refI).max()
    g_ref = oracle.grad(p64, views, G, ocfg, culled=True)[0]
    assert_grads(g_gpu, g_ref)
