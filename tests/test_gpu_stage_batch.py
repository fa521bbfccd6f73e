"""Staging batch sizes of the raster kernels on the GPU.

Every size each raster kernel is built for gives the FP64 oracle's images
(1e-4 of the maximum) and gradients (1e-3 per parameter group) on a dense
scene: 6 000 Gaussians in a 0.6 m box seen in 72 x 56 frames (not multiples
of the 16-pixel tile), so that the tile lists run from under a hundred to
over five thousand Gaussians (one short batch, or five and more batches of
every size with a ragged last one) and rays pass through hundreds of
Gaussians; in both opacity modes, under the one-CTA-per-tile and the
persistent schedule.  The tuner picks a listed size for every kernel and
leaves the optimisation state as it was."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import assert_grads, assert_images, f32

pytestmark = pytest.mark.gpu

KERNELS = ("intensity_fwd", "splat_fwd", "splat_bwd", "intensity_bwd")


def _scene():
    params = sc.vehicle_box_scene(6000, seed=95, extent=(0.6, 0.6, 0.6), log_s_mean=math.log(0.04),
                                  center=(0, 0, 0.3))
    views = [sc.make_view(40.0, 45.0, 0.02, 0.02, 72, 56, center=(0, 0, 0.3)),
             sc.make_view(160.0, 35.0, 0.02, 0.02, 72, 56, center=(0, 0, 0.3))]
    return params, views


@pytest.fixture(scope="module")
def dense():
    params, views = _scene()
    p32, p64 = f32(params)
    rng = np.random.default_rng(96)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    ref = {}
    for am in (0, 1):
        c = oracle.cfg(alpha_mode=am)
        ims = oracle.render(p64, views, c, culled=True)[0]
        g = oracle.grad(p64, views, G, c, culled=True)[0]
        ref[am] = (ims, g)
    return p32, views, G, ref


def _run(p32, views, G, alpha_mode, schedule, batches):
    import torch
    from paper_2506_21633_b300.render import Renderer, split_images
    r = Renderer(alpha_mode=alpha_mode)
    r.set_schedule(schedule)
    for k, nb in batches.items():
        r.set_stage_batch(k, nb)
    p = torch.from_numpy(p32).cuda()
    r.prepare(p, views)
    img = r.forward()
    g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
    grads = r.backward(g)
    torch.cuda.synchronize()
    ims = [x.cpu().numpy().astype(np.float64) for x in split_images(img, views)]
    return ims, grads.cpu().numpy().astype(np.float64), r


def _cases():
    from paper_2506_21633_b300 import _lib as L
    out = []
    for k in KERNELS:
        for nb in L.sdgr_stage_batch_options(k):
            out.append((k, nb))
    return out


def test_every_size_is_listed():
    from paper_2506_21633_b300 import _lib as L
    cases = _cases()
    assert ("intensity_fwd", 512) in cases and ("splat_fwd", 512) in cases and ("splat_bwd", 256) in cases
    assert all(k in L.RASTER_KERNELS for k, _ in cases)


@pytest.mark.parametrize("alpha_mode", [0, 1])
@pytest.mark.parametrize("schedule", ["tiles", "persistent"])
def test_stage_batches_match_oracle(dense, alpha_mode, schedule):
    p32, views, G, ref = dense
    ref_ims, ref_g = ref[alpha_mode]
    for k, nb in _cases():
        ims, grads, r = _run(p32, views, G, alpha_mode, schedule, {k: nb})
        assert r.stage_batch == {k: nb}
        assert_images(ims, ref_ims)
        assert_grads(grads, ref_g)
    # every kernel at its largest size at once
    from paper_2506_21633_b300 import _lib as L
    big = {k: max(L.sdgr_stage_batch_options(k)) for k in KERNELS}
    ims, grads, _ = _run(p32, views, G, alpha_mode, schedule, big)
    assert_images(ims, ref_ims)
    assert_grads(grads, ref_g)


def test_lists_span_several_batches(dense):
    """The scene does what the docstring says: the mean tile list of a
    plane is longer than the largest staging batch (so some lists take
    several batches of every size)."""
    import torch
    from paper_2506_21633_b300.render import Renderer
    p32, views, _, _ = dense
    r = Renderer()
    p = torch.from_numpy(p32).cuda()
    r.prepare(p, views)
    tiles = sum(((v["NA"] + 15) // 16) * ((v["NR"] + 15) // 16) for v in views)
    assert r.n_inst / 2.0 / tiles > 1024


def test_tuner_picks_listed_sizes():
    import torch
    from paper_2506_21633_b300 import _lib as L
    from paper_2506_21633_b300.batch import FusedStep
    params, views = _scene()
    start32 = sc.perturb(params, seed=97).astype(np.float32)
    rng = np.random.default_rng(98)
    tg = torch.from_numpy(rng.uniform(0, 0.1, size=sum(v["NA"] * v["NR"] for v in views)).astype(np.float32)).cuda()
    p = torch.from_numpy(start32.copy()).cuda()
    fs = FusedStep(p, views, tg).capture()
    fs.autotune(steps=1)
    for k in KERNELS:
        opts = L.sdgr_stage_batch_options(k)
        if len(opts) > 1:
            best, ms = fs.stage_batch_ms[k]
            assert set(ms) == set(opts) and best in opts and fs.r.stage_batch[k] == best
            assert all(v > 0 for v in ms.values())
    assert fs.graph is not None
    assert np.array_equal(p.cpu().numpy(), start32)
    fs.step()
    assert fs.check()
