"""Checkpoint / resume: saving the optimisation state after some steps and
resuming from it (in a fresh FusedStep, graph-captured, and in a fresh
reconstruction Trainer) continues the run exactly as an uninterrupted one,
within float32 atomic-order noise."""
import io
import math

import numpy as np
import pytest

import sdgr_scenes as sc

pytestmark = pytest.mark.gpu


def _batch():
    params = sc.vehicle_box_scene(800, seed=61, extent=(2.0, 1.5, 1.0), log_s_mean=math.log(0.08), center=(0, 0, 0.5))
    views = [sc.make_view(20.0 + 90.0 * k, 35.0 + 8.0 * k, 0.05, 0.05, 56, 48, center=(0, 0, 0.5)) for k in range(3)]
    return params, views


def test_fused_step_resume():
    import torch
    from paper_2506_21633_b300.batch import FusedStep
    from paper_2506_21633_b300.render import Renderer
    params, views = _batch()
    tg = Renderer().prepare(torch.from_numpy(params.astype(np.float32)).cuda(), views).forward().clone()
    start = sc.perturb(params, seed=2).astype(np.float32)
    a = FusedStep(torch.from_numpy(start.copy()).cuda(), views, tg).capture()
    for _ in range(3):
        a.step()
    buf = io.BytesIO()
    torch.save(a.state_dict(), buf)
    for _ in range(3):
        a.step()
    assert a.check()
    buf.seek(0)
    state = torch.load(buf)
    b = FusedStep(torch.from_numpy(start.copy()).cuda(), views, tg).capture()
    b.load_state_dict(state)
    for _ in range(3):
        b.step()
    assert b.check()
    pa, pb = a.p.cpu().numpy(), b.p.cpu().numpy()
    moved = np.abs(pa - state["params"].numpy()).max()
    assert moved > 0
    assert np.abs(pa - pb).max() <= 1e-3 * moved
    assert int(b.step_dev.item()) == 6


def test_trainer_resume():
    """Float32 atomic order makes two identical runs differ a little, and Adam
    turns the sign noise of near-zero gradients into lr-sized steps; the
    resumed run must be as close to the uninterrupted one as a second
    uninterrupted run is."""
    import torch
    from paper_2506_21633_b300.render import Renderer
    from paper_2506_21633_b300.train import Trainer, hemisphere_init
    params, views = _batch()
    tg = Renderer().prepare(torch.from_numpy(params.astype(np.float32)).cuda(), views).forward().clone()
    init = hemisphere_init(1500, 2.0, (0, 0, 0), seed=3)

    def run(state=None):
        t = Trainer(init, views, tg, sh_every=2)
        if state is None:
            for _ in range(4):
                t.step()
            t.densify()
            saved = t.state_dict()
        else:
            t.load_state_dict(state)
            saved = state
        for _ in range(4):
            t.step()
        return t, saved

    a, state = run()
    a2, _ = run()
    b, _ = run(state)
    assert a.p.shape == b.p.shape == a2.p.shape
    pa, pa2, pb = (x.p.cpu().numpy() for x in (a, a2, b))
    moved = np.abs(pa - state["params"].numpy()).max()
    noise = np.abs(pa - pa2).max()
    assert moved > 0
    assert np.abs(pa - pb).max() <= max(3.0 * noise, 1e-4 * moved), (np.abs(pa - pb).max(), noise, moved)
    assert b.t == a.t == 8
