"""Batched, graph-captured optimisation steps over scenes of uneven size.

- A captured-and-replayed step sequence gives the same parameters as the
  same steps enqueued eagerly (within float32 atomic-order noise).
- The first step's gradient of a multi-scene, mixed-size batch matches the
  FP64 oracle scene by scene.
- An instance-capacity overflow inside a captured step is reported by
  check(), the workspace grows, the graph is captured again and the next
  step is correct."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import assert_grads, f32

pytestmark = pytest.mark.gpu


def _batch():
    a = sc.vehicle_box_scene(900, seed=71, extent=(2.0, 1.5, 1.0), log_s_mean=math.log(0.08), center=(0, 0, 0.5))
    b = sc.vehicle_box_scene(300, seed=72, extent=(1.0, 1.0, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0.5))
    params = np.concatenate([a, b])
    offs = [0, 900, 1200]
    views = [sc.make_view(20.0, 35.0, 0.05, 0.05, 64, 48, center=(0, 0, 0.5), scene=0),
             sc.make_view(140.0, 50.0, 0.04, 0.05, 40, 72, center=(0, 0, 0.5), scene=1),
             sc.make_view(260.0, 45.0, 0.05, 0.04, 57, 57, center=(0, 0, 0.5), scene=0),
             sc.make_view(320.0, 30.0, 0.03, 0.03, 33, 29, center=(0, 0, 0.5), scene=1)]
    return params, offs, views


def _targets(params32, views, offs):
    import torch
    from paper_2506_21633_b300.render import Renderer
    r = Renderer()
    t = r.prepare(torch.from_numpy(params32).cuda(), views, offs).forward()
    torch.cuda.synchronize()
    return t.clone()


def test_graph_replay_matches_eager():
    import torch
    from paper_2506_21633_b300.batch import FusedStep
    params, offs, views = _batch()
    true32 = params.astype(np.float32)
    start32 = sc.perturb(params, seed=3).astype(np.float32)
    tg = _targets(true32, views, offs)
    runs = []
    for capture in (False, True):
        p = torch.from_numpy(start32.copy()).cuda()
        fs = FusedStep(p, views, tg, offs)
        if capture:
            fs.capture()
        for _ in range(4):
            fs.step()
        assert fs.check()
        runs.append(p.cpu().numpy().astype(np.float64))
    moved = np.abs(runs[0] - start32).max()
    assert moved > 0
    assert np.abs(runs[0] - runs[1]).max() <= 1e-3 * moved


def test_multi_step_graph_with_stage_events():
    """One graph of K consecutive steps (the bench's timed form): a replay
    advances the optimisation like K one-step replays, and the stage events
    captured as graph nodes give that replay's per-stage times (K launches
    of every stage, positive times)."""
    import torch
    from paper_2506_21633_b300 import _lib as L
    from paper_2506_21633_b300.batch import FusedStep
    params, offs, views = _batch()
    start32 = sc.perturb(params, seed=5).astype(np.float32)
    tg = _targets(params.astype(np.float32), views, offs)
    K = 3
    runs = []
    for multi in (False, True):
        p = torch.from_numpy(start32.copy()).cuda()
        fs = FusedStep(p, views, tg, offs)
        if multi:
            g = fs.capture_graph(steps=K, profile=True)
            g.replay()
            torch.cuda.synchronize()
            prof = fs.r.profile_read(reset=True)
            for stage in L.STAGES:
                ms, n = prof[stage]
                assert n == K and ms > 0.0, (stage, ms, n)
            assert fs.graph_launches > 0
        else:
            fs.capture()
            for _ in range(K):
                fs.step()
        assert fs.check()
        runs.append(p.cpu().numpy().astype(np.float64))
    moved = np.abs(runs[0] - start32).max()
    assert moved > 0
    assert np.abs(runs[0] - runs[1]).max() <= 1e-3 * moved


def test_first_step_gradient_multiscene():
    """Seeded targets far above every rendered value: sign(S - S*) = -1 on
    both sides, so the fused step's L1 upstream gradient is exactly -1/npix
    for the GPU and for the oracle."""
    import torch
    from paper_2506_21633_b300.batch import FusedStep
    params, offs, views = _batch()
    start = sc.perturb(params, seed=4)
    p32, p64 = f32(start)
    rng = np.random.default_rng(6)
    targets = [50.0 + rng.uniform(0.0, 1.0, size=(v["NR"], v["NA"])) for v in views]
    tg = torch.from_numpy(np.concatenate([t.ravel() for t in targets]).astype(np.float32)).cuda()
    fs = FusedStep(torch.from_numpy(p32.copy()).cuda(), views, tg, offs)
    fs.enqueue()
    assert fs.check()
    g_gpu = fs.grads.cpu().numpy().astype(np.float64)
    imgs = []
    for v in views:
        s = v["scene"]
        imgs.append(oracle.render(p64[offs[s]:offs[s + 1]], [v], oracle.cfg(), culled=True)[0][0])
    assert max(im.max() for im in imgs) < 50.0
    _, dLdS = oracle.l1(imgs, targets)
    ref = np.zeros_like(p64)
    for s in range(2):
        ks = [k for k, v in enumerate(views) if v["scene"] == s]
        ref[offs[s]:offs[s + 1]] = oracle.grad(p64[offs[s]:offs[s + 1]], [views[k] for k in ks],
                                               [dLdS[k] for k in ks], oracle.cfg(), culled=True)[0]
    assert_grads(g_gpu, ref)


def test_capacity_overflow_recapture():
    import torch
    from paper_2506_21633_b300.batch import FusedStep
    params, offs, views = _batch()
    true32 = params.astype(np.float32)
    start32 = sc.perturb(params, seed=5).astype(np.float32)
    tg = _targets(true32, views, offs)
    p = torch.from_numpy(start32.copy()).cuda()
    fs = FusedStep(p, views, tg, offs)
    need = fs.r.n_inst
    from paper_2506_21633_b300 import _lib as L
    small = L.sdgr_caps_for(L.make_views(views), len(views), L.make_offsets(offs), 2, need // 4)
    fs.r.caps = None
    fs.r._grow(small)  # a workspace too small for this batch: the next step overflows
    fs.r.n_inst = need // 4
    fs.capture()
    before = p.clone()
    fs.step()
    assert not fs.check()  # overflow reported, workspace grown, graph re-captured
    assert torch.equal(p, before)  # the overflowing step skipped its work
    fs.step()
    assert fs.check()
    assert not torch.equal(p, before)
