"""The autograd.Function of the renderer: SDGRRender.apply inside a torch
graph, loss.backward(), params.grad against the FP64 oracle's analytic
adjoint and against FP64 central differences of the oracle (Section II-B:
dL/dS from automatic differentiation, then the hand-written adjoint).
Tolerance per parameter group: ||g_gpu - g_ref||_inf <= 1e-3 ||g_ref||_inf.
Also: a second forward on the same renderer before the backward, and an
in-place change of the parameters, are refused instead of giving the
gradient of another state."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import GRAD_TOL, GROUPS, assert_grads, f32

pytestmark = pytest.mark.gpu


def _scenes():
    a = sc.vehicle_box_scene(300, seed=71, extent=(2.0, 1.0, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0))
    b = sc.vehicle_box_scene(200, seed=72, extent=(1.0, 1.0, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0))
    params = np.concatenate([a, b])
    offs = [0, 300, 500]
    views = [sc.make_view(30.0, 40.0, 0.06, 0.06, 40, 40, scene=0),
             sc.make_view(120.0, 50.0, 0.05, 0.05, 33, 47, scene=1),
             sc.make_view(250.0, 35.0, 0.06, 0.05, 41, 29, scene=0)]
    return params, offs, views


def _torch_grad(p32, views, offs, G, **cfg):
    """params.grad of sum(images * G) through SDGRRender.apply."""
    import torch
    from paper_2506_21633_b300.render import Renderer, SDGRRender
    r = Renderer(**cfg)
    params = torch.from_numpy(p32).cuda().requires_grad_(True)
    g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
    images = SDGRRender.apply(params, r, views, offs)
    loss = (images * g).sum()
    loss.backward()
    torch.cuda.synchronize()
    return params.grad.cpu().numpy().astype(np.float64)


def _oracle_grad(p64, views, offs, G, c):
    ref = np.zeros_like(p64)
    for s in range(len(offs) - 1):
        vs = [dict(v, scene=0) for v in views if v["scene"] == s]
        gs = [g for v, g in zip(views, G) if v["scene"] == s]
        if vs:
            ref[offs[s]:offs[s + 1]] = oracle.grad(p64[offs[s]:offs[s + 1]], vs, gs, c, culled=True)[0]
    return ref


@pytest.mark.parametrize("alpha_mode", [0, 1])
def test_apply_backward_vs_oracle(alpha_mode):
    params, offs, views = _scenes()
    p32, p64 = f32(params)
    rng = np.random.default_rng(73 + alpha_mode)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    g_gpu = _torch_grad(p32, views, offs, G, alpha_mode=alpha_mode)
    ref = _oracle_grad(p64, views, offs, G, oracle.cfg(alpha_mode=alpha_mode))
    assert_grads(g_gpu, ref)


def test_apply_backward_vs_fd():
    params = sc.vehicle_box_scene(60, seed=74, extent=(1.2, 0.8, 0.6), log_s_mean=math.log(0.1), center=(0, 0, 0))
    views = [sc.make_view(25.0, 40.0, 0.05, 0.06, 40, 36), sc.make_view(160.0, 55.0, 0.06, 0.05, 37, 41)]
    p32, p64 = f32(params)
    rng = np.random.default_rng(75)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    g_gpu = _torch_grad(p32, views, None, G)
    g_an = oracle.grad(p64, views, G, oracle.cfg(), culled=False)[0]
    idx = [(int(i), int(j)) for i, j in zip(rng.integers(0, 60, 96), rng.integers(0, 12, 96))]
    fd, bad = oracle.linear_loss_grad_fd(p64, views, G, oracle.cfg(K=0.0), idx=idx)
    for name, cols in GROUPS.items():
        sel = [k for k, (i, j) in enumerate(idx) if j in cols and not bad[k]]
        if not sel:
            continue
        scale = np.abs(g_an[:, cols]).max()
        err = max(abs(g_gpu[idx[k]] - fd[k]) for k in sel)
        assert err <= GRAD_TOL * scale, (name, err, scale)


def test_second_forward_before_backward_is_refused():
    import torch
    from paper_2506_21633_b300.render import Renderer, SDGRRender, StaleRendererError
    params, offs, views = _scenes()
    p32, _ = f32(params)
    r = Renderer()
    a = torch.from_numpy(p32).cuda().requires_grad_(True)
    b = torch.from_numpy(p32 * np.float32(1.01)).cuda().requires_grad_(True)
    img_a = SDGRRender.apply(a, r, views, offs)
    img_b = SDGRRender.apply(b, r, views, offs)  # same renderer, prepared again
    with pytest.raises(StaleRendererError):
        img_a.sum().backward()
    img_b.sum().backward()  # the latest forward still differentiates
    assert b.grad is not None and torch.isfinite(b.grad).all()


def test_in_place_change_is_refused():
    import torch
    from paper_2506_21633_b300.render import Renderer, SDGRRender
    params, offs, views = _scenes()
    p32, _ = f32(params)
    r = Renderer()
    leaf = torch.from_numpy(p32).cuda().requires_grad_(True)
    x = leaf * 1.0
    img = SDGRRender.apply(x, r, views, offs)
    with torch.no_grad():
        x.add_(0.01)  # e.g. an optimiser step between forward and backward
    with pytest.raises(RuntimeError, match="modified by an inplace operation"):
        img.sum().backward()
