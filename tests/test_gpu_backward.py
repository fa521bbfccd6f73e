"""GPU backward parity: gradients of every raw parameter from the CUDA adjoint
against (a) the FP64 oracle's analytic adjoint and (b) FP64 central finite
differences of the oracle's forward.  Tolerance per parameter group (means,
opacity logit, log-scales, P, quaternion): ||g_gpu - g_ref||_inf <= 1e-3
||g_ref||_inf."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import GRAD_TOL, GROUPS, assert_grads, f32, gpu_grad

pytestmark = pytest.mark.gpu


def _upstream(views, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=(v["NR"], v["NA"])) for v in views]


def _ref(p64, views, G, culled=True, **cfg):
    ocfg = oracle.cfg(K=cfg.get("cutoff_K", 5.0), eps=cfg.get("dilation_eps", 0.3), T_min=cfg.get("T_min", 0.0),
                      norm_mode=cfg.get("norm_mode", 0), alpha_mode=cfg.get("alpha_mode", 0))
    return oracle.grad(p64, views, G, ocfg, culled=culled)[0]


def test_tiny_vs_analytic_and_fd():
    params = sc.vehicle_box_scene(60, seed=31, extent=(1.2, 0.8, 0.6), log_s_mean=math.log(0.1), center=(0, 0, 0))
    views = [sc.make_view(25.0, 40.0, 0.05, 0.06, 40, 36), sc.make_view(160.0, 55.0, 0.06, 0.05, 37, 41)]
    G = _upstream(views, 1)
    p32, p64 = f32(params)
    g_gpu, _, _ = gpu_grad(p32, views, G)
    g_an = _ref(p64, views, G, culled=False)
    assert_grads(g_gpu, g_an)
    # central differences of the oracle without cutoff, on a sample of entries
    rng = np.random.default_rng(2)
    idx = [(int(i), int(j)) for i, j in zip(rng.integers(0, 60, 96), rng.integers(0, 12, 96))]
    fd, bad = oracle.linear_loss_grad_fd(p64, views, G, oracle.cfg(K=0.0), idx=idx)
    for name, cols in GROUPS.items():
        sel = [k for k, (i, j) in enumerate(idx) if j in cols and not bad[k]]
        if not sel:
            continue
        scale = np.abs(g_an[:, cols]).max()
        err = max(abs(g_gpu[idx[k]] - fd[k]) for k in sel)
        assert err <= GRAD_TOL * scale, (name, err, scale)


def test_config3_shaped_analytic():
    """Config-3 distributions (random rotations, log-normal scales), denser
    and smaller."""
    params, views = sc.config3_small(n=3000, n_views=3, size=64, res=0.1)
    G = _upstream(views, 3)
    p32, p64 = f32(params)
    g_gpu, _, _ = gpu_grad(p32, views, G)
    g_an = _ref(p64, views, G)
    assert_grads(g_gpu, g_an)


def test_config2_view_l1():
    """Buildings at full 512x512, one view, L1 loss against an oracle-rendered
    target of the unperturbed scene; upstream dL/dS from the oracle's L1."""
    params, views = sc.config2()
    v = [views[9]]
    target = oracle.render(f32(params)[1], v, oracle.cfg(), culled=True)[0]
    start = sc.perturb(params, seed=5)
    p32, p64 = f32(start)
    cur = oracle.render(p64, v, oracle.cfg(), culled=True)[0]
    _, dLdS = oracle.l1(cur, target)
    g_gpu, _, _ = gpu_grad(p32, v, dLdS)
    g_an = _ref(p64, v, dLdS)
    assert_grads(g_gpu, g_an)


@pytest.mark.parametrize("cfg", [dict(norm_mode=1), dict(T_min=1e-4), dict(alpha_mode=1),
                                 dict(alpha_mode=1, T_min=1e-4)])
def test_options(cfg):
    params = sc.vehicle_box_scene(500, seed=33, extent=(2.0, 1.5, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0))
    views = sc.random_views(2, seed=34, size=48, res=0.08, center=(0, 0, 0))
    G = _upstream(views, 4)
    p32, p64 = f32(params)
    g_gpu, _, _ = gpu_grad(p32, views, G, **cfg)
    g_an = _ref(p64, views, G, **cfg)
    assert_grads(g_gpu, g_an)


def test_multi_scene():
    a = sc.vehicle_box_scene(300, seed=35, extent=(2.0, 1.0, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0))
    b = sc.vehicle_box_scene(200, seed=36, extent=(1.0, 1.0, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0))
    params = np.concatenate([a, b])
    offs = [0, 300, 500]
    views = [sc.make_view(30.0, 40.0, 0.06, 0.06, 40, 40, scene=0), sc.make_view(120.0, 50.0, 0.05, 0.05, 33, 47, scene=1),
             sc.make_view(250.0, 35.0, 0.06, 0.05, 41, 29, scene=0)]
    G = _upstream(views, 6)
    p32, p64 = f32(params)
    g_gpu, _, _ = gpu_grad(p32, views, G, scene_offsets=offs)
    ref = np.zeros_like(p64)
    for s in range(2):
        vs = [v for v in views if v["scene"] == s]
        gs = [g for v, g in zip(views, G) if v["scene"] == s]
        ref[offs[s]:offs[s + 1]] = _ref(p64[offs[s]:offs[s + 1]], vs, gs)
    assert_grads(g_gpu, ref)
