"""Densification and pruning on the GPU against the oracle's rules: the same
survivors in the same order (decisions are float32 comparisons on both
sides), the same parameters / moments / SH rows; the capacity check; and
the gradient statistics accumulated by the adjoint."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import f32

pytestmark = pytest.mark.gpu

CFG = dict(grad_threshold=0.003, dense_scale=0.03, max_scale=0.3, min_opacity=0.02, min_P=0.02, split_factor=1.6)


def _cfg(L):
    return L.SdgrDensifyCfg(**CFG)


def _inputs(n=4000, seed=0):
    rng = np.random.default_rng(seed)
    params = sc.vehicle_box_scene(n, seed=seed, log_s_mean=math.log(0.03), log_s_sd=0.8).astype(np.float32)
    params[:, 3] = rng.normal(0.0, 3.0, size=n)          # some opacities below the minimum
    params[:, 7] = rng.uniform(-0.01, 1.0, size=n)       # some P below the minimum
    grads = rng.normal(size=(n, 12)).astype(np.float32)
    count = rng.integers(0, 5, size=n).astype(np.float32)
    accum = (count * rng.exponential(0.003, size=n)).astype(np.float32)
    m = rng.normal(size=(n, 12)).astype(np.float32)
    v = rng.uniform(0, 1, size=(n, 12)).astype(np.float32)
    sh = rng.normal(size=(n, 16)).astype(np.float32)
    return params, grads, accum, count, m, v, sh


def _run(L, torch, arrays, cap):
    params, grads, accum, count, m, v, sh = [torch.from_numpy(a).cuda() for a in arrays]
    n = params.shape[0]
    out = [torch.full((cap, w), -7.0, device="cuda") for w in (12, 12, 12, 16)]
    scratch = torch.empty(L.sdgr_densify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    code, new_n = L.sdgr_densify(params.data_ptr(), grads.data_ptr(), accum.data_ptr(), count.data_ptr(),
                                 m.data_ptr(), v.data_ptr(), sh.data_ptr(), n, _cfg(L),
                                 *[o.data_ptr() for o in out], cap, scratch.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return code, new_n, [o[:new_n].cpu().numpy().astype(np.float64) for o in out]


def test_densify_matches_oracle():
    import torch
    from oracle.densify import densify
    from paper_2506_21633_b300 import _lib as L
    arrays = _inputs()
    code, new_n, (gp, gm, gv, gsh) = _run(L, torch, arrays, cap=3 * arrays[0].shape[0])
    assert code == L.SDGR_OK
    rp, rm, rv, rsh, act = densify(*arrays, **CFG)
    assert {"prune", "keep", "clone", "split"} <= set(act)
    assert new_n == rp.shape[0]
    for a, b in ((gp, rp), (gm, rm), (gv, rv), (gsh, rsh)):
        assert np.abs(a - b).max() <= 2e-6 * max(1.0, np.abs(b).max())


def test_densify_capacity():
    import torch
    from paper_2506_21633_b300 import _lib as L
    arrays = _inputs(n=1000, seed=1)
    code, need, _ = _run(L, torch, arrays, cap=10)
    assert code == L.SDGR_ERR_CAPACITY and need > 10


def test_gradient_statistics():
    import torch
    from paper_2506_21633_b300 import _lib as L
    from paper_2506_21633_b300.render import Renderer
    params = sc.vehicle_box_scene(600, seed=2, extent=(2.0, 1.5, 1.0), log_s_mean=math.log(0.1), center=(0, 0, 0))
    views = sc.random_views(3, seed=3, size=48, res=0.08, center=(0, 0, 0))
    p32, p64 = f32(params)
    rng = np.random.default_rng(4)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    r = Renderer()
    p = torch.from_numpy(p32).cuda()
    r.prepare(p, views)
    accum = torch.zeros(600, device="cuda")
    count = torch.zeros(600, device="cuda")
    r.set_densify_stats(accum, count)
    r.forward()
    g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
    for _ in range(2):  # two backward calls accumulate
        r.backward(g)
    torch.cuda.synchronize()
    _, dI, duI = oracle.grad_uI(p64, views, G, oracle.cfg(), culled=True)
    seen = (dI != 0) | (np.abs(duI).sum(axis=2) != 0)
    ref_count = 2 * seen.sum(axis=0)
    ref_accum = 2 * (np.linalg.norm(duI, axis=2) * seen).sum(axis=0)
    c = count.cpu().numpy()
    agree = c == ref_count
    assert agree.mean() > 0.99
    a = accum.cpu().numpy()
    scale = ref_accum.max()
    assert np.abs(a[agree] - ref_accum[agree]).max() <= 1e-3 * scale
