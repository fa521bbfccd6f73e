"""Serving loop on the GPU.

- A request gives the same images (1e-4 of the maximum) and gradients
  (1e-3 per parameter group) alone and in the middle of a burst of mixed
  render and gradient requests that the scheduler batches and overlaps.
- A served render matches the FP64 oracle.
- Host-side failures stay local: an invalid request (bad geometry, a
  target of the wrong size, more views than a batch holds) fails alone, a
  request above the HBM budget is refused, a cancelled request is dropped,
  and the other requests complete."""
import math

import numpy as np
import pytest

import oracle
import sdgr_scenes as sc
from gpu_helpers import GRAD_TOL, IMG_TOL, assert_grads, assert_images

pytestmark = pytest.mark.gpu


def _scenes():
    out = []
    for k in range(4):
        out.append(sc.vehicle_box_scene(600 + 300 * k, seed=80 + k, extent=(2.0, 1.5, 1.0),
                                        log_s_mean=math.log(0.08), center=(0, 0, 0.5)).astype(np.float32))
    return out


def _views(seed, n):
    return sc.random_views(n, seed=seed, size=48 + 16 * (seed % 3), res=0.06, center=(0, 0, 0.5))


def _target(views, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.0, 0.2, size=(v["NR"], v["NA"])).astype(np.float32) for v in views]


def test_same_alone_and_in_the_mix():
    from paper_2506_21633_b300.serve import Server
    scenes = _scenes()
    srv = Server(scenes, hbm_budget_bytes=8 << 30, n_slots=3, max_batch_views=24)
    try:
        xv = _views(5, 3)
        xt = _target(xv, 1)
        alone = srv.submit(2, xv, "gradient", xt).result(timeout=120)
        rv = _views(6, 2)
        ralone = srv.submit(1, rv, "render").result(timeout=120)
        futs, mine = [], None
        rng = np.random.default_rng(0)
        for k in range(40):
            if k == 17:
                mine = srv.submit(2, xv, "gradient", xt)
                rmine = srv.submit(1, rv, "render")
            s = int(rng.integers(0, 4))
            vs = _views(100 + k, int(rng.integers(1, 5)))
            if rng.uniform() < 0.5:
                futs.append(srv.submit(s, vs, "render"))
            else:
                futs.append(srv.submit(s, vs, "gradient", _target(vs, 200 + k)))
        mixed = mine.result(timeout=300)
        rmixed = rmine.result(timeout=300)
        for f in futs:
            f.result(timeout=300)
        assert srv.stats["batches"] < srv.stats["requests"]  # requests were batched
        assert max(srv.stats["batch_sizes"]) > 1
        assert_images(mixed.images, alone.images)
        assert_images(rmixed.images, ralone.images)
        assert abs(mixed.loss - alone.loss) <= 1e-5 * abs(alone.loss)
        assert_grads(mixed.grads.astype(np.float64), alone.grads.astype(np.float64), tol=GRAD_TOL)
    finally:
        srv.close(timeout=60)


def test_served_render_matches_oracle():
    from paper_2506_21633_b300.serve import Server
    scenes = _scenes()
    srv = Server(scenes, hbm_budget_bytes=4 << 30, n_slots=2)
    try:
        vs = _views(9, 2)
        res = srv.submit(3, vs, "render").result(timeout=120)
        ref = oracle.render(scenes[3].astype(np.float64), vs, oracle.cfg(), culled=True)[0]
        assert_images([x.astype(np.float64) for x in res.images], ref, tol=IMG_TOL)
    finally:
        srv.close(timeout=60)


def test_failures_stay_local():
    from paper_2506_21633_b300.serve import AdmissionError, Server
    scenes = _scenes()
    srv = Server(scenes, hbm_budget_bytes=64 << 20, n_slots=2)
    try:
        good = [srv.submit(k % 4, _views(300 + k, 2), "render") for k in range(6)]
        bad_view = dict(_views(7, 1)[0], theta=2.0)
        bad = srv.submit(0, [bad_view], "render")
        wrong_target = srv.submit(0, _views(8, 1), "gradient", [np.zeros((3, 3), np.float32)])
        huge = srv.submit(0, [sc.make_view(0.0, 45.0, 0.001, 0.001, 2048, 2048, center=(0, 0, 0.5))] * 8, "render")
        too_many = srv.submit(0, _views(11, 2) * 40, "render")  # more views than a batch holds
        cancelled = srv.submit(1, _views(10, 2), "render")
        cancelled.cancel()
        with pytest.raises(ValueError):
            too_many.result(timeout=60)
        with pytest.raises(ValueError):
            bad.result(timeout=60)
        with pytest.raises(ValueError):
            wrong_target.result(timeout=60)
        with pytest.raises(AdmissionError):
            huge.result(timeout=60)
        for f in good:
            assert len(f.result(timeout=120).images) == 2
        assert srv.stats["invalid"] == 3 and srv.stats["refused"] == 1
        assert cancelled.cancelled() or cancelled.done()
    finally:
        srv.close(timeout=60)
