"""Admission and batch formation of the serving loop, on CPU (no GPU: the
scheduler object is built without its device state; only host-side
capacity arithmetic of the C ABI is used)."""
import collections


import sdgr_scenes as sc


def _server(budget, max_views=64, n_scenes=3, n_per_scene=1000):
    from paper_2506_21633_b300 import _lib as L
    from paper_2506_21633_b300.serve import Server
    L.lib()
    s = object.__new__(Server)
    s.offs = [k * n_per_scene for k in range(n_scenes + 1)]
    s.n_total = s.offs[-1]
    s.budget = budget
    s.max_views, s.max_pixels = max_views, 1 << 26
    s.inst_ratio = [16.0] * n_scenes
    s.cfg = L.make_cfg()
    s._pending = collections.deque()
    s.inflight_bytes = 0
    return s


def _req(rid, scene, kind, nviews=2, size=64):
    from paper_2506_21633_b300.serve import Request
    views = [dict(sc.make_view(10.0 * k, 40.0, 0.05, 0.05, size, size), scene=scene) for k in range(nviews)]
    return Request(rid, scene, views, kind, None)


def test_batches_follow_arrival_order_and_kind():
    s = _server(budget=1 << 40)
    for rid, (sc_, kind) in enumerate([(0, "render"), (1, "gradient"), (1, "render"), (2, "render")]):
        s._pending.append(_req(rid, sc_, kind))
    b = s._form_batch()
    assert [r.rid for r in b] == [0, 2, 3]          # renders, in arrival order
    assert [r.rid for r in s._pending] == [1]      # the gradient request waits for its own batch
    b = s._form_batch()
    assert [r.rid for r in b] == [1]


def test_one_gradient_request_per_scene():
    s = _server(budget=1 << 40)
    for rid, sc_ in enumerate([0, 0, 1, 0]):
        s._pending.append(_req(rid, sc_, "gradient"))
    assert [r.rid for r in s._form_batch()] == [0, 2]
    assert [r.rid for r in s._form_batch()] == [1]
    assert [r.rid for r in s._form_batch()] == [3]


def test_budget_and_view_limits():
    one = _server(budget=1 << 40)._footprint([_req(0, 0, "render")])
    s = _server(budget=int(2.5 * one))
    for rid in range(5):
        s._pending.append(_req(rid, rid % 3, "render"))
    b = s._form_batch()
    assert 1 <= len(b) <= 2 and s._footprint(b) <= s.budget
    s.inflight_bytes = s.budget  # everything in flight: nothing more is admitted
    assert s._form_batch() == []
    s.inflight_bytes = 0
    s2 = _server(budget=1 << 40, max_views=5)
    for rid in range(4):
        s2._pending.append(_req(rid, 0, "render", nviews=2))
    assert len(s2._form_batch()) == 2  # 4 views; a third request would exceed 5


def test_cancelled_requests_are_dropped():
    s = _server(budget=1 << 40)
    reqs = [_req(k, 0, "render") for k in range(3)]
    reqs[1].future.cancel()
    s._pending.extend(reqs)
    assert [r.rid for r in s._form_batch()] == [0, 2]


def test_sh_degree_schedule():
    from paper_2506_21633_b300.batch import sh_degree_at
    assert [sh_degree_at(i) for i in (0, 2499, 2500, 4999, 5000, 7500, 30000)] == [0, 0, 1, 1, 2, 3, 3]
