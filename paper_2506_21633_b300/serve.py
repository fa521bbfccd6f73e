"""Serving loop with continuous batching over resident scenes.

Clients `submit()` render or gradient requests (a scene, 1..many views,
for gradients a target image per view) and get a Future.  One scheduler
thread owns the GPU:

- Scenes stay resident: all scene parameters live in one device tensor
  with a scene-offset table; every batch call references it directly.
- Continuous batching: whenever one of `n_slots` execution slots (a CUDA
  stream with its own workspace and buffers) is free, the scheduler forms a
  batch from the pending requests in arrival order -- same kind, at most one
  gradient request per scene (their gradients must not mix), bounded views
  and pixels -- and enqueues it as one multi-scene call sequence on that
  slot's stream.  Requests that arrive while other batches run are admitted
  into the next batch as soon as a slot and memory free up; batches on
  different slots overlap on the device.
- Admission by HBM footprint: a batch starts only if its estimated device
  footprint (workspace for its views and instances, image and gradient
  buffers) plus that of the batches in flight stays within the budget; a
  request that alone exceeds the budget is refused with AdmissionError.
- Instance capacity is estimated per scene (instances per view-Gaussian
  slot, learned from the device status of earlier batches); a batch that
  overflows is re-queued at the head with a larger estimate.
- Results (images, and gradients of the request's scene w.r.t. its own L1
  loss) are copied to page-locked host memory on the slot's stream (two
  buffer sets per slot, used in turn); a second host thread copies them into
  the request's own arrays and resolves its future, so the scheduler thread
  only forms, launches and retires batches.  The request's latency runs
  from submit() to the moment its result is host-visible.

All arithmetic runs in libsdgr.so; this module only schedules.
"""
from __future__ import annotations

import collections
import concurrent.futures
import queue
import threading
import time

import numpy as np
import torch

from . import _lib as L
from .render import Renderer, _stream_handle, l1_loss


class AdmissionError(RuntimeError):
    pass


class Request:
    __slots__ = ("rid", "scene", "views", "kind", "target", "npix", "t_submit", "t_done", "future", "attempts",
                 "sums")

    def __init__(self, rid, scene, views, kind, target):
        self.rid, self.scene, self.views, self.kind, self.target = rid, scene, views, kind, target
        self.npix = sum(int(v["NA"]) * int(v["NR"]) for v in views)
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.future = concurrent.futures.Future()
        self.attempts = 0
        # this request's share of a batch's workspace capacities (views,
        # view-Gaussian slots, pixels, tiles; they add up over a batch), set
        # by the server on first use
        self.sums = None


class Result:
    __slots__ = ("images", "grads", "loss", "latency_s", "batch_size")

    def __init__(self, images, grads, loss, latency_s, batch_size):
        self.images, self.grads, self.loss, self.latency_s, self.batch_size = images, grads, loss, latency_s, batch_size


def _resolve(future, result=None, exc=None):
    """Set a request's outcome unless the client cancelled it meanwhile."""
    try:
        if exc is not None:
            future.set_exception(exc)
        else:
            future.set_result(result)
    except concurrent.futures.InvalidStateError:
        pass


def _grow(buf, n, dtype, device=None, pinned=False):
    if buf is not None and buf.numel() >= n:
        return buf
    n = max(n, 1024)
    if pinned:
        return torch.empty(int(n * 1.25), dtype=dtype, pin_memory=True)
    return torch.empty(int(n * 1.25), dtype=dtype, device=device)


class _HostSet:
    """Page-locked result buffers of one batch.  A slot has two, used in
    turn: the finisher thread copies one batch's results out of one set
    while the slot's next batch writes into the other."""

    def __init__(self):
        self.h_images = self.h_grads = self.h_loss = None
        self.free = threading.Event()
        self.free.set()


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.renderer = Renderer(device=device)
        self.device = device
        self.images = self.dLdS = self.targets = self.loss = None
        self.grads = None
        self.h_targets = None
        self.sets = [_HostSet(), _HostSet()]
        self.flip = 0
        self.hs = None  # the host set of the batch in flight
        self.h_status = torch.zeros(4, dtype=torch.int32, pin_memory=True)
        self.event = torch.cuda.Event(enable_timing=True)
        self.ev_start = torch.cuda.Event(enable_timing=True)
        self.batch = None
        self.footprint = 0
        self.seg = None

    def preallocate(self, npix, nreq, ngrad, device):
        f = torch.float32
        self.images = _grow(None, npix, f, device)
        self.dLdS = _grow(None, npix, f, device)
        self.targets = _grow(None, npix, f, device)
        self.loss = _grow(None, nreq, f, device)
        self.grads = _grow(None, ngrad, f, device)
        self.h_targets = _grow(None, npix, f, pinned=True)
        for hs in self.sets:
            hs.h_images = _grow(None, npix, f, pinned=True)
            hs.h_loss = _grow(None, nreq, f, pinned=True)
            hs.h_grads = _grow(None, ngrad, f, pinned=True)


class Server:
    def __init__(self, scenes, hbm_budget_bytes, n_slots=3, max_batch_views=64, max_batch_pixels=1 << 26,
                 device=None, inst_per_slot=16.0, preallocate=False):
        """preallocate: size every slot's image, target and gradient buffers
        (device and page-locked host) for the largest batch at start-up, so
        that no buffer grows while requests are served (page-locked
        allocations are slow; growing them inside the scheduler thread stalls
        every request queued behind)."""
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        offs = [0]
        for s in scenes:
            offs.append(offs[-1] + int(np.asarray(s).shape[0]))
        self.offs = offs
        host = np.concatenate([np.asarray(s, dtype=np.float32) for s in scenes]) if scenes else np.zeros((0, 12), np.float32)
        self.params = torch.from_numpy(host).to(self.device).contiguous()
        self.n_total = offs[-1]
        self.budget = int(hbm_budget_bytes)
        self.max_views, self.max_pixels = int(max_batch_views), int(max_batch_pixels)
        self.inst_ratio = [float(inst_per_slot)] * len(scenes)
        self.cfg = L.make_cfg()
        self.slots = [_Slot(self.device) for _ in range(n_slots)]
        if preallocate:
            for sl in self.slots:
                sl.preallocate(self.max_pixels, self.max_views, self.n_total * 12, self.device)
        self._pending = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self._next_id = 0
        self.inflight_bytes = 0
        self.stats = {"batches": 0, "requests": 0, "refused": 0, "invalid": 0, "requeued": 0, "batch_sizes": [],
                      "max_inflight": 0, "host_form_s": 0.0, "host_launch_s": 0.0, "host_stage_targets_s": 0.0,
                      "host_prepare_s": 0.0, "host_grow_s": 0.0, "host_retire_s": 0.0, "host_finish_s": 0.0,
                      "gpu_batch_s": 0.0}
        # results are copied out and futures resolved by a second thread, so
        # that the scheduler thread only forms, launches and retires batches
        self._done = queue.SimpleQueue()
        self._finisher = threading.Thread(target=self._finish_loop, name="sdgr-finisher", daemon=True)
        self._finisher.start()
        self._thread = threading.Thread(target=self._loop, name="sdgr-server", daemon=True)
        self._thread.start()

    # -- client side ---------------------------------------------------------
    def submit(self, scene, views, kind="render", target=None):
        """kind: 'render' or 'gradient'; target: host float32 images (list
        of [NR, NA] arrays or one flat array) for gradient requests."""
        with self._cv:
            rid = self._next_id
            self._next_id += 1
        views = [dict(v, scene=int(scene)) for v in views]
        req = Request(rid, int(scene), views, kind, None)
        try:
            if kind not in ("render", "gradient") or not (0 <= req.scene < len(self.offs) - 1) or not views:
                raise ValueError("bad request")
            if len(views) > self.max_views or req.npix > self.max_pixels:
                raise ValueError("request larger than a batch (%d views, %d pixels; limits %d, %d)"
                                 % (len(views), req.npix, self.max_views, self.max_pixels))
            self._sums(req)  # validates the views
            if kind == "gradient":
                # kept as the caller's arrays (no copy here); staged into
                # page-locked memory when the request's batch is launched
                parts = [np.asarray(x, dtype=np.float32) for x in
                         (target if isinstance(target, (list, tuple)) else [target])]
                if sum(x.size for x in parts) != req.npix:
                    raise ValueError("target size does not match the views")
                req.target = parts
        except (ValueError, L.SdgrError, TypeError) as e:
            with self._cv:
                self.stats["invalid"] += 1
            _resolve(req.future, exc=e if isinstance(e, ValueError) else ValueError(str(e)))
            return req.future
        if self._footprint([req]) > self.budget:
            with self._cv:
                self.stats["refused"] += 1
            _resolve(req.future, exc=AdmissionError("request footprint exceeds the HBM budget"))
            return req.future
        with self._cv:
            self._pending.append(req)
            self._cv.notify()
        return req.future

    def close(self, timeout=None):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join(timeout)
        self._done.put(None)
        self._finisher.join(timeout)

    # -- accounting ----------------------------------------------------------
    def _inst_estimate(self, reqs):
        est = 0.0
        for r in reqs:
            n = self.offs[r.scene + 1] - self.offs[r.scene]
            est += len(r.views) * n * self.inst_ratio[r.scene]
        return int(est * 1.25) + 4096

    def _sums(self, r):
        if r.sums is None:
            c = L.sdgr_caps_for(L.make_views(r.views), len(r.views), L.make_offsets(self.offs), len(self.offs) - 1, 0)
            r.sums = (c.max_views, c.max_view_gauss, c.max_pixels, c.max_tiles)
        return r.sums

    def _footprint(self, reqs):
        caps = L.SdgrCaps()
        caps.max_views, caps.max_view_gauss, caps.max_pixels, caps.max_tiles = (
            sum(x) for x in zip(*(self._sums(r) for r in reqs)))
        caps.max_scenes = len(self.offs) - 1
        caps.max_gaussians = self.n_total
        caps.max_instances = min(self._inst_estimate(reqs), 0x7fffffff)
        ws = L.sdgr_workspace_size(self.cfg, caps)
        npix = sum(r.npix for r in reqs)
        grad = any(r.kind == "gradient" for r in reqs)
        return ws + 4 * npix * (3 if grad else 1) + (self.n_total * 48 if grad else 0)

    # -- scheduler -----------------------------------------------------------
    def _form_batch(self):
        """Pending requests in arrival order that can share one call."""
        if not self._pending:
            return []
        kind = self._pending[0].kind
        batch, scenes, views, pixels = [], set(), 0, 0
        keep = collections.deque()
        scanned = 0
        while self._pending and scanned < 512:
            scanned += 1
            r = self._pending.popleft()
            if r.future.cancelled():
                continue
            ok = (r.kind == kind and views + len(r.views) <= self.max_views and pixels + r.npix <= self.max_pixels
                  and not (kind == "gradient" and r.scene in scenes))
            if ok and batch:
                ok = self.inflight_bytes + self._footprint(batch + [r]) <= self.budget
            elif ok:
                ok = self.inflight_bytes + self._footprint([r]) <= self.budget
            if ok:
                batch.append(r)
                scenes.add(r.scene)
                views += len(r.views)
                pixels += r.npix
            else:
                keep.append(r)
            if views >= self.max_views:
                break
        keep.extend(self._pending)
        self._pending = keep
        return batch

    def _launch(self, slot, batch):
        dev = self.device
        grad = batch[0].kind == "gradient"
        views = [v for r in batch for v in r.views]
        npix = sum(r.npix for r in batch)
        s = slot.stream
        sh = _stream_handle(s)
        hs = slot.sets[slot.flip]
        slot.flip ^= 1
        hs.free.wait()  # the finisher is done with this set's previous batch
        hs.free.clear()
        slot.hs = hs
        with torch.cuda.stream(s):
            slot.ev_start.record(s)
            t0 = time.perf_counter()
            slot.images = _grow(slot.images, npix, torch.float32, dev)
            hs.h_images = _grow(hs.h_images, npix, torch.float32, pinned=True)
            self.stats["host_grow_s"] += time.perf_counter() - t0
            r = slot.renderer
            t0 = time.perf_counter()
            r.prepare(self.params, views, self.offs, stream=s, check=False, instances=self._inst_estimate(batch))
            self.stats["host_prepare_s"] += time.perf_counter() - t0
            r.forward(images=slot.images, stream=s)
            seg, off = [], 0
            for q in batch:
                seg.append((off, q.npix))
                off += q.npix
            if grad:
                t0 = time.perf_counter()
                slot.dLdS = _grow(slot.dLdS, npix, torch.float32, dev)
                slot.targets = _grow(slot.targets, npix, torch.float32, dev)
                slot.h_targets = _grow(slot.h_targets, npix, torch.float32, pinned=True)
                slot.loss = _grow(slot.loss, len(batch), torch.float32, dev)
                hs.h_loss = _grow(hs.h_loss, len(batch), torch.float32, pinned=True)
                slot.grads = _grow(slot.grads, self.n_total * 12, torch.float32, dev)
                hs.h_grads = _grow(hs.h_grads, self.n_total * 12, torch.float32, pinned=True)
                self.stats["host_grow_s"] += time.perf_counter() - t0
                t0 = time.perf_counter()
                for q, (o, n) in zip(batch, seg):  # multi-threaded host copies (torch), no GIL held
                    p = o
                    for part in q.target:
                        slot.h_targets[p:p + part.size].copy_(torch.from_numpy(part.reshape(-1)))
                        p += part.size
                self.stats["host_stage_targets_s"] += time.perf_counter() - t0
                slot.targets[:npix].copy_(slot.h_targets[:npix], non_blocking=True)
                for k, (o, n) in enumerate(seg):
                    l1_loss(slot.images[o:o + n], slot.targets[o:o + n], slot.dLdS[o:o + n], slot.loss[k:k + 1],
                            stream=s)
                r.backward(slot.dLdS[:npix], slot.grads[:self.n_total * 12].view(-1, 12), stream=s)
                for q in batch:
                    a, b = self.offs[q.scene] * 12, self.offs[q.scene + 1] * 12
                    hs.h_grads[a:b].copy_(slot.grads[a:b], non_blocking=True)
                hs.h_loss[:len(batch)].copy_(slot.loss[:len(batch)], non_blocking=True)
            hs.h_images[:npix].copy_(slot.images[:npix], non_blocking=True)
            L.sdgr_copy_status_async(r.ws, slot.h_status.data_ptr(), sh)
            slot.event.record(s)
        slot.batch = batch
        slot.seg = seg
        slot.footprint = self._footprint(batch)
        self.inflight_bytes += slot.footprint
        self.stats["batches"] += 1
        self.stats["batch_sizes"].append(len(batch))
        self.stats["max_inflight"] = max(self.stats["max_inflight"], sum(sl.batch is not None for sl in self.slots))

    def _retire(self, slot):
        batch, seg, hs = slot.batch, slot.seg, slot.hs
        slot.batch = None
        slot.hs = None
        self.stats["gpu_batch_s"] += slot.ev_start.elapsed_time(slot.event) / 1e3
        self.inflight_bytes -= slot.footprint
        slot.footprint = 0
        code = int(slot.h_status[0])
        required = (int(slot.h_status[2].item()) & 0xffffffff) | (int(slot.h_status[3].item()) << 32)
        vg = sum(len(q.views) * (self.offs[q.scene + 1] - self.offs[q.scene]) for q in batch)
        if code == L.SDGR_ERR_CAPACITY:
            ratio = required / max(vg, 1) * 1.3
            for q in batch:
                self.inst_ratio[q.scene] = max(self.inst_ratio[q.scene], ratio)
                q.attempts += 1
            with self._cv:
                self.stats["requeued"] += len(batch)
                self._pending.extendleft(reversed(batch))
            hs.free.set()
            return
        if code != L.SDGR_OK:
            for q in batch:
                _resolve(q.future, exc=L.SdgrError("device status", code))
            hs.free.set()
            return
        ratio = required / max(vg, 1)
        for q in batch:  # running estimate of instances per view-Gaussian slot
            self.inst_ratio[q.scene] = 0.7 * self.inst_ratio[q.scene] + 0.3 * max(ratio, 1.0)
        self._done.put((batch, seg, hs))

    def _finish_loop(self):
        while True:
            job = self._done.get()
            if job is None:
                return
            t0 = time.perf_counter()
            try:
                self._finish(*job)
            except Exception as e:  # host-side failure: fail these requests, keep serving
                for q in job[0]:
                    _resolve(q.future, exc=e)
            finally:
                job[2].free.set()
            self.stats["host_finish_s"] += time.perf_counter() - t0

    def _finish(self, batch, seg, hs):
        for k, (q, (o, n)) in enumerate(zip(batch, seg)):
            # the request's own arrays, filled by multi-threaded copies out of
            # the slot's page-locked buffers (which the next batch reuses)
            flat = np.empty(n, dtype=np.float32)
            torch.from_numpy(flat).copy_(hs.h_images[o:o + n])
            imgs, p = [], 0
            for v in q.views:
                m = int(v["NA"]) * int(v["NR"])
                imgs.append(flat[p:p + m].reshape(int(v["NR"]), int(v["NA"])))
                p += m
            grads, loss = None, None
            if q.kind == "gradient":
                a, b = self.offs[q.scene] * 12, self.offs[q.scene + 1] * 12
                grads = np.empty(((b - a) // 12, 12), dtype=np.float32)
                torch.from_numpy(grads).view(-1).copy_(hs.h_grads[a:b])
                loss = float(hs.h_loss[k])
            now = time.perf_counter()
            q.t_done = now
            _resolve(q.future, Result(imgs, grads, loss, now - q.t_submit, len(batch)))
        with self._cv:
            self.stats["requests"] += len(batch)

    def _loop(self):
        while True:
            with self._cv:
                busy = any(sl.batch is not None for sl in self.slots)
                if self._stop and not self._pending and not busy:
                    return
                if not self._pending and not busy:
                    self._cv.wait(timeout=0.05)
                    continue
            progressed = False
            for sl in self.slots:
                if sl.batch is not None and sl.event.query():
                    t0 = time.perf_counter()
                    self._retire(sl)
                    self.stats["host_retire_s"] += time.perf_counter() - t0
                    progressed = True
            for sl in self.slots:
                if sl.batch is None:
                    t0 = time.perf_counter()
                    with self._cv:
                        batch = self._form_batch()
                    t1 = time.perf_counter()
                    self.stats["host_form_s"] += t1 - t0
                    if batch:
                        try:
                            self._launch(sl, batch)
                        except Exception as e:  # host-side failure: fail these requests, keep serving
                            sl.batch = None
                            for q in batch:
                                _resolve(q.future, exc=e)
                        self.stats["host_launch_s"] += time.perf_counter() - t1
                        progressed = True
            if not progressed:
                time.sleep(0.0002)
