"""Batched optimisation steps: many views of many scenes (uneven Gaussian
counts and image sizes) in one call sequence, optionally captured once into
a CUDA graph and replayed.

One step = preprocess -> bin/sort -> intensity pass -> splat -> L1 ->
splat adjoint -> intensity adjoint -> parameter adjoint -> Adam, all on one
stream with no host synchronisation, so the sequence is capturable.  The
instance capacity is data dependent: `check()` reads the device status word
(one host sync); on overflow the workspace grows and the graph is captured
again.
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import tune
from .render import Renderer, _stream_handle, l1_loss, views_npix

DEFAULT_LR = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)  # means, log-scales, quaternions, opacity logit, P


def sh_degree_at(iteration, every=2500, max_degree=3):
    """SH degree schedule of the training set-up (Section III-B-3): one more
    degree every `every` iterations, up to `max_degree`."""
    return min(max_degree, max(0, int(iteration)) // int(every))


class FusedStep:
    """State and call sequence of one optimisation step over a batch.

    params: cuda float32 [N_total, 12] (updated in place); views: list of view
    dicts (each with its 'scene'); targets: cuda float32 flat images in view
    order; scene_offsets: N_total partition into scenes (default: one)."""

    def __init__(self, params, views, targets, scene_offsets=None, lr=DEFAULT_LR, b1=0.9, b2=0.999, eps=1e-15,
                 inst_slack=1.25, **cfg):
        assert params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()
        self.p = params
        self.views = list(views)
        self.scene_offsets = list(scene_offsets) if scene_offsets is not None else [0, params.shape[0]]
        self.targets = targets
        self.lr, self.b1, self.b2, self.eps = list(lr), b1, b2, eps
        dev = params.device
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grads = torch.zeros_like(params)
        npix = views_npix(self.views)
        assert targets.numel() == npix
        self.images = torch.empty(npix, dtype=torch.float32, device=dev)
        self.dLdS = torch.empty_like(self.images)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        self.r = Renderer(device=dev, inst_slack=inst_slack, **cfg)
        self.inst_slack = inst_slack
        self.r.prepare(self.p, self.views, self.scene_offsets)  # learns the instance count (host sync)
        self._reserve(int(self.r.n_inst * inst_slack) + 4096)
        self.graph = None

    def _reserve(self, instances):
        self.r.prepare(self.p, self.views, self.scene_offsets, instances=instances)

    def enqueue(self, stream=None):
        """Enqueue one step on `stream` (default: the current stream)."""
        r = self.r
        r.prepare(self.p, self.views, self.scene_offsets, stream=stream, check=False)
        r.forward(images=self.images, stream=stream)
        l1_loss(self.images, self.targets, self.dLdS, self.loss, stream=stream)
        r.backward(self.dLdS, self.grads, stream=stream)
        L.sdgr_adam_step_device(self.p.data_ptr(), self.grads.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                self.p.shape[0], self.lr, self.b1, self.b2, self.eps, self.step_dev.data_ptr(),
                                _stream_handle(stream))

    def capture(self):
        """Capture one step into a CUDA graph (the step's launches, memsets
        and plan uploads become graph nodes); replaying it runs the step."""
        self.graph = self.capture_graph()
        return self

    def capture_graph(self, steps=1, targets=None, profile=False):
        """A new CUDA graph of `steps` consecutive optimisation steps (one
        replay runs them all, back to back, with no host work between).

        targets: flat target images this graph's L1 reads (default: the
        current ones); the graph keeps their address, so two graphs over two
        target buffers let a caller refill one buffer while the other is in
        use.  profile=True: the stage events of the captured calls become
        graph nodes; once a replay has finished, `self.r.profile_read()`
        returns that replay's per-stage times.  Sets `self.graph_launches`
        to the kernel launches one replay runs."""
        if targets is not None:
            assert targets.numel() == self.targets.numel() and targets.device == self.targets.device
            self.targets = targets
        side = torch.cuda.Stream(device=self.p.device)
        side.wait_stream(torch.cuda.current_stream(self.p.device))
        # one step on a side stream before capture (library set-up, lazy module
        # loading); the optimiser state is restored afterwards, so capturing
        # does not advance the optimisation
        state = (self.p, self.m, self.v, self.step_dev)
        saved = [t.clone() for t in state]
        with torch.cuda.stream(side):
            self.enqueue(side)
        torch.cuda.current_stream(self.p.device).wait_stream(side)
        torch.cuda.synchronize(self.p.device)
        for t, s0 in zip(state, saved):
            t.copy_(s0)
        torch.cuda.synchronize(self.p.device)
        g = torch.cuda.CUDAGraph()
        if profile:
            self.r.profile(True)
            self.r.profile_read(reset=True)  # nothing pending but the captured steps' events
        l0 = L.sdgr_launch_count()
        with torch.cuda.graph(g):
            for _ in range(int(steps)):
                self.enqueue()
        self.graph_launches = L.sdgr_launch_count() - l0  # kernel launches captured = launches per replay
        if profile:
            self.r.profile(False)  # later eager calls record nothing; the captured events stay pending
        return g

    def autotune(self, schedules=("tiles", "ordered", "persistent"), steps=3, stage_batches=True):
        """Pick the raster schedule (whole steps timed under each, re-capturing
        the graph if one is captured) and then each raster kernel's staging
        batch (that kernel's device time, eager steps); see `tune`.  The
        optimiser state is restored afterwards, so tuning does not advance the
        optimisation.  Returns (best schedule, {schedule: ms per step}); the
        staging batches chosen and their times are in `self.stage_batch_ms`."""
        state = (self.p, self.m, self.v, self.step_dev)
        saved = [t.clone() for t in state]
        captured = self.graph is not None

        def recapture():
            if captured:
                self.graph = None
                self.capture()

        best, times = tune.tune_schedule(self.r, self.step, steps=steps, schedules=schedules, on_change=recapture)
        if not self.check():
            raise RuntimeError("instance capacity exceeded while tuning")
        self.stage_batch_ms = {}
        if stage_batches:
            self.graph = None  # staging batches are tuned on eager steps
            self.stage_batch_ms = tune.tune_stage_batches(self.r, self.enqueue, steps=steps)
            if not self.check():
                raise RuntimeError("instance capacity exceeded while tuning")
            recapture()
        for t, s0 in zip(state, saved):
            t.copy_(s0)
        torch.cuda.synchronize(self.p.device)
        self.schedule_ms = times
        return best, times

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.enqueue()

    def check(self):
        """Host sync; on instance overflow grow the workspace (and recapture).
        Returns True if the last step ran within capacity."""
        torch.cuda.synchronize(self.p.device)
        code, required = self.r.status()
        if code == L.SDGR_OK:
            return True
        if code != L.SDGR_ERR_CAPACITY:
            raise L.SdgrError("device status", code)
        had_graph = self.graph is not None
        self.graph = None
        self._reserve(int(required * self.inst_slack) + 4096)
        if had_graph:
            self.capture()
        return False

    def loss_value(self):
        return float(self.loss.item())

    # -- checkpoint / resume ---------------------------------------------------
    def state_dict(self):
        """Optimisation state (parameters, Adam moments, device step count,
        learning rates) as host tensors; `torch.save` writes it."""
        torch.cuda.synchronize(self.p.device)
        return {"params": self.p.detach().cpu().clone(), "m": self.m.cpu().clone(), "v": self.v.cpu().clone(),
                "step": self.step_dev.cpu().clone(), "lr": list(self.lr), "b1": self.b1, "b2": self.b2,
                "eps": self.eps, "scene_offsets": list(self.scene_offsets)}

    def load_state_dict(self, state):
        """Restore a state_dict() in place (same Gaussian count); a captured
        graph stays valid because the tensors keep their storage."""
        if tuple(state["params"].shape) != tuple(self.p.shape):
            raise ValueError("checkpoint holds %s parameters, this step %s" % (tuple(state["params"].shape),
                                                                              tuple(self.p.shape)))
        with torch.no_grad():
            self.p.copy_(state["params"])
            self.m.copy_(state["m"])
            self.v.copy_(state["v"])
            self.step_dev.copy_(state["step"])
        self.lr = list(state["lr"])
        self.b1, self.b2, self.eps = state["b1"], state["b2"], state["eps"]
        torch.cuda.synchronize(self.p.device)


def plain_step(renderer, params, views, targets, grads, images, dLdS, loss, scene_offsets=None, stream=None):
    """Reference schedule without batching: one view at a time (preprocess,
    sort, forward, loss, adjoint into the accumulated gradient), with a
    stream synchronisation after each view."""
    s = stream if stream is not None else torch.cuda.current_stream()
    offs = list(scene_offsets) if scene_offsets is not None else [0, params.shape[0]]
    off = 0
    for k, v in enumerate(views):
        n = int(v["NA"]) * int(v["NR"])
        sc = int(v.get("scene", 0))
        # one view of one scene: pass that scene's slice with a one-scene table
        sub = params[offs[sc]:offs[sc + 1]]
        gsub = grads[offs[sc]:offs[sc + 1]]
        vv = dict(v, scene=0)
        renderer.prepare(sub, [vv], [0, sub.shape[0]], stream=s, check=False)
        renderer.forward(images=images[off:off + n], stream=s)
        l1_loss(images[off:off + n], targets[off:off + n], dLdS[off:off + n], loss, stream=s)
        renderer.backward(dLdS[off:off + n], gsub, accumulate=k > 0 and _seen(views[:k], sc), stream=s)
        s.synchronize()
        off += n


def _seen(prev_views, scene):
    return any(int(v.get("scene", 0)) == scene for v in prev_views)
