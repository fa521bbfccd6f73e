"""Autotuner of the raster launches.

Two knobs, both results-neutral (the images and gradients do not depend on
them beyond the order of float atomics across tiles):

- the schedule: how CTAs map to tiles ('tiles': one CTA per tile;
  'ordered': one CTA per non-empty tile, longest list first; 'persistent':
  resident CTAs pulling that list from a device counter);
- the staging batch of each raster kernel: how many Gaussian records a CTA
  stages into shared memory per batch (sdgr_stage_batch_options lists the
  sizes each kernel is built for).

The schedule is chosen on whole-step time; each kernel's staging batch on
that kernel's own device time (the workspace's stage events), one kernel at
a time with the others at their current choice.
"""
from __future__ import annotations

import torch

from . import _lib as L


def _time_steps(step, n, stream):
    step()  # first step under the new setting: not timed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / n


def tune_schedule(r, step, steps=2, schedules=("tiles", "ordered", "persistent"), on_change=None):
    """Time `steps` calls of step() (after one untimed call) under each
    schedule and keep the fastest.  r: the Renderer step() launches through;
    on_change(): called after each change of setting (e.g. to capture a CUDA
    graph of step again).  Returns (best, {schedule: ms per step})."""
    stream = torch.cuda.current_stream(r.device)
    times = {}
    for name in schedules:
        r.set_schedule(name)
        if on_change:
            on_change()
        times[name] = _time_steps(step, steps, stream)
    best = min(times, key=times.get)
    r.set_schedule(best)
    if on_change:
        on_change()
    return best, times


def tune_stage_batches(r, step, steps=2, kernels=L.RASTER_KERNELS):
    """For each raster kernel with more than one staging batch size, run
    step() once untimed and `steps` times with the stage events on under each
    size, and keep the size with the least device time in that kernel.
    step() must launch eagerly (not replay a graph captured earlier: a graph
    keeps the launch configuration it was captured with).  Returns
    {kernel: (best size, {size: ms per launch})}."""
    out = {}
    for kname in kernels:
        opts = L.sdgr_stage_batch_options(kname)
        if len(opts) < 2:
            continue
        cur = r.stage_batch.get(kname, opts[0])
        ms = {}
        for nb in opts:
            r.set_stage_batch(kname, nb)
            step()
            torch.cuda.synchronize(r.device)
            r.profile(True)
            r.profile_read(reset=True)
            for _ in range(steps):
                step()
            torch.cuda.synchronize(r.device)
            total, launches = r.profile_read(reset=True)[kname]
            r.profile(False)
            ms[nb] = total / max(launches, 1)
        best = min(ms, key=ms.get) if ms else cur
        r.set_stage_batch(kname, best)
        out[kname] = (best, ms)
    return out
