#!/usr/bin/env python
"""Benchmark of the B300 SAR Gaussian rasterizer (SDGR of SAR-GS).

One step = one fused optimisation step over a batch of views: preprocess
(projection), bin/sort, intensity pass, imaging splat, L1 loss, splat
adjoint, intensity adjoint, parameter adjoint, Adam -- every kernel of the
hot path, on synthetic inputs shaped like the paper's (a 6x3x2 m vehicle-
sized box of 300k randomly rotated Gaussians, 64 views with grazing angles
U[30, 60] deg, 1024x1024 images at 0.01 m).  The L1 target is the rendering
of the unperturbed scene; the optimised scene is a perturbed copy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sdgr|reference]

For N > 1 (one process per GPU under torchrun) every rank runs its own
independent replica of the workload (different views): weak scaling, no
collective on the data path; rank 0 prints one JSON line.  `--impl
reference` times the FP64 CPU oracle on the host cores instead (the paper
ships no code to run), one view per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd views/s at 300k Gaussians, 1024² (batched vs plain); serving p50/p99 ms"
UNIT = "views/s"

# Algorithmic work per in-cutoff (pixel, Gaussian) pair: (FP32 ops, MUFU ops).
# FP32-pipe-equivalent ops = fp32 + 8 * mufu (the SFU has 16 lanes per SM,
# the FP32 pipe 128).  The exponent counts 5 ops (a quadratic in the pixel's
# tile-local coordinates with per-tile coefficients).  Derivation in the
# design notes.
ALG_OPS = {
    "intensity_fwd": (11, 1),
    "splat_fwd": (7, 1),
    "splat_bwd": (18, 1),
    "intensity_bwd": (26, 2),
}
PLANE = {"intensity_fwd": 0, "splat_fwd": 1, "splat_bwd": 1, "intensity_bwd": 0}
KERNEL_NAME = {"intensity_fwd": "k_intensity_fwd", "splat_fwd": "k_splat_fwd", "splat_bwd": "k_splat_bwd",
               "intensity_bwd": "k_intensity_bwd", "preprocess": "k_preprocess", "depth_sort": "k_radix_*",
               "bin": "k_emit+k_radix_*+k_ranges", "param_bwd": "k_param_bwd"}
LR = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]  # means, log-scales, quaternions, opacity logit, P


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["sdgr", "reference"], default="sdgr")
    ap.add_argument("--requests", type=int, default=1000, help="serving: measured requests")
    ap.add_argument("--workload", choices=["config3", "medium", "small", "config4", "serve"], default="config3",
                    help="medium: the config-3 scene with 8 views (profiling); small: a reduced scene for "
                         "quick checks (neither is a bench line)")
    ap.add_argument("--schedule", choices=["auto", "tiles", "ordered", "persistent"], default="auto",
                    help="raster launch policy; auto times each before the timed region and keeps the fastest")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------
def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_setup(backend):
    import torch.distributed as dist
    rank, world, _ = rank_info()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
      "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
      "clocks_event_reasons.sw_power_cap")
_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x for x in vis.split(",") if x.strip() != ""]
        self.index = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + _Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.index],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            out = self.proc.communicate(timeout=10)[0]
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out = ""
        sm, smax, power, reasons = [], [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(_REASONS, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": "no samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# peaks
# ---------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def alu_peak_tops(sms, mhz):
    """FP32-pipe peak: SMs x 128 lanes x clock (ops/s), in Tops/s."""
    return sms * 128 * mhz * 1e6 / 1e12


def kernel_traffic(stage):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    rec = d.get(KERNEL_NAME.get(stage, stage))
    if not rec:
        return None
    src = os.path.join(ROOT, rec.get("source", ""))
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != rec.get("source_sha256_16"):
        return None
    return rec.get("dram_bytes_per_launch_full")


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload(name, rank):
    import sdgr_scenes as sc
    if name == "medium":
        params, views = sc.config3()
        views = views[:8]
        desc = "profiling case: the 300k-Gaussian config-3 scene, 8 of its 64 views (not the headline workload)"
    elif name == "small":
        params, views = sc.config3(n=30000, n_views=8, size=256, res=0.04)
        desc = "reduced check: 30k Gaussians, 8 views, 256x256 (not the headline workload)"
    else:
        params, views = sc.config3()
        desc = ("fused fwd+bwd+Adam step: 300k Gaussians in a 6x3x2 m box (random rotations, log-normal "
                "scales), 64 views (grazing U[30,60] deg), 1024x1024 at 0.01 m, batched")
    if rank > 0:  # independent replica: same shape, other views
        views = sc.random_views(len(views), seed=303 + 1000 * rank, size=views[0]["NA"], res=views[0]["dA"])
    start = sc.perturb(params, seed=17)
    return params, start, views, desc


def run_sdgr(args):
    import numpy as np
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist_setup("nccl")
    dev = torch.device("cuda", local)
    from paper_2506_21633_b300 import _lib, tune
    from paper_2506_21633_b300.render import Renderer, adam_step, l1_loss, views_npix

    params, start, views, desc = workload(args.workload, rank)
    V = len(views)
    npix = views_npix(views)
    stream = torch.cuda.current_stream(dev)

    # targets: rendering of the unperturbed scene
    tgt_renderer = Renderer(device=dev)
    p_true = torch.from_numpy(params.astype(np.float32)).to(dev).contiguous()
    tgt_renderer.prepare(p_true, views)
    targets = tgt_renderer.forward()
    torch.cuda.synchronize(dev)
    del tgt_renderer

    p = torch.from_numpy(start.astype(np.float32)).to(dev).contiguous()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    grads = torch.empty_like(p)
    images = torch.empty(npix, dtype=torch.float32, device=dev)
    dLdS = torch.empty_like(images)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    r = Renderer(device=dev)
    r.prepare(p, views)  # learns the instance capacity (one host sync)
    state = {"t": 0}

    def step():
        state["t"] += 1
        r.prepare(p, views, check=False)
        r.forward(images=images)
        l1_loss(images, targets, dLdS, loss)
        r.backward(dLdS, grads)
        adam_step(p, grads, m, v, LR, state["t"])

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    code, required = r.status()
    if code != _lib.SDGR_OK:  # capacity grew during warm-up: re-plan once
        r.prepare(p, views, instances=int(required * 1.2))
        for _ in range(max(args.warmup, 1)):
            step()
        torch.cuda.synchronize(dev)
        code, required = r.status()
        assert code == _lib.SDGR_OK, "device status %d" % code
    pairs = r.count_pairs()
    schedule_ms, stage_batch_ms = None, None
    if args.schedule == "auto":  # untimed: the schedule, then each raster kernel's staging batch
        _, schedule_ms = tune.tune_schedule(r, step, steps=2)
        schedule_ms = {k: round(v, 3) for k, v in schedule_ms.items()}
        stage_batch_ms = {k: {nb: round(ms, 3) for nb, ms in d.items()}
                          for k, (_, d) in tune.tune_stage_batches(r, step, steps=2).items()}
    else:
        r.set_schedule(args.schedule)
    r.profile(True)
    r.profile_read(reset=True)

    # ---- timed region (device time, CUDA events on the launching stream)
    sampler = ClockSampler(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = _lib.sdgr_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = _lib.sdgr_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    barrier()
    ms_local = ev0.elapsed_time(ev1)
    prof = r.profile_read(reset=True)
    r.profile(False)
    code, _ = r.status()
    assert code == _lib.SDGR_OK, "device status %d after the timed region" % code
    ms_max = max_over_ranks(ms_local, dev)
    views_total = sum_over_ranks(V * args.steps, dev)
    value = views_total / (ms_max / 1e3)
    ms_per_step = ms_max / args.steps

    # ---- plain: per-view calls with a stream sync after each view
    plain = None
    if not args.no_plain and rank == 0:
        rp = Renderer(device=dev)
        gacc = torch.empty_like(p)
        one = [views[0]]
        rp.prepare(p, one, instances=r.n_inst)  # the batch total bounds any single view
        n_plain_steps = 2
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        off = 0
        for s in range(n_plain_steps):
            off = 0
            for k, vw in enumerate(views):
                n = vw["NA"] * vw["NR"]
                rp.prepare(p, [vw], check=False)
                img_k = images[off:off + n]
                rp.forward(images=img_k)
                l1_loss(img_k, targets[off:off + n], dLdS[off:off + n], loss)
                rp.backward(dLdS[off:off + n], gacc, accumulate=k > 0)
                stream.synchronize()
                off += n
        torch.cuda.synchronize(dev)
        t_plain = (time.perf_counter() - t0) / n_plain_steps
        code, _ = rp.status()
        plain = {"value": V / t_plain, "unit": UNIT, "ms_per_step": t_plain * 1e3,
                 "how": "per-view preprocess/sort/fwd/loss/bwd calls, stream sync after each view"}
        del rp

    # ---- end to end through the public API with host buffers: every step copies
    # its targets from pinned host memory (on a copy stream, into one of two
    # device buffers, while the previous step computes) and reads its loss back
    # to the host (read after the next step has been enqueued)
    e2e = None
    if not args.no_e2e:
        host_t = torch.empty(npix, dtype=torch.float32, pin_memory=True)
        host_t.copy_(targets.cpu())
        tbuf = [torch.empty_like(targets) for _ in range(2)]
        loss_host = torch.zeros(2, dtype=torch.float32, pin_memory=True)
        copy_stream = torch.cuda.Stream(device=dev)
        ev_copied = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        ev_loss = [torch.cuda.Event() for _ in range(2)]
        n_e2e = max(3, min(args.steps, 10))
        losses = []

        def h2d(k):
            b = k % 2
            with torch.cuda.stream(copy_stream):
                if k >= 2:
                    copy_stream.wait_event(ev_used[b])  # step k - 2 has read this buffer
                tbuf[b].copy_(host_t, non_blocking=True)
                ev_copied[b].record(copy_stream)

        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h2d(0)
        for k in range(n_e2e):
            b = k % 2
            if k + 1 < n_e2e:
                h2d(k + 1)
            stream.wait_event(ev_copied[b])
            state["t"] += 1
            r.prepare(p, views, check=False)
            r.forward(images=images)
            l1_loss(images, tbuf[b], dLdS, loss)
            ev_used[b].record(stream)
            r.backward(dLdS, grads)
            adam_step(p, grads, m, v, LR, state["t"])
            loss_host[b].copy_(loss[0], non_blocking=True)
            ev_loss[b].record(stream)
            if k >= 1:
                ev_loss[1 - b].synchronize()
                losses.append(float(loss_host[1 - b]))
        ev_loss[(n_e2e - 1) % 2].synchronize()
        losses.append(float(loss_host[(n_e2e - 1) % 2]))
        torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        views_e2e = sum_over_ranks(V * n_e2e, dev)
        assert len(losses) == n_e2e and all(math.isfinite(x) for x in losses)
        e2e = {"value": views_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(npix * 4),
               "d2h_bytes_per_step": 4, "steps": n_e2e,
               "how": "every step: host->device copy of its 64 target images from pinned memory (copy stream, "
                      "double-buffered, overlapping the previous step) + the step + its loss read back to the host"}

    if rank != 0:
        return None

    # ---- roofline of the dominant kernel (live per-stage CUDA-event times)
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stage_ms = {k: (ms / max(n, 1), n) for k, (ms, n) in prof.items()}
    dom = max(prof, key=lambda k: prof[k][0])
    ms_launch, nl = stage_ms[dom]
    share = {k: round(prof[k][0] / max(sum(x[0] for x in prof.values()), 1e-9), 4) for k in prof}
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    if dom in ALG_OPS:
        fp, mu = ALG_OPS[dom]
        ops = pairs[PLANE[dom]] * (fp + 8 * mu)
        achieved = ops / (ms_launch / 1e3) / 1e12
        peak = alu_peak_tops(sms, sm_max)
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
                "frac": round(achieved / peak, 4), "traffic": kernel_traffic(dom), "kernel": KERNEL_NAME[dom],
                "peak_source": "SMs x 128 FP32 lanes x %.0f MHz (sm_max_mhz, %s)" % (sm_max, peak_src),
                "ops_per_pair": fp + 8 * mu, "pairs_per_launch": pairs[PLANE[dom]],
                "ms_per_launch": round(ms_launch, 4)}
        if clocks and clocks.get("sm_mhz"):
            roof["frac_at_measured_clock"] = round(achieved / alu_peak_tops(sms, clocks["sm_mhz"]), 4)
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": None,
                "traffic": kernel_traffic(dom), "kernel": KERNEL_NAME.get(dom, dom)}
    roof["stage_ms_per_step"] = {k: round(prof[k][0] / max(args.steps, 1), 4) for k in prof}
    roof["stage_share"] = share
    # every raster kernel against the same FP32-pipe peak (algorithmic ops per in-cutoff pair)
    alu_peak = alu_peak_tops(sms, sm_max)
    roof["raster_kernels"] = {}
    for k, (fp, mu) in ALG_OPS.items():
        if k in stage_ms and stage_ms[k][0] > 0:
            ach = pairs[PLANE[k]] * (fp + 8 * mu) / (stage_ms[k][0] / 1e3) / 1e12
            roof["raster_kernels"][KERNEL_NAME[k]] = {"ms_per_launch": round(stage_ms[k][0], 4),
                                                      "ops_per_pair": fp + 8 * mu, "achieved": round(ach, 3),
                                                      "frac": round(ach / alu_peak, 4)}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "gaussians": int(params.shape[0]), "views_per_step": V,
                   "image": [views[0]["NR"], views[0]["NA"]], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (workspace %.1f GB per step)" % (r.workspace_bytes() / 1e9),
                   "pairs_per_step": {"computation_plane": pairs[0], "imaging_plane": pairs[1]},
                   "instances_per_step": int(r.n_inst), "schedule": r.schedule,
                   "schedule_ms_per_step": schedule_ms, "stage_batch": stage_batches(r),
                   "stage_batch_ms_per_launch": stage_batch_ms},
        "gaussian_pixel_evals_per_s": round((pairs[0] + pairs[1]) * world * args.steps / (ms_max / 1e3), 1),
        "plain": plain, "e2e": e2e, "roofline": roof, "gpu_launches": int(launches), "clocks": clocks,
    }
    return out, params, start, views


def stage_batches(r):
    """Staging batch of each raster kernel in use (chosen, else the default)."""
    from paper_2506_21633_b300 import _lib
    return {k: r.stage_batch.get(k, _lib.sdgr_stage_batch_options(k)[0]) for k in _lib.RASTER_KERNELS}


def cpu_baseline(params, views, npix_view=None):
    """The FP64 oracle as it stands, on the host cores: one view of the same
    workload (forward + L1 + adjoint), timed once."""
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    p64 = np.asarray(params, dtype=np.float32).astype(np.float64)
    v = [views[0]]
    rng = np.random.default_rng(99)
    tgt = [rng.uniform(0.0, 0.05, size=(v[0]["NR"], v[0]["NA"]))]
    t0 = time.perf_counter()
    oracle.step(p64, v, tgt, oracle.cfg(), culled=True)
    dt = time.perf_counter() - t0
    return {"value": round(1.0 / dt, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "1 of the %d views (all %d Gaussians, %dx%d): FP64 forward + L1 + adjoint, culled mode, "
                      "%.1f s" % (len(views), p64.shape[0], v[0]["NR"], v[0]["NA"], dt)}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, one view of the
    workload per step (rank 0 only)."""
    rank, world, _ = rank_info()
    if rank != 0:
        return None
    import numpy as np
    import oracle
    params, start, views, desc = workload(args.workload, 0)
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    p64 = np.asarray(start, dtype=np.float32).astype(np.float64)
    rng = np.random.default_rng(99)

    def one(k):
        v = [views[k % len(views)]]
        tgt = [rng.uniform(0.0, 0.05, size=(v[0]["NR"], v[0]["NA"]))]
        oracle.step(p64, v, tgt, oracle.cfg(), culled=True)

    for k in range(max(args.warmup, 0)):
        one(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(k)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = ("one of the %d views per step (all %d Gaussians, %dx%d): FP64 forward + L1 + adjoint, culled mode"
              % (len(views), p64.shape[0], views[0]["NR"], views[0]["NA"]))
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "gaussians": int(p64.shape[0]), "views_per_step": 1,
                       "image": [views[0]["NR"], views[0]["NA"]], "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_uneven(args):
    """Uneven batch: 256 scenes (log-uniform 1k-500k Gaussians, vehicle boxes
    and buildings alternating), image sizes 256/512/1024, 8 views each; the
    whole batch is one graph-captured step, against plain per-view calls."""
    import numpy as np
    import torch
    import sdgr_scenes as sc
    from paper_2506_21633_b300 import _lib
    from paper_2506_21633_b300.batch import FusedStep, plain_step
    from paper_2506_21633_b300.render import Renderer, views_npix
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scenes, views = sc.uneven_batch(seed=4 + rank)
    offs = [0]
    for p in scenes:
        offs.append(offs[-1] + p.shape[0])
    true = np.concatenate(scenes)
    start = np.concatenate([sc.perturb(p, seed=17 + k) for k, p in enumerate(scenes)])
    V = len(views)
    tr = Renderer(device=dev)
    targets = tr.prepare(torch.from_numpy(true.astype(np.float32)).to(dev), views, offs).forward().clone()
    torch.cuda.synchronize(dev)
    del tr
    p = torch.from_numpy(start.astype(np.float32)).to(dev).contiguous()
    fs = FusedStep(p, views, targets, offs)
    fs.capture()
    schedule_ms = None
    if args.schedule == "auto":
        _, schedule_ms = fs.autotune(steps=2)
    elif args.schedule != fs.r.schedule:
        fs.r.set_schedule(args.schedule)
        fs.graph = None
        fs.capture()
    for _ in range(max(args.warmup, 1)):
        fs.step()
    fs.check()
    pairs = fs.r.count_pairs()
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        fs.step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    assert fs.check()
    ms = ev0.elapsed_time(ev1) / args.steps
    # plain: one view at a time, stream sync after each
    rp = Renderer(device=dev)
    rp.prepare(p[offs[0]:offs[1]], [dict(views[0], scene=0)], [0, offs[1]], instances=fs.r.n_inst)
    grads = torch.zeros_like(p)
    images = torch.empty(views_npix(views), dtype=torch.float32, device=dev)
    dLdS = torch.empty_like(images)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plain_step(rp, p, views, targets, grads, images, dLdS, loss, offs)
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    sizes = sorted({v["NA"] for v in views})
    return {"metric": "uneven-batch fwd+bwd views/s (batched graph-captured step vs plain per-view calls)",
            "value": round(V / (ms / 1e3), 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "uneven batch: %d scenes, %d..%d Gaussians (total %d), images %s, %d views"
                                   % (len(scenes), min(s.shape[0] for s in scenes), max(s.shape[0] for s in scenes),
                                      offs[-1], sizes, V),
                       "pairs_per_step": {"computation_plane": pairs[0], "imaging_plane": pairs[1]},
                       "instances_per_step": int(fs.r.n_inst), "schedule": fs.r.schedule,
                       "schedule_ms_per_step": {k: round(v, 3) for k, v in schedule_ms.items()} if schedule_ms else None,
                       "stage_batch": stage_batches(fs.r),
                       "stage_batch_ms_per_launch": {k: {nb: round(ms, 3) for nb, ms in d.items()}
                                                     for k, (_, d) in getattr(fs, "stage_batch_ms", {}).items()}
                       or None},
            "plain": {"value": round(V / t_plain, 3), "unit": UNIT, "s_per_step": round(t_plain, 3)},
            "gpu_launches": int(fs.graph_launches) * args.steps,
            "gpu_launches_how": "kernel launches captured in the step's graph x steps"}


def run_serving(args):
    """Serving: Poisson arrivals (mean 2 ms apart) of render and gradient
    requests over 32 resident scenes of 10k-1M Gaussians; 1-16 views per
    request, images of 256..2048 pixels, half render, half gradient."""
    import numpy as np
    import torch
    import sdgr_scenes as sc
    from paper_2506_21633_b300.serve import Server
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    rng = np.random.default_rng(5 + rank)
    scenes, meta = [], []
    for s in range(32):
        n = int(math.exp(rng.uniform(math.log(1e4), math.log(1e6))))
        if s % 2 == 0:
            scale = (n / 300000.0) ** (1.0 / 3.0)
            ext = (6.0 * scale, 3.0 * scale, 2.0 * scale)
            scenes.append(sc.vehicle_box_scene(n, seed=500 + s, extent=ext, center=(0.0, 0.0, ext[2] / 2)))
            meta.append((1.7 * max(ext), (0.0, 0.0, ext[2] / 2)))
        else:
            r2 = np.random.default_rng(500 + s)
            scenes.append(sc.box_surface_scene(n, sc._place_boxes(r2, 3, 60.0, 5.0, 20.0), r2))
            meta.append((76.8, (30.0, 30.0, 5.0)))
    sizes = (256, 512, 1024, 2048)
    pool = {sz: np.random.default_rng(sz).uniform(0.0, 0.05, size=(sz, sz)).astype(np.float32) for sz in sizes}
    budget = int(torch.cuda.get_device_properties(local).total_memory * 0.6)

    def drive(mean_s, n_warm, n_meas, seed):
        """Submit n_warm + n_meas requests with exponential inter-arrival
        times of mean `mean_s`; latency and throughput of the measured ones."""
        g = np.random.default_rng(seed)
        srv = Server(scenes, hbm_budget_bytes=budget, n_slots=3, max_batch_views=64, max_batch_pixels=1 << 26)
        futs, t_sched = [], time.perf_counter()
        nviews, t_sub = [], []
        for k in range(n_warm + n_meas):
            t_sched += g.exponential(mean_s)
            dt = t_sched - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            t_sub.append(time.perf_counter())
            s = int(g.integers(0, 32))
            nv = int(g.integers(1, 17))
            sz = int(g.choice(sizes))
            frame, center = meta[s]
            vs = sc.random_views(nv, seed=10000 + k, size=sz, res=frame / sz, center=center)
            if g.uniform() < 0.5:
                futs.append(srv.submit(s, vs, "render"))
            else:
                futs.append(srv.submit(s, vs, "gradient", [pool[sz]] * nv))
            nviews.append(nv)
        res = [f.result(timeout=3600) for f in futs]
        srv.close(timeout=600)
        meas = res[n_warm:]
        lat = np.array([r.latency_s for r in meas]) * 1e3
        done_views = sum(nviews[n_warm:])
        window = max(t + r.latency_s for t, r in zip(t_sub[n_warm:], meas)) - t_sub[n_warm]
        return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "mean_ms": round(float(lat.mean()), 3), "views_per_s": round(done_views / window, 2),
                "views": done_views, "requests": n_meas, "warmup_requests": n_warm, "window_s": round(window, 3),
                "offered_views_per_s": round(8.5 / mean_s, 1), "arrival_mean_ms": round(mean_s * 1e3, 3),
                "batches": srv.stats["batches"], "mean_batch": round(float(np.mean(srv.stats["batch_sizes"])), 2),
                "max_inflight": srv.stats["max_inflight"], "requeued": srv.stats["requeued"]}

    spec = drive(0.002, 50, args.requests, 5 + rank)
    # second run at 70 % of the throughput the first one sustained (1-16 views
    # per request: 8.5 on average): latency without a growing queue
    mean_s = 8.5 / (0.7 * spec["views_per_s"])
    sus = drive(mean_s, 20, max(100, min(args.requests, int(20.0 / mean_s))), 7 + rank)
    return {"metric": "serving p50/p99 ms and views/s (continuous batching, Poisson arrivals mean 2 ms)",
            "value": spec["p50_ms"], "unit": "ms (p50)", "p99_ms": spec["p99_ms"], "mean_ms": spec["mean_ms"],
            "views_per_s": spec["views_per_s"], "views": spec["views"], "requests": spec["requests"],
            "warmup_requests": spec["warmup_requests"], "window_s": spec["window_s"],
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "32 resident scenes, %d..%d Gaussians; requests 1-16 views, images 256..2048, "
                                   "render/gradient 1:1, Poisson arrivals mean 2 ms" %
                                   (min(s.shape[0] for s in scenes), max(s.shape[0] for s in scenes)),
                       "hbm_budget_bytes": budget, "slots": 3},
            "batches": spec["batches"], "mean_batch": spec["mean_batch"], "max_inflight": spec["max_inflight"],
            "requeued": spec["requeued"],
            "at_70pct_load": sus}


def main():
    args = parse()
    if args.workload == "serve" and args.impl == "sdgr":
        t0 = time.perf_counter()
        out = run_serving(args)
        out["wall_s"] = round(time.perf_counter() - t0, 2)
        if rank_info()[0] == 0:
            print(json.dumps(out), flush=True)
        return 0
    if args.workload == "config4" and args.impl == "sdgr":
        out = run_uneven(args)
        if out is not None and rank_info()[0] == 0:
            print(json.dumps(out), flush=True)
        return 0
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return 0
    res = run_sdgr(args)
    if res is None:
        return 0
    out, params, start, views = res
    _, world, _ = rank_info()
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(start, views)
    else:
        out["cpu_baseline"] = None
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
