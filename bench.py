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
# the FP32 pipe 128).  Derivation in the design notes.
ALG_OPS = {
    "intensity_fwd": (13, 1),
    "splat_fwd": (9, 1),
    "splat_bwd": (20, 1),
    "intensity_bwd": (28, 2),
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
    ap.add_argument("--workload", choices=["config3", "medium", "small"], default="config3",
                    help="medium: the config-3 scene with 8 views (profiling); small: a reduced scene for "
                         "quick checks (neither is a bench line)")
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
    from paper_2506_21633_b300 import _lib
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

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_t = torch.empty(npix, dtype=torch.float32, pin_memory=True)
        host_t.copy_(targets.cpu())
        tdev = torch.empty_like(targets)
        n_e2e = max(3, min(args.steps, 10))
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            tdev.copy_(host_t, non_blocking=True)
            state["t"] += 1
            r.prepare(p, views, check=False)
            r.forward(images=images)
            l1_loss(images, tdev, dLdS, loss)
            r.backward(dLdS, grads)
            adam_step(p, grads, m, v, LR, state["t"])
            _ = loss.item()
        torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        views_e2e = sum_over_ranks(V * n_e2e, dev)
        e2e = {"value": views_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(npix * 4),
               "d2h_bytes_per_step": 4, "steps": n_e2e,
               "how": "host->device copy of the 64 target images from pinned memory + the step + loss.item()"}

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

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "gaussians": int(params.shape[0]), "views_per_step": V,
                   "image": [views[0]["NR"], views[0]["NA"]], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (workspace %.1f GB per step)" % (r.workspace_bytes() / 1e9),
                   "pairs_per_step": {"computation_plane": pairs[0], "imaging_plane": pairs[1]},
                   "instances_per_step": int(r.n_inst)},
        "gaussian_pixel_evals_per_s": round((pairs[0] + pairs[1]) * world * args.steps / (ms_max / 1e3), 1),
        "plain": plain, "e2e": e2e, "roofline": roof, "gpu_launches": int(launches), "clocks": clocks,
    }
    return out, params, start, views


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


def main():
    args = parse()
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
