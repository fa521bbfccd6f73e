"""Seeded synthetic scenes and radar view sets.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle.  It draws raw Gaussian parameters and radar geometries from
fixed distributions and holds none of the renderer's arithmetic (no
projection, no activation, no compositing).

Raw parameter layout, one row of 12 per Gaussian (float32 for the GPU,
float64 for the oracle):
    [ mu_x, mu_y, mu_z, opacity_logit,
      log_s_x, log_s_y, log_s_z, P,
      q_w, q_x, q_y, q_z ]

A view is a dict {phi, theta, dA, dR, NA, NR, center(3), scene}:
phi = radar azimuth angle and theta = grazing angle (radians), dA/dR =
azimuth / slant-range pixel size (m), NA/NR = image columns / rows, center
= the world point the beam is centred on.

The workloads mirror the paper's experiments (simplified buildings in the
forward-rendering study, vehicle-sized targets, multi-view circular tracks
at a fixed altitude); the data sets themselves (MSTAR, CAD renders) are not
available, so these seeded scenes stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

OPACITY_MAX = 1.0 - 2.0 ** -20


def _logit(o):
    # raw parameter for a drawn opacity value (input generation only)
    o = np.clip(o, 1e-12, OPACITY_MAX)
    return np.log(o) - np.log1p(-o)


def make_view(phi_deg, theta_deg, dA, dR, NA, NR, center=(0.0, 0.0, 0.0), scene=0):
    return {
        "phi": math.radians(phi_deg),
        "theta": math.radians(theta_deg),
        "dA": float(dA),
        "dR": float(dR),
        "NA": int(NA),
        "NR": int(NR),
        "center": tuple(float(c) for c in center),
        "scene": int(scene),
    }


def _pack(mu, opa, log_s, P, q):
    n = mu.shape[0]
    out = np.empty((n, 12), dtype=np.float64)
    out[:, 0:3] = mu
    out[:, 3] = _logit(opa)
    out[:, 4:7] = log_s
    out[:, 7] = P
    out[:, 8:12] = q
    return out


def random_cube_scene(n, half=5.0, s_lo=0.05, s_hi=0.5, seed=1, center=(0.0, 0.0, 0.0)):
    """Isotropic Gaussians, means uniform in a cube, log-uniform scales."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-half, half, size=(n, 3)) + np.asarray(center)
    s = np.exp(rng.uniform(math.log(s_lo), math.log(s_hi), size=n))
    log_s = np.repeat(np.log(s)[:, None], 3, axis=1)
    P = rng.uniform(0.0, 1.0, size=n)
    opa = rng.uniform(0.2, 1.0, size=n)
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    return _pack(mu, opa, log_s, P, q)


def config1():
    """Plain forward: 2,000 Gaussians in a 10 m cube, one 128x128 view at
    0.1 m, 45 deg."""
    params = random_cube_scene(2000, seed=1)
    views = [make_view(0.0, 45.0, 0.1, 0.1, 128, 128)]
    return params, views


def _place_boxes(rng, count, area, lo, hi):
    boxes = []
    tries = 0
    while len(boxes) < count:
        tries += 1
        if tries > 10000:
            raise RuntimeError("could not place boxes")
        sx, sy, sz = rng.uniform(lo, hi, size=3)
        x0 = rng.uniform(0.0, area - sx)
        y0 = rng.uniform(0.0, area - sy)
        ok = True
        for (bx, by, _, bsx, bsy, _) in boxes:
            if x0 < bx + bsx + 1.0 and bx < x0 + sx + 1.0 and y0 < by + bsy + 1.0 and by < y0 + sy + 1.0:
                ok = False
                break
        if ok:
            boxes.append((x0, y0, 0.0, sx, sy, sz))
    return boxes


def box_surface_scene(n, boxes, rng, s_lo=0.05, s_hi=0.3, s_normal=0.01, ground=None):
    """Gaussians on the exposed faces of axis-aligned boxes (4 walls + roof),
    area-weighted, flattened along each face normal; optional ground plane
    rectangle (x0, y0, x1, y1) at z=0 with its own share of the points."""
    faces = []  # (origin, u_axis, v_axis, normal_axis, size_u, size_v)
    for (x0, y0, z0, sx, sy, sz) in boxes:
        faces.append(((x0, y0, z0 + sz), 0, 1, 2, sx, sy))         # roof
        faces.append(((x0, y0, z0), 0, 2, 1, sx, sz))              # wall y=y0
        faces.append(((x0, y0 + sy, z0), 0, 2, 1, sx, sz))         # wall y=y1
        faces.append(((x0, y0, z0), 1, 2, 0, sy, sz))              # wall x=x0
        faces.append(((x0 + sx, y0, z0), 1, 2, 0, sy, sz))         # wall x=x1
    if ground is not None:
        gx0, gy0, gx1, gy1 = ground
        faces.append(((gx0, gy0, 0.0), 0, 1, 2, gx1 - gx0, gy1 - gy0))
    areas = np.array([f[4] * f[5] for f in faces])
    which = rng.choice(len(faces), size=n, p=areas / areas.sum())
    mu = np.zeros((n, 3))
    log_s = np.zeros((n, 3))
    in_face = rng.uniform(math.log(s_lo), math.log(s_hi), size=(n, 2))
    for k, (org, ua, va, na, su, sv) in enumerate(faces):
        sel = which == k
        m = int(sel.sum())
        if m == 0:
            continue
        pts = np.zeros((m, 3))
        pts[:, 0], pts[:, 1], pts[:, 2] = org
        pts[:, ua] += rng.uniform(0.0, su, size=m)
        pts[:, va] += rng.uniform(0.0, sv, size=m)
        mu[sel] = pts
        ls = np.zeros((m, 3))
        ls[:, ua] = in_face[sel, 0]
        ls[:, va] = in_face[sel, 1]
        ls[:, na] = math.log(s_normal)
        log_s[sel] = ls
    P = rng.uniform(0.0, 1.0, size=n)
    opa = rng.uniform(0.2, 1.0, size=n)
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    return _pack(mu, opa, log_s, P, q)


def tank_scene(n, seed, s_lo=0.03, s_hi=0.12):
    """Vehicle-shaped reconstruction target (stand-in for the paper's tank
    CAD renders): Gaussians on the faces of a lower hull with tracks, an upper
    hull, a turret and a gun barrel (metres, ground at z = 0, centred on the
    origin)."""
    rng = np.random.default_rng(seed)
    boxes = [(-3.4, -1.8, 0.0, 6.8, 3.6, 0.5),    # tracks / lower hull
             (-3.1, -1.5, 0.5, 6.2, 3.0, 0.8),    # upper hull
             (-1.4, -1.1, 1.3, 2.4, 2.2, 0.7),    # turret
             (1.0, -0.12, 1.62, 3.2, 0.24, 0.24)]  # barrel
    return box_surface_scene(n, boxes, rng, s_lo=s_lo, s_hi=s_hi, s_normal=0.01)


def circular_views(thetas_deg, n_az, size, res, center=(0.0, 0.0, 0.8), phase_deg=0.0):
    """Circular tracks: n_az azimuths 360/n_az apart at each grazing angle
    (the multi-view acquisition of the paper's simulated targets)."""
    return [make_view(phase_deg + 360.0 * k / n_az, t, res, res, size, size, center)
            for t in thetas_deg for k in range(n_az)]


def config2(n=50000, n_views=72):
    """Forward+backward: 50k Gaussians on the faces of 3 boxes (5-20 m sides)
    in a 60x60 m area, 512x512 at 0.15 m, 72 views every 5 deg at 40 deg."""
    rng = np.random.default_rng(2)
    boxes = _place_boxes(rng, 3, 60.0, 5.0, 20.0)
    params = box_surface_scene(n, boxes, rng)
    center = (30.0, 30.0, 5.0)
    views = [make_view(5.0 * k, 40.0, 0.15, 0.15, 512, 512, center) for k in range(n_views)]
    return params, views


def vehicle_box_scene(n, seed, extent=(6.0, 3.0, 2.0), log_s_mean=math.log(0.02), log_s_sd=0.5,
                      center=(0.0, 0.0, 1.0)):
    """Vehicle-sized box of randomly rotated, log-normal-scaled Gaussians."""
    rng = np.random.default_rng(seed)
    ex = np.asarray(extent)
    mu = (rng.uniform(-0.5, 0.5, size=(n, 3)) * ex) + np.asarray(center)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    log_s = rng.normal(log_s_mean, log_s_sd, size=(n, 3))
    P = rng.uniform(0.0, 1.0, size=n)
    opa = rng.uniform(0.2, 1.0, size=n)
    return _pack(mu, opa, log_s, P, q)


def random_views(n_views, seed, size, res, theta_lo=30.0, theta_hi=60.0, center=(0.0, 0.0, 1.0), scene=0):
    rng = np.random.default_rng(seed)
    phis = rng.uniform(0.0, 360.0, size=n_views)
    thetas = rng.uniform(theta_lo, theta_hi, size=n_views)
    return [make_view(p, t, res, res, size, size, center, scene) for p, t in zip(phis, thetas)]


def config3(n=300000, n_views=64, size=1024, res=0.01):
    """Fused step: 300k Gaussians in a 6x3x2 m box, random rotations,
    log-normal scales, 64 views with grazing angle U[30,60] deg, 1024^2 at
    0.01 m."""
    params = vehicle_box_scene(n, seed=3)
    views = random_views(n_views, seed=303, size=size, res=res)
    return params, views


def config3_small(n=3000, n_views=4, size=64, res=0.1, seed=33):
    """Config-3-shaped tiny scene (same distributions, fewer points, coarser
    grid) for finite differences."""
    params = vehicle_box_scene(n, seed=seed, log_s_mean=math.log(0.2))
    views = random_views(n_views, seed=seed + 100, size=size, res=res)
    return params, views


def perturb(params, seed, mu_sd=0.1, log_s_sd=0.2):
    """Optimisation start: mean jitter, log-scale jitter, P resampled."""
    rng = np.random.default_rng(seed)
    out = params.copy()
    out[:, 0:3] += rng.normal(0.0, mu_sd, size=(params.shape[0], 3))
    out[:, 4:7] += rng.normal(0.0, log_s_sd, size=(params.shape[0], 3))
    out[:, 7] = rng.uniform(0.0, 1.0, size=params.shape[0])
    return out


def uneven_batch(n_scenes=256, views_per_scene=8, seed=4, n_lo=1000, n_hi=500000,
                 sizes=(256, 512, 1024)):
    """Uneven batch: scenes with log-uniform Gaussian counts, alternating
    vehicle-box and building scenes, image sizes drawn from `sizes`."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_scenes)).astype(np.int64)
    scenes, views = [], []
    for s in range(n_scenes):
        n = int(counts[s])
        size = int(rng.choice(sizes))
        if s % 2 == 0:
            scale = (n / 300000.0) ** (1.0 / 3.0)
            ext = (6.0 * scale, 3.0 * scale, 2.0 * scale)
            p = vehicle_box_scene(n, seed=seed * 1000 + s, extent=ext, center=(0.0, 0.0, ext[2] / 2))
            frame = 1.7 * max(ext)
            center = (0.0, 0.0, ext[2] / 2)
        else:
            r2 = np.random.default_rng(seed * 1000 + s)
            boxes = _place_boxes(r2, 3, 60.0, 5.0, 20.0)
            p = box_surface_scene(n, boxes, r2)
            frame = 76.8
            center = (30.0, 30.0, 5.0)
        scenes.append(p)
        vs = random_views(views_per_scene, seed=seed * 7919 + s, size=size, res=frame / size,
                          center=center, scene=s)
        views.extend(vs)
    return scenes, views
