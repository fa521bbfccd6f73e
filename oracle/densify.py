"""Densification and pruning, written plainly from the rules (TEST
INFRASTRUCTURE ONLY; see the package docstring).

The paper (Section II-B, "Densification and Pruning Operation"; thresholds
in Section III-D) duplicates Gaussians whose positional gradient exceeds a
threshold and moves the copies along the gradient direction, splits
oversized ones and moves the parts the same way, and removes Gaussians that
are too large or scatter too little.  Readings: statistic = mean over views
of |dL/du_I| (image-plane pixel units), over the views in which the
Gaussian received weight; clone = a copy moved by its largest scale along
-dL/dmu; split = two children half that scale from the centre along the
axis of the largest scale, child 0 on the -dL/dmu side, log-scales reduced
by ln(split_factor); prune on opacity, P or largest scale.  Every decision
is taken in float32 (the precision of the GPU kernel), with the thresholds
converted once from float64.
"""
from __future__ import annotations

import math

import numpy as np


def thresholds(grad_threshold=0.003, dense_scale=0.05, max_scale=1.0, min_opacity=0.005, min_P=1e-3,
               split_factor=1.6):
    f = np.float32
    return {
        "grad": f(grad_threshold),
        "log_dense": f(math.log(dense_scale)),
        "log_max": f(math.log(max_scale)),
        "logit_min_o": f(math.log(min_opacity) - math.log1p(-min_opacity)),
        "min_P": f(min_P),
        "log_split": f(math.log(split_factor)),
    }


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify(params, grads, accum, count, m, v, sh=None, **cfg):
    """params, grads, m, v: float32 [N,12]; accum, count: float32 [N];
    sh: float32 [N,16] or None.  Returns float64 arrays (params, m, v, sh)
    of the survivors, in order, and the per-Gaussian action list."""
    th = thresholds(**cfg)
    out_p, out_m, out_v, out_sh, actions = [], [], [], [], []
    zero = np.zeros(12)
    for i in range(params.shape[0]):
        p = params[i].astype(np.float64)
        lsmax = np.float32(max(params[i, 4], params[i, 5], params[i, 6]))
        if np.float32(params[i, 3]) < th["logit_min_o"] or np.float32(params[i, 7]) < th["min_P"] \
                or lsmax > th["log_max"]:
            actions.append("prune")
            continue
        act = "keep"
        c = np.float32(count[i])
        if c > 0 and np.float32(np.float32(accum[i]) / c) > th["grad"]:
            act = "clone" if lsmax <= th["log_dense"] else "split"
        actions.append(act)
        row_sh = None if sh is None else sh[i].astype(np.float64)
        g = grads[i, 0:3].astype(np.float64)
        gn = np.linalg.norm(g)
        u = -g / gn if gn > 0 else np.zeros(3)
        ax = int(np.argmax(params[i, 4:7]))
        smax = math.exp(p[4 + ax])
        if act in ("keep", "clone"):
            out_p.append(p)
            out_m.append(m[i].astype(np.float64))
            out_v.append(v[i].astype(np.float64))
            out_sh.append(row_sh)
        if act == "clone":
            q = p.copy()
            q[0:3] += smax * u
            out_p.append(q)
            out_m.append(zero)
            out_v.append(zero)
            out_sh.append(row_sh)
        elif act == "split":
            e = _rot(p[8:12])[:, ax]
            sgn = -1.0 if float(e @ u) < 0 else 1.0
            for child in (0, 1):
                q = p.copy()
                q[0:3] += (0.5 if child == 0 else -0.5) * sgn * smax * e
                q[4:7] -= float(th["log_split"])
                out_p.append(q)
                out_m.append(zero)
                out_v.append(zero)
                out_sh.append(row_sh)
    n = len(out_p)
    P = np.array(out_p).reshape(n, 12)
    M = np.array(out_m).reshape(n, 12)
    V = np.array(out_v).reshape(n, 12)
    S = None if sh is None else np.array(out_sh).reshape(n, 16)
    return P, M, V, S, actions
