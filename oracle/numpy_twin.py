"""NumPy FP64 forward of the SAR differentiable Gaussian rasterizer for tiny
scenes (a handful of Gaussians, images up to ~32x32).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written separately
from `sdgr_oracle.c` and organised differently: vectorised over pixels,
geometry built from the line-of-sight / azimuth / elevation unit vectors of
Section II-A-1 (eq. R_r) and the 2D covariance taken as the marginal of the
3D one on each plane (eq. Sigmaprime, orthographic reading), compositing of
Section II-A-2 (eq. I_i) and the layover sum of Section II-A-3 (eq. S_{n,m}),
with the same readings (energy-normalised beta with the 1/2 and the inverse,
dilation eps, cutoff K, pixel centres at integers, depth order on the
float32-rounded slant-range offset with index tie-break).
"""
from __future__ import annotations

import numpy as np


def _axes(phi, theta):
    # unit vectors of the radar frame in world coordinates: flight (azimuth)
    # direction, in-plane normal ("elevation"), line of sight (pointing away
    # from the radar, downwards at the grazing angle)
    az = np.array([-np.sin(phi), -np.cos(phi), 0.0])
    el = np.array([-np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    los = np.array([-np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    return az, el, los


def _cov3(p):
    w, x, y, z = p[8:12] / np.linalg.norm(p[8:12])
    R = np.array([
        [w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z],
    ])
    s2 = np.exp(2.0 * p[4:7])
    return (R * s2) @ R.T


def render(params, view, K=5.0, eps=0.3, norm_mode=0):
    """Returns (image [NR,NA], A [N])."""
    params = np.asarray(params, dtype=np.float64)
    N = params.shape[0]
    NA, NR = view["NA"], view["NR"]
    az, el, los = _axes(view["phi"], view["theta"])
    c = np.asarray(view["center"], dtype=np.float64)
    cell_y = view["dR"] * np.tan(view["theta"])
    cols, rows = np.meshgrid(np.arange(NA, dtype=np.float64), np.arange(NR, dtype=np.float64))
    K2 = K * K if K > 0 else np.inf

    geo = []
    for i in range(N):
        p = params[i]
        d = p[0:3] - c
        a, y, rho = az @ d, el @ d, los @ d
        S3 = _cov3(p)
        # computation plane: axes (az, el) scaled to cells
        Bc = np.stack([az / view["dA"], el / cell_y])
        Sc = Bc @ S3 @ Bc.T + eps * np.eye(2)
        # imaging plane: axes (az, los) scaled to pixels
        Bi = np.stack([az / view["dA"], los / view["dR"]])
        Si = Bi @ S3 @ Bi.T + eps * np.eye(2)
        uc = np.array([a / view["dA"] + NA / 2 - 0.5, y / cell_y + NR / 2 - 0.5])
        ui = np.array([a / view["dA"] + NA / 2 - 0.5, rho / view["dR"] + NR / 2 - 0.5])
        o = 1.0 / (1.0 + np.exp(-p[3]))
        geo.append((uc, np.linalg.inv(Sc), ui, np.linalg.inv(Si), np.linalg.det(Si), o, p[7],
                    float(np.float32(rho))))

    def weight(u, Cinv):
        dx, dy = cols - u[0], rows - u[1]
        delta = Cinv[0, 0] * dx * dx + 2.0 * Cinv[0, 1] * dx * dy + Cinv[1, 1] * dy * dy
        return np.where(delta <= K2, np.exp(-0.5 * delta), 0.0)

    order = sorted(range(N), key=lambda i: (geo[i][7], i))
    T = np.ones((NR, NA))
    A = np.zeros(N)
    for i in order:
        uc, Cc, _, _, _, o, _, _ = geo[i]
        alpha = o * weight(uc, Cc)
        A[i] = float((alpha * T).sum())
        T = T * (1.0 - alpha)

    img = np.zeros((NR, NA))
    for i in range(N):
        _, _, ui, Ci, detI, _, P, _ = geo[i]
        cn = 1.0 / (2.0 * np.pi * np.sqrt(detI)) if norm_mode == 0 else 1.0
        img += cn * weight(ui, Ci) * (P * A[i])
    return img, A
