"""Pins of the FP64 oracle against facts that do not come from the oracle.

Which pin covers which step of the method (Section II of the paper):
  geometry (eqs. W, R_r, x_r, P_C, P_I, Sigmaprime)
      - test_p1_*: sensor-geometry facts (a raised point moves to near range by
        h sin(theta) -- layover; ground points sit on the same row of both
        planes; points on one line of sight share a ray; azimuth shifts move
        columns by 1/dA), rotation equivariance of the azimuth angle, and the
        rendered splat centroid
      - test_p7_buildings: layover / roof / shadow extents of the paper's
        three 45-deg building cases (tests/golden/buildings_45deg.txt)
  intensity pass (eq. I_i)
      - test_p3: isolated Gaussian, closed form P o 2 pi sqrt(det Sigma'_C)
      - test_p4: Gaussians stacked on one line of sight, binomial closed form
      - test_p5: telescoping sum_i A_i + sum_rays T_final = #rays (P = 1)
      - test_p9: faint limit o -> 0, every Gaussian at its closed form
      - test_bl_*: Beer-Lambert opacity 1 - exp(-tau G): isolated and stacked
        Gaussians against the entire exponential integral Ein (scipy's E1),
        telescoping, and the adjoint against central differences
  imaging pass (eq. S_{n,m})
      - test_p2: splat integral equals the intensity (energy normalisation)
      - test_p6: layover additivity, permutation invariance
  depth order
      - test_depth_order_ties: index tie-break on equal float32 keys
  gradients (Section II-B)
      - test_grad_uI_closed_form: dL/du_I equals (I, 0) / (0, I) for linear ramps
      - test_sh_basis_matches_scipy: SH basis against SciPy (constants, signs, order)
      - test_p10: analytic adjoint vs FP64 central differences, all 12 raw
        parameters, two views
  cutoff / culling, loss, optimiser
      - test_cutoff_tail, test_culled_equals_brute, test_l1_vs_torch,
        test_adam_vs_torch
  second implementation
      - test_p8: NumPy twin agrees to 1e-10 on tiny scenes
"""
import math

import numpy as np
import pytest

import sdgr_scenes as sc


def one(mu, s=0.3, P=0.7, o=0.5, q=(1.0, 0.0, 0.0, 0.0), log_s=None):
    p = np.zeros((1, 12))
    p[0, 0:3] = mu
    p[0, 3] = math.log(o) - math.log1p(-o)
    p[0, 4:7] = np.log(s) if log_s is None else log_s
    p[0, 7] = P
    p[0, 8:12] = q
    return p


def stack(*ps):
    return np.concatenate(ps, axis=0)


# Orientation convention of eq. R_r: at azimuth angle phi the radar sits, seen
# from the scene, in the horizontal direction (cos phi, -sin phi, 0) and looks
# down at the grazing angle theta; the azimuth (column) axis is the horizontal
# direction (-sin phi, -cos phi, 0).
def toward_radar(phi):
    return np.array([math.cos(phi), -math.sin(phi), 0.0])


def azimuth_dir(phi):
    return np.array([-math.sin(phi), -math.cos(phi), 0.0])


def los_dir(phi, theta):
    # from the radar into the scene
    return -math.cos(theta) * toward_radar(phi) + np.array([0.0, 0.0, -math.sin(theta)])


VIEWS = [(0.0, 45.0), (30.0, 30.0), (-75.0, 60.0), (200.0, 17.0), (123.0, 73.0)]


@pytest.mark.parametrize("phi_deg,theta_deg", VIEWS)
def test_p1_sensor_geometry(orc, phi_deg, theta_deg):
    v = sc.make_view(phi_deg, theta_deg, 0.1, 0.15, 64, 48, center=(1.0, -2.0, 0.5))
    phi, th = v["phi"], v["theta"]
    c = np.array(v["center"])
    h, g, f, t = 0.8, 0.6, 0.9, 0.7
    pts = stack(one(c), one(c + [0, 0, h]), one(c + g * toward_radar(phi)),
                one(c + f * azimuth_dir(phi)), one(c + t * los_dir(phi, th)))
    pr = orc.project(pts, v)
    col0, row0 = v["NA"] / 2 - 0.5, v["NR"] / 2 - 0.5
    tol = 1e-9
    # the scene centre is the image centre on both planes
    assert abs(pr["uIx"][0] - col0) < tol and abs(pr["uIy"][0] - row0) < tol
    assert abs(pr["uCx"][0] - col0) < tol and abs(pr["uCy"][0] - row0) < tol
    # a point raised by h moves to nearer slant range by h sin(theta) (layover),
    # same azimuth
    assert abs(pr["uIy"][1] - (row0 - h * math.sin(th) / v["dR"])) < tol
    assert abs(pr["uIx"][1] - col0) < tol
    # a ground point moved toward the radar by g: nearer by g cos(theta); it
    # stays on the same row of the computation plane as of the imaging plane
    assert abs(pr["uIy"][2] - (row0 - g * math.cos(th) / v["dR"])) < tol
    assert abs(pr["uCy"][2] - pr["uIy"][2]) < tol
    # an azimuth shift moves the column by f / dA on both planes, rows fixed
    assert abs(pr["uIx"][3] - (col0 + f / v["dA"])) < tol
    assert abs(pr["uCx"][3] - (col0 + f / v["dA"])) < tol
    assert abs(pr["uIy"][3] - row0) < tol and abs(pr["uCy"][3] - row0) < tol
    # a shift along the line of sight: same ray of the computation plane,
    # farther by t in slant range
    assert abs(pr["uCx"][4] - col0) < tol and abs(pr["uCy"][4] - row0) < tol
    assert abs(pr["uIy"][4] - (row0 + t / v["dR"])) < tol
    # slant range itself: z_r is the distance from a radar at altitude 10 km
    # (plane-wave approximation; exact up to r^2 / (2 R0))
    R0 = 10000.0 / math.sin(th)
    radar = c - R0 * los_dir(phi, th)
    for k in range(5):
        mu = pts[k, 0:3]
        exact = np.linalg.norm(mu - radar)
        assert abs(pr["zr"][k] - exact) < 1e-3


def _rotz(beta):
    cb, sb = math.cos(beta), math.sin(beta)
    return np.array([[cb, -sb, 0.0], [sb, cb, 0.0], [0.0, 0.0, 1.0]])


def _qmul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def test_p1_rotation_equivariance(orc):
    """Turning the scene by beta about the vertical through the beam centre
    is the same as turning the radar azimuth by beta."""
    rng = np.random.default_rng(11)
    params = sc.vehicle_box_scene(40, seed=5, log_s_mean=math.log(0.25), center=(0.3, 0.2, 1.0))
    c = np.array([0.3, 0.2, 1.0])
    beta = 0.6
    Rz = _rotz(beta)
    qz = np.array([math.cos(beta / 2), 0.0, 0.0, math.sin(beta / 2)])
    rot = params.copy()
    rot[:, 0:3] = (params[:, 0:3] - c) @ Rz.T + c
    for i in range(params.shape[0]):
        rot[i, 8:12] = _qmul(qz, params[i, 8:12])
    phi = float(rng.uniform(0, 360))
    v1 = sc.make_view(phi, 40.0, 0.1, 0.1, 48, 48, center=c)
    v2 = sc.make_view(phi - math.degrees(beta), 40.0, 0.1, 0.1, 48, 48, center=c)
    cfg = orc.cfg(K=0.0)
    im1, A1, _ = orc.render(params, [v1], cfg)
    im2, A2, _ = orc.render(rot, [v2], cfg)
    assert np.abs(im1[0] - im2[0]).max() <= 1e-9 * np.abs(im1[0]).max()
    assert np.abs(A1 - A2).max() <= 1e-9 * np.abs(A1).max()


def test_p1_render_centroid(orc):
    v = sc.make_view(20.0, 35.0, 0.05, 0.05, 64, 64, center=(0, 0, 0))
    mu = np.array([0.31, -0.22, 0.4])
    p = one(mu, s=(0.12, 0.2, 0.15), q=(0.9, 0.1, -0.3, 0.2))
    cfg = orc.cfg(K=0.0)
    pr = orc.project(p, v, cfg)
    im, _, _ = orc.render(p, [v], cfg)
    S = im[0]
    rows, cols = np.mgrid[0:S.shape[0], 0:S.shape[1]]
    cx, cy = (S * cols).sum() / S.sum(), (S * rows).sum() / S.sum()
    assert abs(cx - pr["uIx"][0]) < 1e-6 and abs(cy - pr["uIy"][0]) < 1e-6


@pytest.mark.parametrize("K,tol", [(0.0, 1e-9), (5.0, 5e-6)])
def test_p2_splat_integral(orc, K, tol):
    """Energy normalisation: an isolated Gaussian deposits exactly its
    intensity I = P A in the image."""
    v = sc.make_view(10.0, 50.0, 0.05, 0.05, 96, 96)
    p = stack(one((0.1, 0.2, 0.0), s=(0.15, 0.25, 0.1), q=(0.8, 0.3, 0.1, -0.5), P=0.6, o=0.7),
              one((-1.2, 1.0, 0.4), s=0.2, P=0.9, o=0.4))
    # make sure the two do not overlap on either plane
    cfg = orc.cfg(K=K)
    pr = orc.project(p, v, cfg)
    assert min(pr["SIxx"].min(), pr["SIyy"].min()) > 1.5 ** 2
    im, A, _ = orc.render(p, [v], cfg)
    I = p[:, 7] * A[0]
    for k in range(2):
        single, Ak, _ = orc.render(p[k:k + 1], [v], cfg)
        assert abs(single[0].sum() - p[k, 7] * Ak[0, 0]) <= tol * p[k, 7] * Ak[0, 0]
    assert abs(im[0].sum() - I.sum()) <= tol * I.sum()


@pytest.mark.parametrize("theta_deg", [20.0, 45.0, 70.0])
def test_p3_isolated_intensity(orc, theta_deg):
    """Isotropic Gaussian of scale s: Sigma'_C = diag(s^2/dA^2, s^2/(dR tan
    theta)^2) + eps I, and the ray sum of o exp(-delta/2) is o 2 pi
    sqrt(det Sigma'_C)."""
    v = sc.make_view(33.0, theta_deg, 0.05, 0.06, 128, 256)
    s, o, P, eps = 0.2, 0.35, 0.8, 0.3
    p = one((0.05, -0.03, 0.02), s=s, o=o, P=P)
    cfg = orc.cfg(K=0.0, eps=eps)
    _, A, _ = orc.render(p, [v], cfg)
    cy = v["dR"] * math.tan(v["theta"])
    det = (s * s / v["dA"] ** 2 + eps) * (s * s / cy ** 2 + eps)
    expect = o * 2 * math.pi * math.sqrt(det)
    assert abs(A[0, 0] - expect) <= 1e-9 * expect
    assert abs(P * A[0, 0] - P * expect) <= 1e-9 * P * expect


@pytest.mark.parametrize("k", [2, 3, 4])
def test_p4_stacked_shadow(orc, k):
    """k identical Gaussians on one line of sight: the j-th (0 = nearest the
    radar) receives sum_rays o e (1 - o e)^j = 2 pi sqrt(det) sum_m C(j,m)
    (-1)^m o^(m+1) / (m+1).  For k = 2: I_back / I_front = 1 - o/2."""
    v = sc.make_view(70.0, 40.0, 0.05, 0.05, 96, 96)
    s, o, eps = 0.25, 0.6, 0.3
    los = los_dir(v["phi"], v["theta"])
    pts = stack(*[one(0.3 * j * los, s=s, o=o, P=1.0) for j in range(k)])
    # store in reverse so that storage order differs from depth order
    pts = pts[::-1].copy()
    cfg = orc.cfg(K=0.0, eps=eps)
    _, A, _ = orc.render(pts, [v], cfg)
    A = A[0][::-1]
    cy = v["dR"] * math.tan(v["theta"])
    det = (s * s / v["dA"] ** 2 + eps) * (s * s / cy ** 2 + eps)
    base = 2 * math.pi * math.sqrt(det)
    for j in range(k):
        expect = base * sum(math.comb(j, m) * (-1) ** m * o ** (m + 1) / (m + 1) for m in range(j + 1))
        assert abs(A[j] - expect) <= 1e-9 * base, (j, A[j], expect)
    assert abs(A[1] / A[0] - (1 - o / 2)) < 1e-9


def _ein(x):
    """Entire exponential integral Ein(x) = int_0^x (1 - e^-t) / t dt =
    gamma + ln x + E1(x) (x > 0)."""
    from scipy.special import exp1
    return np.euler_gamma + math.log(x) + float(exp1(x))


@pytest.mark.parametrize("o", [0.2, 0.6, 0.95])
def test_bl_isolated_intensity(orc, o):
    """Beer-Lambert opacity: the ray sum of 1 - exp(-tau exp(-delta/2)) over
    the plane is 2 pi sqrt(det Sigma'_C) int_0^inf (1 - exp(-tau e^-s)) ds =
    2 pi sqrt(det) Ein(tau), with tau = -log(1 - o) (peak opacity o)."""
    v = sc.make_view(33.0, 45.0, 0.05, 0.06, 128, 256)
    s, P, eps = 0.2, 0.8, 0.3
    p = one((0.05, -0.03, 0.02), s=s, o=o, P=P)
    _, A, _ = orc.render(p, [v], orc.cfg(K=0.0, eps=eps, alpha_mode=1))
    cy = v["dR"] * math.tan(v["theta"])
    det = (s * s / v["dA"] ** 2 + eps) * (s * s / cy ** 2 + eps)
    expect = 2 * math.pi * math.sqrt(det) * _ein(-math.log1p(-o))
    assert abs(A[0, 0] - expect) <= 1e-9 * expect
    # the default opacity o exp(-delta/2) gives a different profile with the same peak
    _, A0, _ = orc.render(p, [v], orc.cfg(K=0.0, eps=eps))
    assert abs(A0[0, 0] - o * 2 * math.pi * math.sqrt(det)) <= 1e-9 * A0[0, 0]
    assert A[0, 0] > A0[0, 0]  # 1 - (1 - o)^G > o G for 0 < G < 1


@pytest.mark.parametrize("k", [2, 3])
def test_bl_stacked_shadow(orc, k):
    """Identical Gaussians on one line of sight, Beer-Lambert opacity: the
    j-th receives sum_rays (1 - e^{-tau G}) e^{-j tau G} = 2 pi sqrt(det)
    (Ein((j + 1) tau) - Ein(j tau))."""
    v = sc.make_view(70.0, 40.0, 0.05, 0.05, 96, 96)
    s, o, eps = 0.25, 0.6, 0.3
    tau = -math.log1p(-o)
    los = los_dir(v["phi"], v["theta"])
    pts = stack(*[one(0.3 * j * los, s=s, o=o, P=1.0) for j in range(k)])[::-1].copy()
    _, A, _ = orc.render(pts, [v], orc.cfg(K=0.0, eps=eps, alpha_mode=1))
    A = A[0][::-1]
    cy = v["dR"] * math.tan(v["theta"])
    base = 2 * math.pi * math.sqrt((s * s / v["dA"] ** 2 + eps) * (s * s / cy ** 2 + eps))
    for j in range(k):
        expect = base * (_ein((j + 1) * tau) - (_ein(j * tau) if j else 0.0))
        assert abs(A[j] - expect) <= 1e-9 * base, (j, A[j], expect)


def test_bl_telescoping(orc):
    params, views = sc.config1()
    params = params[:300].copy()
    params[:, 7] = 1.0
    views = [dict(views[0], NA=64, NR=48, dA=0.2, dR=0.25)]
    _, A, Tf = orc.render(params, views, orc.cfg(alpha_mode=1))
    nrays = views[0]["NA"] * views[0]["NR"]
    assert abs(A.sum() + Tf[0].sum() - nrays) <= 1e-12 * nrays


def test_bl_gradients_fd(orc):
    params = sc.vehicle_box_scene(6, seed=23, extent=(1.0, 0.8, 0.6), log_s_mean=math.log(0.15), center=(0, 0, 0))
    views = [sc.make_view(25.0, 40.0, 0.06, 0.07, 24, 20), sc.make_view(160.0, 55.0, 0.07, 0.06, 20, 24)]
    # step 1e-5: at 1e-6 the differences of this scene carry ~1.5e-6 of roundoff in both opacity modes
    _fd_check(orc, params, views, orc.cfg(K=0.0, alpha_mode=1), h_rel=1e-5)


def test_grad_uI_closed_form(orc):
    """dL/du_I, the image-plane position gradient behind the densification
    statistic: with the upstream image equal to the column index x, L = I sum_pix
    x beta(x - u) = I u_x sum beta = I u_x (energy normalisation, sigma >= 1.5
    px), so dL/du_I = (I, 0); with the row index y, (0, I)."""
    v = sc.make_view(33.0, 45.0, 0.05, 0.06, 96, 112)
    p = one((0.05, -0.03, 0.02), s=0.2, o=0.4, P=0.7)
    c = orc.cfg(K=0.0)
    _, A, _ = orc.render(p, [v], c)
    I = 0.7 * A[0, 0]
    X, Y = np.meshgrid(np.arange(v["NA"], dtype=float), np.arange(v["NR"], dtype=float))
    _, _, dx = orc.grad_uI(p, [v], [X], c)
    _, _, dy = orc.grad_uI(p, [v], [Y], c)
    assert np.allclose(dx[0, 0], [I, 0.0], rtol=1e-9, atol=1e-9 * I)
    assert np.allclose(dy[0, 0], [0.0, I], rtol=1e-9, atol=1e-9 * I)


def test_p5_telescoping(orc):
    params, views = sc.config1()
    params = params[:300].copy()
    params[:, 7] = 1.0
    views = [dict(views[0], NA=64, NR=48, dA=0.2, dR=0.25)]
    _, A, Tf = orc.render(params, views)
    nrays = views[0]["NA"] * views[0]["NR"]
    total = A.sum() + Tf[0].sum()
    assert abs(total - nrays) <= 1e-12 * nrays


def test_p6_layover_and_permutation(orc):
    v = sc.make_view(15.0, 35.0, 0.05, 0.05, 64, 96)
    el = np.array([-math.sin(v["theta"]) * math.cos(v["phi"]), math.sin(v["theta"]) * math.sin(v["phi"]),
                   math.cos(v["theta"])])
    # el spans the layover direction: it changes neither azimuth nor range.
    # Two identical Gaussians separated along it do not shade each other and
    # land on the same pixels: the image is exactly twice the single one.
    cfg = orc.cfg(K=0.0)
    single, _, _ = orc.render(one(-0.7 * el, s=0.08), [v], cfg)
    pair, _, _ = orc.render(stack(one(-0.7 * el, s=0.08), one(0.7 * el, s=0.08)), [v], cfg)
    assert np.abs(pair[0] - 2 * single[0]).max() <= 1e-12 * single[0].max()
    # permuting storage order leaves the image unchanged
    params, _ = sc.config1()
    params = params[:200]
    views = [sc.make_view(0.0, 45.0, 0.2, 0.2, 48, 48)]
    perm = np.random.default_rng(0).permutation(200)
    im1, A1, _ = orc.render(params, views)
    im2, A2, _ = orc.render(params[perm], views)
    assert np.abs(im1[0] - im2[0]).max() <= 1e-12 * im1[0].max()
    assert np.array_equal(A1[0][perm], A2[0])


def _building(h, w, seed=0):
    rng = np.random.default_rng(seed)
    box = (-w / 2, -5.0, 0.0, w, 10.0, h)
    n_b = int(40 * (w * 10 + 2 * 10 * h + 2 * w * h))
    b = sc.box_surface_scene(n_b, [box], rng, s_lo=0.12, s_hi=0.18)
    # ground: two strips in front of / behind the footprint plus the sides
    ground = []
    for (x0, x1, y0, y1) in [(w / 2, 22.0, -8.0, 8.0), (-22.0, -w / 2, -8.0, 8.0),
                             (-w / 2, w / 2, -8.0, -5.0), (-w / 2, w / 2, 5.0, 8.0)]:
        n = int(12 * (x1 - x0) * (y1 - y0))
        g = sc.box_surface_scene(n, [], rng, s_lo=0.15, s_hi=0.25, ground=(x0, y0, x1, y1))
        ground.append(g)
    params = np.concatenate([b] + ground, axis=0)
    params[:, 3] = math.log(0.95) - math.log(0.05)  # nearly opaque
    params[:, 7] = 1.0
    return params


def _runs(mask):
    runs, start = [], None
    for k, m in enumerate(mask):
        if m and start is None:
            start = k
        if not m and start is not None:
            runs.append((start, k))
            start = None
    if start is not None:
        runs.append((start, len(mask)))
    return runs


def _golden_buildings():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "buildings_45deg.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append((f[0],) + tuple(float(x) for x in f[1:]))
    return rows


@pytest.mark.parametrize("case", _golden_buildings(), ids=lambda c: c[0])
def test_p7_buildings(orc, case):
    name, h, w, theta, lay_m, roof_m, dark_m = case
    res = 0.2
    v = sc.make_view(0.0, theta, res, res, 64, 200, center=(0.0, 0.0, 0.0))
    params = _building(h, w)
    im, _, _ = orc.render(params, [v], orc.cfg(), culled=True)
    S = im[0]
    prof = S[:, 30:34].mean(axis=1)
    th = math.radians(theta)
    row0 = v["NR"] / 2 - 0.5
    rho_foot = -math.cos(th) * (w / 2)         # slant range of the front foot
    r_foot = rho_foot / res + row0
    ground_level = np.median(prof[int(r_foot - h * math.sin(th) / res) - 25:int(r_foot - h * math.sin(th) / res) - 5])
    bright = _runs(prof > 1.5 * ground_level)
    dark = _runs(prof < 0.15 * ground_level)
    # the layover band ends at the front foot, the dark band is the longest run
    lay = max(bright, key=lambda r: r[1] - r[0])
    drk = max(dark, key=lambda r: r[1] - r[0])
    tol_px = 2.5
    assert abs((lay[1] - lay[0]) - lay_m / res) <= tol_px, (lay, lay_m / res)
    assert abs((drk[1] - drk[0]) - dark_m / res) <= tol_px, (drk, dark_m / res)
    assert abs((drk[0] - lay[1]) - roof_m / res) <= tol_px, (lay, drk, roof_m / res)
    if name == "B":
        # the paper: the shadow is twice as long as the scattering band
        assert abs((drk[1] - drk[0]) / (lay[1] - lay[0]) - 2.0) < 0.15


def test_p8_numpy_twin(orc):
    from oracle import numpy_twin
    rng = np.random.default_rng(8)
    for trial in range(4):
        n = int(rng.integers(1, 9))
        params = sc.vehicle_box_scene(n, seed=100 + trial, extent=(1.5, 1.0, 0.8),
                                      log_s_mean=math.log(0.12), center=(0, 0, 0))
        NA, NR = int(rng.integers(8, 33)), int(rng.integers(8, 33))
        v = sc.make_view(float(rng.uniform(0, 360)), float(rng.uniform(20, 70)), 0.08, 0.09, NA, NR)
        for K in (5.0, 0.0):
            img_c, A_c, _ = orc.render(params, [v], orc.cfg(K=K))
            img_n, A_n = numpy_twin.render(params, v, K=K)
            scale = max(np.abs(img_n).max(), 1e-300)
            assert np.abs(img_c[0] - img_n).max() <= 1e-10 * scale
            assert np.abs(A_c[0] - A_n).max() <= 1e-10 * max(np.abs(A_n).max(), 1e-300)


def test_p9_faint_limit(orc):
    """o -> 0: no shading, every isotropic Gaussian gets o 2 pi sqrt(det
    Sigma'_C) and the image is the plain sum of normalised 2D Gaussians of
    mass P_i A_i."""
    rng = np.random.default_rng(9)
    v = sc.make_view(0.0, 45.0, 0.1, 0.1, 96, 96)
    n = 30
    mu = rng.uniform(-1.5, 1.5, size=(n, 3))
    s = rng.uniform(0.2, 0.3, size=n)
    o = 1e-7
    p = stack(*[one(mu[i], s=s[i], o=o, P=float(rng.uniform(0.2, 1.0))) for i in range(n)])
    cfg = orc.cfg(K=0.0)
    im, A, _ = orc.render(p, [v], cfg)
    cy = v["dR"] * math.tan(v["theta"])
    pr = orc.project(p, v, cfg)
    expect = np.empty(n)
    for i in range(n):
        det = (s[i] ** 2 / v["dA"] ** 2 + 0.3) * (s[i] ** 2 / cy ** 2 + 0.3)
        expect[i] = o * 2 * math.pi * math.sqrt(det)
    inside = (pr["uCx"] > 12) & (pr["uCx"] < 84) & (pr["uCy"] > 12) & (pr["uCy"] < 84)
    assert inside.sum() > 10
    assert np.all(np.abs(A[0][inside] - expect[inside]) <= 1e-5 * expect[inside])
    # image: plain sum of normalised Gaussians, isotropic in metric units
    rows, cols = np.mgrid[0:96, 0:96].astype(np.float64)
    ref = np.zeros((96, 96))
    for i in range(n):
        sx2 = s[i] ** 2 / v["dA"] ** 2 + 0.3
        sy2 = s[i] ** 2 / v["dR"] ** 2 + 0.3
        g = np.exp(-0.5 * ((cols - pr["uIx"][i]) ** 2 / sx2 + (rows - pr["uIy"][i]) ** 2 / sy2))
        ref += p[i, 7] * A[0][i] * g / (2 * math.pi * math.sqrt(sx2 * sy2))
    assert np.abs(im[0] - ref).max() <= 1e-12 * ref.max()


def test_depth_order_ties(orc):
    """Equal float32 slant-range keys are ordered by index; the order is
    front (near range) to back."""
    v = sc.make_view(0.0, 45.0, 0.1, 0.1, 32, 32)
    los = los_dir(v["phi"], v["theta"])
    az = azimuth_dir(v["phi"])
    # 0 and 2 at the same range (shifted in azimuth), 1 nearer, 3 farther
    p = stack(one(0.2 * az), one(-0.3 * los), one(-0.2 * az), one(0.5 * los))
    assert list(orc.depth_order(p, v)) == [1, 0, 2, 3]
    # a shift far below float32 resolution of the key does not reorder
    q = p.copy()
    q[2, 0:3] += 1e-12 * los
    assert list(orc.depth_order(q, v)) == [1, 0, 2, 3]


def _fd_check(orc, params, views, cfg, rel=1e-6, h_rel=1e-6):
    rng = np.random.default_rng(1)
    G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
    g_an, _ = orc.grad(params, views, G, cfg)
    idx = [(i, j) for i in range(params.shape[0]) for j in range(12)]
    fd, bad = orc.linear_loss_grad_fd(params, views, G, cfg, idx=idx, h_rel=h_rel)
    groups = {"mean": [0, 1, 2], "opacity": [3], "scale": [4, 5, 6], "P": [7], "quat": [8, 9, 10, 11]}
    an = np.array([g_an[i, j] for (i, j) in idx])
    comp = np.array([j for (_, j) in idx])
    ok = ~np.array(bad)
    for name, cols in groups.items():
        sel = np.isin(comp, cols) & ok
        scale = np.abs(an[np.isin(comp, cols)]).max()
        assert scale > 0
        err = np.abs(an[sel] - fd[sel]).max()
        assert err <= rel * scale, (name, err, scale)


def test_p10_gradients_fd(orc):
    params = sc.vehicle_box_scene(6, seed=21, extent=(1.0, 0.8, 0.6), log_s_mean=math.log(0.15), center=(0, 0, 0))
    views = [sc.make_view(25.0, 40.0, 0.06, 0.07, 24, 20), sc.make_view(160.0, 55.0, 0.07, 0.06, 20, 24)]
    _fd_check(orc, params, views, orc.cfg(K=0.0))


def test_p10_gradients_fd_peak_mode(orc):
    params = sc.vehicle_box_scene(5, seed=22, extent=(1.0, 0.8, 0.6), log_s_mean=math.log(0.15), center=(0, 0, 0))
    views = [sc.make_view(300.0, 35.0, 0.06, 0.06, 22, 22)]
    _fd_check(orc, params, views, orc.cfg(K=0.0, norm_mode=1))


def test_cutoff_tail(orc):
    params, views = sc.config1()
    params = params[:400]
    views = [dict(views[0], NA=48, NR=48, dA=0.25, dR=0.25)]
    a, _, _ = orc.render(params, views, orc.cfg(K=5.0))
    b, _, _ = orc.render(params, views, orc.cfg(K=0.0))
    assert np.abs(a[0] - b[0]).max() <= 1e-5 * b[0].max()


def test_culled_equals_brute(orc):
    params, views = sc.config1()
    params = params[:500]
    views = [dict(views[0], NA=64, NR=56, dA=0.2, dR=0.2)]
    a, Aa, Ta = orc.render(params, views, culled=False)
    b, Ab, Tb = orc.render(params, views, culled=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(Aa, Ab) and np.array_equal(Ta[0], Tb[0])
    G = [np.random.default_rng(3).normal(size=a[0].shape)]
    ga, _ = orc.grad(params, views, G, culled=False)
    gb, _ = orc.grad(params, views, G, culled=True)
    assert np.array_equal(ga, gb)


def test_l1_vs_torch(orc):
    import torch
    rng = np.random.default_rng(4)
    S = [rng.normal(size=(5, 7)), rng.normal(size=(3, 4))]
    T = [rng.normal(size=(5, 7)), S[1].copy()]
    loss, g = orc.l1(S, T)
    ts = [torch.tensor(x, requires_grad=True) for x in S]
    flat = torch.cat([x.reshape(-1) for x in ts])
    tgt = torch.cat([torch.tensor(x).reshape(-1) for x in T])
    ref = torch.nn.functional.l1_loss(flat, tgt)
    ref.backward()
    assert abs(loss - ref.item()) < 1e-14
    for a, b in zip(g, ts):
        assert np.allclose(a, b.grad.numpy(), rtol=0, atol=1e-15)


def test_adam_vs_torch(orc):
    import torch
    rng = np.random.default_rng(5)
    N = 17
    p = rng.normal(size=(N, 12))
    m = np.zeros((N, 12))
    v = np.zeros((N, 12))
    lr = np.array([1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3])
    groups = {0: [0, 1, 2], 1: [4, 5, 6], 2: [8, 9, 10, 11], 3: [3], 4: [7]}
    tp = [torch.tensor(p[:, cols].copy(), requires_grad=True) for cols in groups.values()]
    opt = torch.optim.Adam([{"params": [t], "lr": float(lr[k])} for k, t in zip(groups.keys(), tp)],
                           betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        g = rng.normal(size=(N, 12))
        orc.adam(p, g, m, v, lr, 0.9, 0.999, 1e-15, step)
        for k, t in zip(groups.keys(), tp):
            t.grad = torch.tensor(g[:, groups[k]].copy())
        opt.step()
    for k, t in zip(groups.keys(), tp):
        assert np.allclose(p[:, groups[k]], t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_step_matches_render_l1_grad(orc):
    """The one-call training step equals render + L1 + adjoint."""
    params, views = sc.config3_small(n=400, n_views=2, size=40, res=0.1)
    rng = np.random.default_rng(12)
    targets = [rng.uniform(0, 0.05, size=(v["NR"], v["NA"])) for v in views]
    loss, imgs, g = orc.step(params, views, targets)
    ref_imgs, _, _ = orc.render(params, views, culled=True)
    ref_loss, dLdS = orc.l1(ref_imgs, targets)
    ref_g, _ = orc.grad(params, views, dLdS, culled=True)
    assert abs(loss - ref_loss) <= 1e-15 * max(1.0, ref_loss)
    for a, b in zip(imgs, ref_imgs):
        assert np.array_equal(a, b)
    assert np.array_equal(g, ref_g)


# ---------------------------------------------------------------------------
# view-dependent scattering (spherical harmonics of the direction to the radar)
# ---------------------------------------------------------------------------
def test_sh_basis_orthonormal(orc):
    """Gauss-Legendre x uniform-azimuth quadrature (exact for these
    polynomials) of Y_a Y_b over the sphere is the identity."""
    nz, nphi = 12, 24
    z, wz = np.polynomial.legendre.leggauss(nz)
    G = np.zeros((15, 15))
    for zi, wi in zip(z, wz):
        r = math.sqrt(1 - zi * zi)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = orc.sh_basis([r * math.cos(ph), r * math.sin(ph), zi])
            G += wi * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(15)).max() < 1e-12


def test_sh_basis_matches_scipy(orc):
    """The 15 basis values against SciPy's complex spherical harmonics turned
    real (m > 0: sqrt2 (-1)^m Re Y_l^m, m < 0: sqrt2 (-1)^m Im Y_l^|m|, m = 0:
    Y_l^0 -- the (-1)^m removes the Condon-Shortley phase), in the order
    l = 1..3, m = -l..l.  Pins every constant, sign and the ordering, which
    orthonormality alone leaves free."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(7)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        ref = []
        for l in (1, 2, 3):
            for m in range(-l, l + 1):
                c = sph_harm_y(l, abs(m), theta, phi)
                ref.append(math.sqrt(2) * (-1) ** m * (c.real if m > 0 else c.imag) if m else c.real)
        assert np.abs(np.asarray(orc.sh_basis(d)) - np.array(ref)).max() < 1e-13


def test_sh_degree_zero_and_direction(orc):
    params = sc.vehicle_box_scene(30, seed=41, extent=(1.0, 1.0, 1.0), log_s_mean=math.log(0.12), center=(0, 0, 0))
    v = sc.make_view(35.0, 40.0, 0.05, 0.05, 40, 40)
    sh = np.random.default_rng(1).normal(size=(30, 16))
    base, A0, _ = orc.render(params, [v], orc.cfg())
    same, A1, _ = orc.render(params, [v], orc.cfg(sh=sh, sh_degree=0))
    assert np.array_equal(base[0], same[0])
    # a pure l=1, m=0 coefficient (c1 z) changes P by c1 * sin(theta): the
    # direction toward the radar has vertical component sin(theta)
    sh1 = np.zeros((30, 16))
    sh1[:, 1] = 1.0
    d = np.array([math.cos(v["theta"]) * math.cos(v["phi"]), -math.cos(v["theta"]) * math.sin(v["phi"]),
                  math.sin(v["theta"])])
    p2 = params.copy()
    p2[:, 7] += math.sqrt(3 / (4 * math.pi)) * d[2]
    a, _, _ = orc.render(params, [v], orc.cfg(sh=sh1, sh_degree=1))
    b, _, _ = orc.render(p2, [v], orc.cfg())
    assert np.abs(a[0] - b[0]).max() <= 1e-13 * np.abs(b[0]).max()


def test_sh_gradients_fd(orc):
    params = sc.vehicle_box_scene(5, seed=43, extent=(1.0, 0.8, 0.6), log_s_mean=math.log(0.15), center=(0, 0, 0))
    views = [sc.make_view(25.0, 40.0, 0.06, 0.07, 24, 20), sc.make_view(160.0, 55.0, 0.07, 0.06, 20, 24)]
    sh = np.random.default_rng(2).normal(scale=0.2, size=(5, 16))
    G = [np.random.default_rng(3).normal(size=(v["NR"], v["NA"])) for v in views]
    c = orc.cfg(K=0.0, sh=sh, sh_degree=3)
    _, dsh = orc.grad_sh(params, views, G, c)
    def L(shv):
        imgs, _, _ = orc.render(params, views, orc.cfg(K=0.0, sh=shv, sh_degree=3))
        return sum(float((g * im).sum()) for g, im in zip(G, imgs))
    scale = np.abs(dsh).max()
    assert scale > 0
    for i in range(5):
        for k in (0, 1, 4, 7, 11, 14):
            h = 1e-6
            a, b = sh.copy(), sh.copy()
            a[i, k] += h
            b[i, k] -= h
            fd = (L(a) - L(b)) / (2 * h)
            assert abs(fd - dsh[i, k]) <= 1e-6 * scale
    assert np.all(dsh[:, 15] == 0)


# ---------------------------------------------------------------------------
# densification and pruning rules
# ---------------------------------------------------------------------------
def test_densify_rules():
    from oracle.densify import densify
    f = np.float32
    P = np.zeros((7, 12), f)
    P[:, 8] = 1.0                       # identity rotations
    P[:, 3] = 2.0                       # opacity ~0.88
    P[:, 7] = 0.5
    P[:, 4:7] = math.log(0.01)
    P[:, 0] = np.arange(7)              # distinct means
    P[0, 3] = math.log(0.001 / 0.999)   # opacity 0.001 < 0.005: pruned
    P[1, 7] = 1e-5                      # P below 1e-3: pruned
    P[2, 4] = math.log(2.0)             # larger than max_scale 1.0: pruned
    P[4, 4] = math.log(0.02)            # small, above threshold: cloned
    P[5, 4:7] = [math.log(0.2), math.log(0.05), math.log(0.05)]   # large: split along x
    grads = np.zeros((7, 12), f)
    grads[4, 0:3] = [1.0, 0.0, 0.0]
    grads[5, 0:3] = [-1.0, 0.0, 0.0]    # -dL/dmu points along +x
    accum = np.array([1, 1, 1, 0.001, 1, 1, 5.0], f)
    count = np.array([1, 1, 1, 1, 1, 1, 0], f)   # G6: no views, never densified
    m = np.full((7, 12), 0.25, f)
    v = np.full((7, 12), 0.5, f)
    out, om, ov, _, act = densify(P, grads, accum, count, m, v)
    assert act == ["prune", "prune", "prune", "keep", "clone", "split", "keep"]
    assert out.shape == (6, 12)
    # kept Gaussians keep their moments, new ones start from zero
    assert np.all(om[0] == 0.25) and np.all(ov[0] == 0.5)
    # clone: original, then the copy one largest scale along -dL/dmu
    assert np.allclose(out[1], P[4]) and np.allclose(out[2, 0:3], P[4, 0:3] + [-0.02, 0, 0])
    assert np.all(om[2] == 0) and np.all(ov[2] == 0)
    # split: children at +-0.1 along the largest axis, child 0 on the -dL/dmu side, scales / 1.6
    assert np.allclose(out[3, 0:3], P[5, 0:3] + [0.1, 0, 0]) and np.allclose(out[4, 0:3], P[5, 0:3] - [0.1, 0, 0])
    assert np.allclose(np.exp(out[3, 4:7]), np.exp(P[5, 4:7]) / 1.6, rtol=1e-6)
    assert np.allclose(out[5], P[6])
