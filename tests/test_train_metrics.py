"""Host-side parts of the reconstruction demo: the image metrics against
their definitions (PSNR closed forms; SSIM against a direct evaluation of
the Gaussian-window formula on a small image) and the hemispherical
initialisation."""
import math

import numpy as np


def test_psnr_closed_forms():
    from paper_2506_21633_b300.train import psnr
    ref = np.zeros((8, 8))
    ref[3, 4] = 2.0
    img = ref + 0.1  # MSE = 0.01, MAX = 2
    assert abs(psnr(img, ref) - 10 * math.log10(4.0 / 0.01)) < 1e-12
    assert psnr(ref, ref) == math.inf


def _ssim_direct(x, y, sigma=1.5, radius=5, k1=0.01, k2=0.03):
    """The SSIM formula evaluated pixel by pixel: Gaussian weights over a
    (2 radius + 1)^2 window, image edges mirrored (half-sample symmetric)."""
    D = y.max() - y.min()
    c1, c2 = (k1 * D) ** 2, (k2 * D) ** 2
    t = np.arange(-radius, radius + 1)
    w1 = np.exp(-0.5 * (t / sigma) ** 2)
    w1 /= w1.sum()
    W = np.outer(w1, w1)
    H, Wd = x.shape

    def refl(i, n):
        while i < 0 or i >= n:
            i = -i - 1 if i < 0 else 2 * n - i - 1
        return i
    total = 0.0
    for r in range(H):
        for c in range(Wd):
            xs = np.array([[x[refl(r + a, H), refl(c + b, Wd)] for b in t] for a in t])
            ys = np.array([[y[refl(r + a, H), refl(c + b, Wd)] for b in t] for a in t])
            mx, my = (W * xs).sum(), (W * ys).sum()
            vx = (W * xs * xs).sum() - mx * mx
            vy = (W * ys * ys).sum() - my * my
            cxy = (W * xs * ys).sum() - mx * my
            total += ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    return total / (H * Wd)


def test_ssim_against_direct_formula():
    from paper_2506_21633_b300.train import ssim
    rng = np.random.default_rng(0)
    y = rng.uniform(0, 1, size=(12, 13))
    x = y + rng.normal(0, 0.1, size=y.shape)
    assert abs(ssim(x, y) - _ssim_direct(x, y)) < 1e-12
    assert abs(ssim(y, y) - 1.0) < 1e-12
    assert ssim(x, y) < ssim(y + rng.normal(0, 0.01, size=y.shape), y) < 1.0


def test_hemisphere_init():
    from paper_2506_21633_b300.train import hemisphere_init
    p = hemisphere_init(5000, 4.0, (1.0, -2.0, 0.5), seed=3, scale=0.05, opacity=0.2, P=0.3)
    d = p[:, 0:3] - np.array([1.0, -2.0, 0.5])
    assert np.allclose(np.linalg.norm(d, axis=1), 4.0, rtol=1e-5)
    assert (d[:, 2] >= 0).all()
    assert abs(d[:, 0].mean()) < 0.15 and abs(d[:, 1].mean()) < 0.15  # uniform in azimuth
    assert np.allclose(1 / (1 + np.exp(-p[:, 3])), 0.2, rtol=1e-5)
    assert np.allclose(np.exp(p[:, 4:7]), 0.05, rtol=1e-5) and np.allclose(p[:, 7], 0.3)
    assert np.allclose(p[:, 8:12], [1, 0, 0, 0])
