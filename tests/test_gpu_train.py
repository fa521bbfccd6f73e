"""Reconstruction demo on the GPU (Section III-B-3 set-up, shortened): from a
hemispherical initialisation, a few hundred batched iterations with the SH
schedule and densification raise PSNR and SSIM on held-out views of a
synthetic vehicle, lower the training loss, change the Gaussian count and
keep every parameter finite."""
import numpy as np
import pytest

import sdgr_scenes as sc

pytestmark = pytest.mark.gpu


def test_short_reconstruction():
    from paper_2506_21633_b300.train import reconstruct
    target = sc.tank_scene(3000, seed=1)
    views = sc.circular_views((35.0, 55.0), 12, 48, 0.25, center=(0.0, 0.0, 0.8))
    train = [v for k, v in enumerate(views) if k % 3 == 0]
    test = [v for k, v in enumerate(views) if k % 3 != 0]
    rep, tr = reconstruct(target, train, test, iters=300, n_init=3000, init_radius=4.5, seed=2,
                          sh_every=100, densify_from=100, densify_until=250, densify_every=25, log_every=50,
                          lr=(5e-3, 5e-3, 1e-3, 5e-2, 5e-3))
    b, a = rep["before"]["test"], rep["after"]["test"]
    assert a["psnr"] > b["psnr"] + 2.0, rep
    assert a["ssim"] > b["ssim"], rep
    assert rep["loss_curve"][-1][1] < 0.5 * rep["loss_curve"][0][1], rep
    assert rep["densify_events"] == 6 and 3000 < rep["gaussians"]["final"] <= 6000
    assert np.isfinite(tr.p.cpu().numpy()).all() and np.isfinite(tr.sh.cpu().numpy()).all()
