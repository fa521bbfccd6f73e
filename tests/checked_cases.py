"""Tiny cases for the index-checked library, run in a child process with
SDGR_CHECKED=1 by test_gpu_checked.py: 1-4 Gaussians, 8x8 and ragged 9x7
images, every raster schedule, forward + backward against the oracle, and
the status word after each call (a bounds violation would report
SDGR_ERR_BOUNDS)."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
import sdgr_scenes as sc  # noqa: E402
from gpu_helpers import assert_grads, assert_images, f32  # noqa: E402


def main():
    import torch
    from paper_2506_21633_b300 import _lib as L
    from paper_2506_21633_b300.render import Renderer, split_images
    assert os.path.basename(L.LIB_PATH) == "libsdgr_checked.so", L.LIB_PATH
    rng = np.random.default_rng(0)
    cases = 0
    for n in (1, 2, 3, 4):
        params = sc.vehicle_box_scene(n, seed=n, extent=(0.3, 0.3, 0.3), log_s_mean=math.log(0.08), center=(0, 0, 0))
        views = [sc.make_view(30.0 * n, 40.0, 0.06, 0.06, 8, 8), sc.make_view(200.0, 55.0, 0.05, 0.07, 9, 7)]
        p32, p64 = f32(params)
        G = [rng.normal(size=(v["NR"], v["NA"])) for v in views]
        ref_img, _, _ = oracle.render(p64, views, oracle.cfg())
        ref_g = oracle.grad(p64, views, G, oracle.cfg())[0]
        for sched in ("tiles", "ordered", "persistent"):
            r = Renderer()
            r.set_schedule(sched)
            p = torch.from_numpy(p32).cuda()
            img = r.prepare(p, views).forward()
            g = torch.from_numpy(np.concatenate([x.ravel() for x in G]).astype(np.float32)).cuda()
            grads = r.backward(g)
            torch.cuda.synchronize()
            code, _ = r.status()
            assert code == L.SDGR_OK, (n, sched, L.status_string(code))
            assert_images([x.cpu().numpy().astype(np.float64) for x in split_images(img, views)], ref_img)
            assert_grads(grads.cpu().numpy().astype(np.float64), ref_g)
            cases += 1
    print("checked tiny cases ok: %d" % cases)


if __name__ == "__main__":
    main()
