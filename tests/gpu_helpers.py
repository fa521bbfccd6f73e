"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI (via the package's ctypes binding) and the FP64 oracle on the same
seeded float32 inputs."""
import numpy as np

import oracle

IMG_TOL = 1e-4      # max |S_gpu - S_ref| <= IMG_TOL * max S_ref
GRAD_TOL = 1e-3     # per group: ||g_gpu - g_ref||_inf <= GRAD_TOL * ||g_ref||_inf

GROUPS = {"mean": [0, 1, 2], "opacity": [3], "scale": [4, 5, 6], "P": [7], "quat": [8, 9, 10, 11]}


def f32(params):
    """The float32 parameters the GPU sees, and their exact float64 values
    for the oracle."""
    p32 = np.ascontiguousarray(params, dtype=np.float32)
    return p32, p32.astype(np.float64)


def gpu_forward(params32, views, scene_offsets=None, renderer=None, **cfg):
    import torch
    from paper_2506_21633_b300.render import Renderer, split_images
    r = renderer or Renderer(**cfg)
    p = torch.from_numpy(params32).cuda().contiguous()
    r.prepare(p, views, scene_offsets)
    vg = r.view_gauss()
    inten = torch.zeros(max(vg, 1), dtype=torch.float32, device="cuda")
    img = r.forward(intensity=inten)
    torch.cuda.synchronize()
    ims = [x.cpu().numpy().astype(np.float64) for x in split_images(img, views)]
    return ims, inten[:vg].cpu().numpy().astype(np.float64), r, p


def gpu_grad(params32, views, dLdS, scene_offsets=None, **cfg):
    import torch
    ims, inten, r, p = gpu_forward(params32, views, scene_offsets, **cfg)
    g = torch.from_numpy(np.concatenate([np.asarray(x, np.float32).ravel() for x in dLdS])).cuda()
    grads = r.backward(g)
    torch.cuda.synchronize()
    return grads.cpu().numpy().astype(np.float64), ims, inten


def assert_images(gpu, ref, tol=IMG_TOL):
    for k, (a, b) in enumerate(zip(gpu, ref)):
        scale = max(np.abs(b).max(), 1e-30)
        err = np.abs(a - b).max()
        assert err <= tol * scale, "view %d: max err %.3e, max ref %.3e" % (k, err, scale)


def assert_grads(gpu, ref, tol=GRAD_TOL, mask=None):
    # a group whose reference is exactly zero (a symmetry of the scene, e.g. the
    # rotation of isotropic Gaussians) has no scale of its own: it is held to
    # tol times the largest reference gradient of any group
    overall = max(np.abs(ref[:, cols]).max() if ref.size else 0.0 for cols in GROUPS.values())
    for name, cols in GROUPS.items():
        r = ref[:, cols]
        gpu_g = gpu[:, cols]
        scale = np.abs(r).max()
        if scale == 0:
            assert np.abs(gpu_g).max() <= tol * overall, "%s: reference 0, gpu %.3e" % (name, np.abs(gpu_g).max())
            continue
        d = np.abs(gpu_g - r)
        if mask is not None:
            d = d[mask]
        err = d.max()
        assert err <= tol * scale, "%s: max err %.3e vs scale %.3e (rel %.2e)" % (name, err, scale, err / scale)
