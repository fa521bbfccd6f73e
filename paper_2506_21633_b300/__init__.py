"""B300-native SAR Differentiable Gaussian Rasterizer (SDGR) of SAR-GS
(arXiv 2506.21633): hand-written sm_103a CUDA kernels behind a C ABI
(include/sdgr.h), with a thin ctypes binding and a torch.autograd.Function.
"""
from ._lib import LIB_PATH, SdgrError, lib  # noqa: F401


def __getattr__(name):
    # torch-dependent front end, imported on first use
    if name in ("Renderer", "SDGRRender", "render", "l1_loss", "adam_step", "split_images", "params_tensor"):
        from . import render as _r
        return getattr(_r, name)
    raise AttributeError(name)
