"""FP64 CPU oracle of the SAR differentiable Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`; the product package never imports
it, and it imports nothing from the product package.

`sdgr_oracle.c` holds the renderer and its adjoint (brute force, double
precision, following Section II of the paper in order); `numpy_twin.py` is a
separately written NumPy forward for tiny scenes.  This module only
marshals arguments for the C code through ctypes.

Parity status: every function here is pinned by the `-m "not gpu"` tests in
`tests/test_oracle_pins.py` (closed forms, invariants, finite differences,
library routines); see the header of that file for which pin covers which
step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdgr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


class OrcView(ctypes.Structure):
    _fields_ = [
        ("phi", ctypes.c_double), ("theta", ctypes.c_double),
        ("dA", ctypes.c_double), ("dR", ctypes.c_double),
        ("NA", ctypes.c_int32), ("NR", ctypes.c_int32),
        ("pad0", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("center", ctypes.c_double * 3),
    ]


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_double), ("eps", ctypes.c_double), ("T_min", ctypes.c_double),
        ("norm_mode", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
        ("alpha_mode", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("sh", ctypes.POINTER(ctypes.c_double)), ("dsh", ctypes.POINTER(ctypes.c_double)),
        ("duI", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, OpenMP) if missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        # SDGR_ORACLE_LIB: another build of sdgr_oracle.c (the mutation test
        # plants mistakes in copies of the source and runs the pins on them)
        path = os.environ.get("SDGR_ORACLE_LIB")
        if not path:
            build()
            path = _LIB
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_render.argtypes = [dp, ctypes.c_int32, ctypes.POINTER(OrcView), ctypes.c_int32,
                                 ctypes.POINTER(OrcCfg), ctypes.c_int32, dp, dp, dp]
        L.orc_grad.argtypes = [dp, ctypes.c_int32, ctypes.POINTER(OrcView), ctypes.c_int32,
                               ctypes.POINTER(OrcCfg), ctypes.c_int32, dp, dp, dp]
        L.orc_project.argtypes = [dp, ctypes.c_int32, ctypes.POINTER(OrcView), ctypes.POINTER(OrcCfg), dp]
        L.orc_depth_order.argtypes = [dp, ctypes.c_int32, ctypes.POINTER(OrcView), ctypes.POINTER(OrcCfg),
                                      ctypes.POINTER(ctypes.c_int32)]
        L.orc_adam.argtypes = [dp, dp, dp, dp, ctypes.c_int64, dp, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int32]
        L.orc_l1.argtypes = [dp, dp, ctypes.c_int64, dp]
        L.orc_l1.restype = ctypes.c_double
        L.orc_step.argtypes = [dp, ctypes.c_int32, ctypes.POINTER(OrcView), ctypes.c_int32,
                               ctypes.POINTER(OrcCfg), ctypes.c_int32, dp, dp, dp]
        L.orc_step.restype = ctypes.c_double
        L.orc_sh_basis.argtypes = [dp, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def cfg(K=5.0, eps=0.3, T_min=0.0, norm_mode=0, sh=None, sh_degree=0, alpha_mode=0) -> OrcCfg:
    """sh: optional [N,16] float64 coefficients of the SH degrees 1..3
    (view-dependent scattering), used up to sh_degree.  alpha_mode 1: the
    Beer-Lambert opacity 1 - exp(-tau G), tau = softplus(opacity logit)."""
    c = OrcCfg(K=float(K), eps=float(eps), T_min=float(T_min), norm_mode=int(norm_mode), sh_degree=int(sh_degree),
               alpha_mode=int(alpha_mode))
    if sh is not None:
        a = np.ascontiguousarray(sh, dtype=np.float64)
        assert a.ndim == 2 and a.shape[1] == 16
        c._sh = a  # keep alive
        c.sh = _dp(a)
    return c


def sh_basis(d):
    """The 15 real SH values of degrees 1..3 at unit direction d."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    Y = np.zeros(15)
    lib().orc_sh_basis(_dp(d), _dp(Y))
    return Y


def _views(views):
    arr = (OrcView * max(1, len(views)))()
    for k, v in enumerate(views):
        arr[k].phi, arr[k].theta = v["phi"], v["theta"]
        arr[k].dA, arr[k].dR = v["dA"], v["dR"]
        arr[k].NA, arr[k].NR = v["NA"], v["NR"]
        for j in range(3):
            arr[k].center[j] = v["center"][j]
    return arr


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    assert p.ndim == 2 and p.shape[1] == 12
    return p


def split_images(flat, views):
    out, off = [], 0
    for v in views:
        n = v["NA"] * v["NR"]
        out.append(flat[off:off + n].reshape(v["NR"], v["NA"]))
        off += n
    return out


def render(params, views, c=None, culled=False):
    """Returns (images list [NR,NA] per view, A [V,N], Tfinal list per view)."""
    c = c or cfg()
    p = _params(params)
    N, V = p.shape[0], len(views)
    npix = sum(v["NA"] * v["NR"] for v in views)
    img = np.zeros(npix)
    A = np.zeros((V, max(N, 1)))
    Tf = np.zeros(npix)
    rc = lib().orc_render(_dp(p), N, _views(views), V, ctypes.byref(c), int(culled), _dp(img), _dp(A), _dp(Tf))
    if rc:
        raise ValueError("oracle: invalid arguments")
    return split_images(img, views), A[:, :N], split_images(Tf, views)


def grad(params, views, dLdS, c=None, culled=False):
    """dLdS: list of [NR,NA] arrays (one per view).  Returns (grads [N,12],
    dL/dI [V,N])."""
    c = c or cfg()
    p = _params(params)
    N, V = p.shape[0], len(views)
    g = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in dLdS]))
    out = np.zeros((max(N, 1), 12))
    dI = np.zeros((V, max(N, 1)))
    rc = lib().orc_grad(_dp(p), N, _views(views), V, ctypes.byref(c), int(culled), _dp(g), _dp(out), _dp(dI))
    if rc:
        raise ValueError("oracle: invalid arguments")
    return out[:N], dI[:, :N]


def grad_sh(params, views, dLdS, c, culled=False):
    """As grad(), plus dL/dsh [N,16] for a cfg built with sh coefficients."""
    p = _params(params)
    dsh = np.zeros((max(p.shape[0], 1), 16))
    c.dsh = _dp(dsh)
    try:
        g, dI = grad(p, views, dLdS, c, culled)
    finally:
        c.dsh = ctypes.POINTER(ctypes.c_double)()
    return g, dsh[:p.shape[0]]


def grad_uI(params, views, dLdS, c=None, culled=False):
    """As grad(), plus dL/du_I (image-plane pixel coordinates) per view and
    Gaussian, [V, N, 2]."""
    c = c or cfg()
    p = _params(params)
    duI = np.zeros((max(len(views), 1), max(p.shape[0], 1), 2))
    c.duI = _dp(duI)
    try:
        g, dI = grad(p, views, dLdS, c, culled)
    finally:
        c.duI = ctypes.POINTER(ctypes.c_double)()
    return g, dI, duI[:len(views), :p.shape[0]]


def step(params, views, targets, c=None, culled=True):
    """Forward, L1 against targets, adjoint.  Returns (loss, images list,
    grads [N,12])."""
    c = c or cfg()
    p = _params(params)
    N, V = p.shape[0], len(views)
    t = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in targets]))
    img = np.zeros(t.size)
    out = np.zeros((max(N, 1), 12))
    loss = lib().orc_step(_dp(p), N, _views(views), V, ctypes.byref(c), int(culled), _dp(t), _dp(img), _dp(out))
    if loss != loss:
        raise ValueError("oracle: invalid arguments")
    return loss, split_images(img, views), out[:N]


PROJ_FIELDS = ["uCx", "uCy", "SCxx", "SCxy", "SCyy", "uIx", "uIy", "SIxx", "SIxy", "SIyy",
               "key", "cnorm", "o", "zr", "detC", "detI"]


def project(params, view, c=None):
    """Per-Gaussian projected quantities of one view as a dict of arrays."""
    c = c or cfg()
    p = _params(params)
    N = p.shape[0]
    out = np.zeros((max(N, 1), 16))
    rc = lib().orc_project(_dp(p), N, _views([view]), ctypes.byref(c), _dp(out))
    if rc:
        raise ValueError("oracle: invalid arguments")
    return {k: out[:N, j] for j, k in enumerate(PROJ_FIELDS)}


def depth_order(params, view, c=None):
    c = c or cfg()
    p = _params(params)
    N = p.shape[0]
    out = np.zeros(max(N, 1), dtype=np.int32)
    rc = lib().orc_depth_order(_dp(p), N, _views([view]), ctypes.byref(c),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc:
        raise ValueError("oracle: invalid arguments")
    return out[:N]


def adam(params, grads, m, v, lr, b1, b2, eps, step):
    """In-place Adam update on float64 [N,12] arrays; lr = 5 group rates."""
    for a in (params, grads, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lr = np.ascontiguousarray(lr, dtype=np.float64)
    rc = lib().orc_adam(_dp(params), _dp(grads), _dp(m), _dp(v), params.shape[0], _dp(lr), b1, b2, eps, step)
    if rc:
        raise ValueError("oracle: invalid arguments")


def l1(images, targets):
    """Mean L1 over all pixels of all views and dL/dS (list per view)."""
    S = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).ravel() for x in images]))
    T = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).ravel() for x in targets]))
    g = np.zeros_like(S)
    loss = lib().orc_l1(_dp(S), _dp(T), S.size, _dp(g))
    shapes = [np.asarray(x).shape for x in images]
    out, off = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(g[off:off + n].reshape(sh))
        off += n
    return loss, out


def linear_loss_grad_fd(params, views, G, c=None, idx=None, h_rel=1e-6, culled=False):
    """Central finite differences of L = sum_v sum_pix G_v * S_v with respect
    to the raw parameters listed in idx (pairs (gaussian, component)).
    Returns (fd values, list of flags: True where the depth order or the set
    of contributing pixels changed between p-h and p+h, so the difference
    straddles a discontinuity)."""
    c = c or cfg()
    p0 = _params(params).copy()
    out, bad = [], []
    orders0 = [depth_order(p0, v, c) for v in views]
    for (i, j) in idx:
        h = h_rel * max(1.0, abs(p0[i, j]))
        vals = []
        disc = False
        for sgn in (+1, -1):
            p = p0.copy()
            p[i, j] += sgn * h
            imgs, _, _ = render(p, views, c, culled)
            vals.append(sum(float((np.asarray(g) * im).sum()) for g, im in zip(G, imgs)))
            for v, o0 in zip(views, orders0):
                if not np.array_equal(depth_order(p, v, c), o0):
                    disc = True
        out.append((vals[0] - vals[1]) / (2 * h))
        bad.append(disc)
    return np.array(out), bad
