"""ctypes binding of libsdgr.so (the C ABI in include/sdgr.h).

Argument marshalling only: every step of the renderer runs in the CUDA
kernels of libsdgr.so.  Device pointers are passed as integers (e.g.
`tensor.data_ptr()`), streams as integers (`torch.cuda.Stream.cuda_stream`).
Loading fails loudly (ImportError) if the library has not been built; there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# SDGR_CHECKED=1: the build with index checks (see build.py)
LIB_PATH = os.path.join(_HERE, "libsdgr_checked.so" if os.environ.get("SDGR_CHECKED") == "1" else "libsdgr.so")

SDGR_OK, SDGR_ERR_INVALID, SDGR_ERR_CUDA, SDGR_ERR_CAPACITY, SDGR_ERR_TIMEOUT, SDGR_ERR_STATE, SDGR_ERR_BOUNDS = range(7)

# every function the header declares (checked by tests/test_abi.py)
EXPORTS = (
    "sdgr_caps_for", "sdgr_workspace_size", "sdgr_ws_create", "sdgr_ws_destroy", "sdgr_preprocess",
    "sdgr_bin_sort", "sdgr_render_fwd", "sdgr_render_bwd", "sdgr_adam_step", "sdgr_l1_loss",
    "sdgr_read_status", "sdgr_status_string", "sdgr_profile_enable", "sdgr_profile_read",
    "sdgr_count_pairs", "sdgr_launch_count", "sdgr_render_fwd_noalloc", "sdgr_adam_step_device",
    "sdgr_copy_status_async", "sdgr_set_sh", "sdgr_set_densify_stats", "sdgr_densify_scratch_bytes",
    "sdgr_densify", "sdgr_set_schedule", "sdgr_adam_step_flat", "sdgr_stage_batch_options",
    "sdgr_set_stage_batch", "sdgr_device_selfcheck", "sdgr_pipe_rates",
)

SELFCHECK_ALL = 1  # every bit sdgr_device_selfcheck defines

SCHED_ORDERED = 1
SCHED_PERSISTENT = 2
SCHEDULES = {"tiles": 0, "ordered": SCHED_ORDERED, "persistent": SCHED_ORDERED | SCHED_PERSISTENT}

# raster kernels by their index in sdgr_set_stage_batch
RASTER_KERNELS = ("intensity_fwd", "splat_fwd", "splat_bwd", "intensity_bwd")

STAGES = ("preprocess", "depth_sort", "bin", "intensity_fwd", "splat_fwd", "splat_bwd", "intensity_bwd",
          "param_bwd")


class SdgrView(ctypes.Structure):
    _fields_ = [
        ("phi", ctypes.c_double), ("theta", ctypes.c_double),
        ("dA", ctypes.c_double), ("dR", ctypes.c_double),
        ("NA", ctypes.c_int32), ("NR", ctypes.c_int32),
        ("scene", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("center", ctypes.c_double * 3),
    ]


class SdgrCfg(ctypes.Structure):
    _fields_ = [
        ("cutoff_K", ctypes.c_float), ("dilation_eps", ctypes.c_float),
        ("T_min", ctypes.c_float), ("norm_mode", ctypes.c_int32), ("alpha_mode", ctypes.c_int32),
    ]


class SdgrCaps(ctypes.Structure):
    _fields_ = [
        ("max_views", ctypes.c_int32), ("max_scenes", ctypes.c_int32),
        ("max_gaussians", ctypes.c_int64), ("max_view_gauss", ctypes.c_int64),
        ("max_pixels", ctypes.c_int64), ("max_tiles", ctypes.c_int64),
        ("max_instances", ctypes.c_int64),
    ]


class SdgrDensifyCfg(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("dense_scale", ctypes.c_float),
                ("max_scale", ctypes.c_float), ("min_opacity", ctypes.c_float),
                ("min_P", ctypes.c_float), ("split_factor", ctypes.c_float)]


class SdgrError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__("%s: %s (%d)" % (fn, status_string(code), code))


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built (run `python -m paper_2506_21633_b300.build`)"
                              % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        P = ctypes.POINTER
        L.sdgr_caps_for.argtypes = [P(SdgrView), i32, P(ctypes.c_int64), i32, i64, P(SdgrCaps)]
        L.sdgr_workspace_size.argtypes = [P(SdgrCfg), P(SdgrCaps), P(ctypes.c_size_t)]
        L.sdgr_ws_create.argtypes = [P(vp), vp, ctypes.c_size_t, P(SdgrCfg), P(SdgrCaps)]
        L.sdgr_ws_destroy.argtypes = [vp]
        L.sdgr_preprocess.argtypes = [vp, vp, P(ctypes.c_int64), i32, P(SdgrView), i32, vp]
        L.sdgr_bin_sort.argtypes = [vp, vp]
        L.sdgr_render_fwd.argtypes = [vp, vp, vp, vp]
        L.sdgr_render_bwd.argtypes = [vp, vp, vp, i32, vp]
        L.sdgr_count_pairs.argtypes = [vp, P(ctypes.c_int64), vp]
        L.sdgr_launch_count.argtypes = []
        L.sdgr_render_fwd_noalloc.argtypes = [vp, i64, P(SdgrView), i32, P(SdgrCfg), vp, vp, vp]
        L.sdgr_adam_step.argtypes = [vp, vp, vp, vp, i64, P(ctypes.c_float), f32, f32, f32, i32, vp]
        L.sdgr_adam_step_flat.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp]
        L.sdgr_l1_loss.argtypes = [vp, vp, i64, vp, vp, vp]
        L.sdgr_adam_step_device.argtypes = [vp, vp, vp, vp, i64, P(ctypes.c_float), f32, f32, f32, vp, vp]
        L.sdgr_read_status.argtypes = [vp, P(ctypes.c_int64)]
        L.sdgr_copy_status_async.argtypes = [vp, vp, vp]
        L.sdgr_set_sh.argtypes = [vp, vp, vp, i32]
        L.sdgr_set_densify_stats.argtypes = [vp, vp, vp]
        L.sdgr_set_schedule.argtypes = [vp, i32]
        L.sdgr_stage_batch_options.argtypes = [i32, P(ctypes.c_int32), i32]
        L.sdgr_stage_batch_options.restype = i32
        L.sdgr_set_stage_batch.argtypes = [vp, i32, i32]
        L.sdgr_device_selfcheck.argtypes = [vp, vp]
        L.sdgr_pipe_rates.argtypes = [vp, P(ctypes.c_double), vp]
        L.sdgr_densify_scratch_bytes.argtypes = [i64]
        L.sdgr_densify.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, P(SdgrDensifyCfg), vp, vp, vp, vp, i64, vp,
                                   P(ctypes.c_int64), vp]
        L.sdgr_profile_enable.argtypes = [vp, i32]
        L.sdgr_profile_read.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int64), i32]
        L.sdgr_status_string.argtypes = [ctypes.c_int]
        L.sdgr_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "sdgr_status_string":
                getattr(L, name).restype = ctypes.c_int
        L.sdgr_launch_count.restype = ctypes.c_int64
        L.sdgr_densify_scratch_bytes.restype = ctypes.c_size_t
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().sdgr_status_string(int(code)).decode()


def _check(fn, code):
    if code != SDGR_OK:
        raise SdgrError(fn, code)


def make_views(views):
    arr = (SdgrView * max(1, len(views)))()
    for k, v in enumerate(views):
        a = arr[k]
        a.phi, a.theta, a.dA, a.dR = v["phi"], v["theta"], v["dA"], v["dR"]
        a.NA, a.NR = v["NA"], v["NR"]
        a.scene = int(v.get("scene", 0))
        for j in range(3):
            a.center[j] = float(v["center"][j])
    return arr


def make_offsets(scene_offsets):
    arr = (ctypes.c_int64 * len(scene_offsets))()
    for k, o in enumerate(scene_offsets):
        arr[k] = int(o)
    return arr


def make_cfg(cutoff_K=5.0, dilation_eps=0.3, T_min=0.0, norm_mode=0, alpha_mode=0):
    return SdgrCfg(cutoff_K=cutoff_K, dilation_eps=dilation_eps, T_min=T_min, norm_mode=norm_mode,
                   alpha_mode=alpha_mode)


# -- thin wrappers with the C names ------------------------------------------

def sdgr_caps_for(views_arr, V, offsets_arr, n_scenes, instances):
    caps = SdgrCaps()
    _check("sdgr_caps_for", lib().sdgr_caps_for(views_arr, V, offsets_arr, n_scenes, int(instances),
                                                ctypes.byref(caps)))
    return caps


def sdgr_workspace_size(cfg, caps):
    n = ctypes.c_size_t()
    _check("sdgr_workspace_size", lib().sdgr_workspace_size(ctypes.byref(cfg), ctypes.byref(caps), ctypes.byref(n)))
    return n.value


def sdgr_ws_create(device_ptr, nbytes, cfg, caps):
    h = ctypes.c_void_p()
    _check("sdgr_ws_create", lib().sdgr_ws_create(ctypes.byref(h), ctypes.c_void_p(device_ptr), nbytes,
                                                  ctypes.byref(cfg), ctypes.byref(caps)))
    return h


def sdgr_ws_destroy(ws):
    _check("sdgr_ws_destroy", lib().sdgr_ws_destroy(ws))


def sdgr_preprocess(ws, params_ptr, offsets_arr, n_scenes, views_arr, V, stream):
    _check("sdgr_preprocess", lib().sdgr_preprocess(ws, ctypes.c_void_p(params_ptr), offsets_arr, n_scenes,
                                                    views_arr, V, ctypes.c_void_p(stream)))


def sdgr_bin_sort(ws, stream):
    _check("sdgr_bin_sort", lib().sdgr_bin_sort(ws, ctypes.c_void_p(stream)))


def sdgr_render_fwd(ws, images_ptr, intensity_ptr, stream):
    _check("sdgr_render_fwd", lib().sdgr_render_fwd(ws, ctypes.c_void_p(images_ptr),
                                                    ctypes.c_void_p(intensity_ptr or None),
                                                    ctypes.c_void_p(stream)))


def sdgr_render_bwd(ws, dLdS_ptr, grads_ptr, accumulate, stream):
    _check("sdgr_render_bwd", lib().sdgr_render_bwd(ws, ctypes.c_void_p(dLdS_ptr), ctypes.c_void_p(grads_ptr),
                                                    int(bool(accumulate)), ctypes.c_void_p(stream)))


def sdgr_count_pairs(ws, stream):
    out = (ctypes.c_int64 * 2)()
    _check("sdgr_count_pairs", lib().sdgr_count_pairs(ws, out, ctypes.c_void_p(stream)))
    return int(out[0]), int(out[1])


def sdgr_launch_count():
    return int(lib().sdgr_launch_count())


def sdgr_adam_step(p, g, m, v, N, lr, b1, b2, eps, step, stream):
    lr_arr = (ctypes.c_float * 5)(*[float(x) for x in lr])
    _check("sdgr_adam_step", lib().sdgr_adam_step(ctypes.c_void_p(p), ctypes.c_void_p(g), ctypes.c_void_p(m),
                                                  ctypes.c_void_p(v), int(N), lr_arr, b1, b2, eps, int(step),
                                                  ctypes.c_void_p(stream)))


def sdgr_adam_step_flat(x, g, m, v, n, lr, b1, b2, eps, step, stream):
    _check("sdgr_adam_step_flat", lib().sdgr_adam_step_flat(ctypes.c_void_p(x), ctypes.c_void_p(g), ctypes.c_void_p(m),
                                                            ctypes.c_void_p(v), int(n), float(lr), b1, b2, eps,
                                                            int(step), ctypes.c_void_p(stream)))


def sdgr_adam_step_device(p, g, m, v, N, lr, b1, b2, eps, step_ptr, stream):
    lr_arr = (ctypes.c_float * 5)(*[float(x) for x in lr])
    _check("sdgr_adam_step_device", lib().sdgr_adam_step_device(
        ctypes.c_void_p(p), ctypes.c_void_p(g), ctypes.c_void_p(m), ctypes.c_void_p(v), int(N), lr_arr, b1, b2, eps,
        ctypes.c_void_p(step_ptr), ctypes.c_void_p(stream)))


def sdgr_l1_loss(images, targets, npix, dLdS, loss, stream):
    _check("sdgr_l1_loss", lib().sdgr_l1_loss(ctypes.c_void_p(images), ctypes.c_void_p(targets), int(npix),
                                              ctypes.c_void_p(dLdS), ctypes.c_void_p(loss), ctypes.c_void_p(stream)))


def sdgr_set_densify_stats(ws, accum_ptr, count_ptr):
    _check("sdgr_set_densify_stats", lib().sdgr_set_densify_stats(ws, ctypes.c_void_p(accum_ptr or None),
                                                                  ctypes.c_void_p(count_ptr or None)))


def sdgr_set_schedule(ws, mode):
    _check("sdgr_set_schedule", lib().sdgr_set_schedule(ws, int(mode)))


def sdgr_stage_batch_options(kernel):
    """Supported staging batch sizes of raster kernel `kernel` (index or
    name), the default first."""
    k = RASTER_KERNELS.index(kernel) if isinstance(kernel, str) else int(kernel)
    buf = (ctypes.c_int32 * 8)()
    n = int(lib().sdgr_stage_batch_options(k, buf, 8))
    return tuple(int(buf[i]) for i in range(min(n, 8)))


def sdgr_set_stage_batch(ws, kernel, records):
    k = RASTER_KERNELS.index(kernel) if isinstance(kernel, str) else int(kernel)
    _check("sdgr_set_stage_batch", lib().sdgr_set_stage_batch(ws, k, int(records)))


def sdgr_device_selfcheck(flags_ptr, stream=None):
    """Enqueue the device self-check; it writes its bit mask to the device
    word at flags_ptr (uint32)."""
    _check("sdgr_device_selfcheck", lib().sdgr_device_selfcheck(ctypes.c_void_p(flags_ptr), stream))


PIPE_RATES_SCRATCH = 8192
PIPE_RATE_KINDS = ("ffma", "ex2", "rcp", "ex2_in_ffma_stream", "rcp_in_ffma_stream", "ffma2",
                   "ffma_and_lop3", "ffma2_and_lop3")


def sdgr_pipe_rates(scratch_ptr, stream=None):
    """Measured per-SM rates (thread-instructions per SM cycle) of fma, ex2,
    rcp, of streams of one ex2 per seven fma and one rcp per eight fma, of
    fma.f32x2 (two FMAs each) and of fma or fma.f32x2 alternating with an
    integer lop3; synchronous.
    scratch_ptr: device memory of PIPE_RATES_SCRATCH bytes."""
    out = (ctypes.c_double * len(PIPE_RATE_KINDS))()
    _check("sdgr_pipe_rates", lib().sdgr_pipe_rates(ctypes.c_void_p(scratch_ptr), out, ctypes.c_void_p(stream)))
    return dict(zip(PIPE_RATE_KINDS, (float(x) for x in out)))


def sdgr_densify_scratch_bytes(N):
    return int(lib().sdgr_densify_scratch_bytes(int(N)))


def sdgr_densify(params, grads, accum, count, m, v, sh, N, cfg, out_p, out_m, out_v, out_sh, cap, scratch, stream):
    """Returns (status code, new_N); pointers as integers (sh/out_sh may be None)."""
    n = ctypes.c_int64()
    code = lib().sdgr_densify(*[ctypes.c_void_p(x) for x in (params, grads, accum, count, m, v, sh)], int(N),
                              ctypes.byref(cfg), *[ctypes.c_void_p(x) for x in (out_p, out_m, out_v, out_sh)],
                              int(cap), ctypes.c_void_p(scratch), ctypes.byref(n), ctypes.c_void_p(stream))
    if code not in (SDGR_OK, SDGR_ERR_CAPACITY):
        raise SdgrError("sdgr_densify", code)
    return code, n.value


def sdgr_set_sh(ws, sh_ptr, dsh_ptr, degree):
    _check("sdgr_set_sh", lib().sdgr_set_sh(ws, ctypes.c_void_p(sh_ptr or None), ctypes.c_void_p(dsh_ptr or None),
                                            int(degree)))


def sdgr_copy_status_async(ws, host_ptr, stream):
    _check("sdgr_copy_status_async", lib().sdgr_copy_status_async(ws, ctypes.c_void_p(host_ptr),
                                                                  ctypes.c_void_p(stream)))


def sdgr_read_status(ws):
    req = ctypes.c_int64()
    code = lib().sdgr_read_status(ws, ctypes.byref(req))
    if code not in (SDGR_OK, SDGR_ERR_CAPACITY, SDGR_ERR_TIMEOUT):
        raise SdgrError("sdgr_read_status", code)
    return code, req.value


def sdgr_profile_enable(ws, enable=True):
    _check("sdgr_profile_enable", lib().sdgr_profile_enable(ws, int(bool(enable))))


def sdgr_profile_read(ws, reset=True):
    """{stage name: (total ms, launches)} since the last reset."""
    n = len(STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check("sdgr_profile_read", lib().sdgr_profile_read(ws, ms, cnt, int(bool(reset))))
    return {STAGES[k]: (ms[k], cnt[k]) for k in range(n)}
