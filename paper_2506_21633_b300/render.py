"""Python front end of the B300 SAR Gaussian rasterizer.

`Renderer` owns a workspace (one torch uint8 device buffer handed to the C
ABI) and sequences the C calls of one step; `SDGRRender` is the
torch.autograd.Function whose backward is the hand-written adjoint.  PyTorch
provides device memory and streams only: all arithmetic runs in libsdgr.so.
"""
from __future__ import annotations

import torch

from . import _lib as L

_CAP_FIELDS = ("max_views", "max_scenes", "max_gaussians", "max_view_gauss", "max_pixels", "max_tiles",
               "max_instances")


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def views_npix(views):
    return sum(int(v["NA"]) * int(v["NR"]) for v in views)


def split_images(flat, views):
    out, off = [], 0
    for v in views:
        n = int(v["NA"]) * int(v["NR"])
        out.append(flat[off:off + n].view(int(v["NR"]), int(v["NA"])))
        off += n
    return out


class Renderer:
    """Workspace plus the call sequence preprocess -> bin_sort -> render_fwd
    [-> render_bwd].  Capacities grow on demand; the instance count of a new
    scene/view set is learned from the device status word (one host sync in
    `prepare(check=True)`)."""

    def __init__(self, cutoff_K=5.0, dilation_eps=0.3, T_min=0.0, norm_mode=0, device=None, inst_slack=1.15,
                 alpha_mode=0):
        L.lib()  # fail loudly if the library is missing
        self.cfg = L.make_cfg(cutoff_K, dilation_eps, T_min, norm_mode, alpha_mode)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.inst_slack = inst_slack
        self.ws = None
        self.buf = None
        self.caps = None
        self.views = None
        self.scene_offsets = None
        self.params = None
        self.n_inst = None
        self.schedule = "persistent"
        self.stage_batch = {}  # raster kernel name -> staging batch (absent: the kernel's default)
        # bumped by every prepare(): the workspace then holds another scene or
        # view set, and an adjoint of an earlier forward is no longer possible
        self.generation = 0

    def __del__(self):
        try:
            if self.ws is not None:
                L.sdgr_ws_destroy(self.ws)
        except Exception:
            pass

    # -- workspace -----------------------------------------------------------
    def _grow(self, need):
        if self.caps is not None and all(getattr(need, f) <= getattr(self.caps, f) for f in _CAP_FIELDS):
            return
        caps = L.SdgrCaps()
        for f in _CAP_FIELDS:
            cur = getattr(self.caps, f) if self.caps is not None else 0
            setattr(caps, f, max(cur, getattr(need, f)))
        nbytes = L.sdgr_workspace_size(self.cfg, caps)
        if self.ws is not None:
            torch.cuda.synchronize(self.device)
            L.sdgr_ws_destroy(self.ws)
            self.ws = None
            self.buf = None
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ws = L.sdgr_ws_create(self.buf.data_ptr(), nbytes, self.cfg, caps)
        self.caps = caps
        pend = getattr(self, "_sh_state", None)
        if pend is not None:  # the SH binding belongs to the workspace: carry it over
            L.sdgr_set_sh(self.ws, *pend)
        dens = getattr(self, "_dens_state", None)
        if dens is not None:
            L.sdgr_set_densify_stats(self.ws, *dens)
        L.sdgr_set_schedule(self.ws, L.SCHEDULES[self.schedule])
        for k, nb in self.stage_batch.items():
            L.sdgr_set_stage_batch(self.ws, k, nb)

    def workspace_bytes(self):
        return 0 if self.buf is None else self.buf.numel()

    # -- step calls ----------------------------------------------------------
    def prepare(self, params, views, scene_offsets=None, stream=None, check=True, instances=None):
        """preprocess + bin_sort.  params: cuda float32 [N, 12] contiguous."""
        assert params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()
        if scene_offsets is None:
            scene_offsets = [0, params.shape[0]]
        vs = L.make_views(views)
        offs = L.make_offsets(scene_offsets)
        n_scenes = len(scene_offsets) - 1
        s = _stream_handle(stream)
        self.generation += 1
        guess = instances if instances is not None else (self.n_inst if self.n_inst is not None else None)
        if guess is None:
            base = L.sdgr_caps_for(vs, len(views), offs, n_scenes, 0)
            guess = 8 * base.max_view_gauss + 2 * base.max_tiles
        for attempt in range(3):
            need = L.sdgr_caps_for(vs, len(views), offs, n_scenes, min(int(guess), 0x7fffffff))
            self._grow(need)
            L.sdgr_preprocess(self.ws, params.data_ptr(), offs, n_scenes, vs, len(views), s)
            L.sdgr_bin_sort(self.ws, s)
            if not check:
                break
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
            code, required = L.sdgr_read_status(self.ws)
            if code == L.SDGR_OK:
                self.n_inst = required
                break
            if code != L.SDGR_ERR_CAPACITY:
                raise L.SdgrError("device status", code)
            guess = int(required * self.inst_slack) + 1024
        else:
            raise L.SdgrError("prepare", L.SDGR_ERR_CAPACITY)
        self.views = views
        self.scene_offsets = list(scene_offsets)
        self.params = params
        return self

    def forward(self, images=None, intensity=None, stream=None):
        npix = views_npix(self.views)
        if images is None:
            images = torch.empty(npix, dtype=torch.float32, device=self.device)
        L.sdgr_render_fwd(self.ws, images.data_ptr(), intensity.data_ptr() if intensity is not None else None,
                          _stream_handle(stream))
        return images

    def backward(self, dL_dimages, grads=None, accumulate=False, stream=None):
        """Adjoint; grads is overwritten, or added to with accumulate=True."""
        if grads is None:
            grads = torch.empty_like(self.params)
            accumulate = False
        assert dL_dimages.is_contiguous() and dL_dimages.dtype == torch.float32
        L.sdgr_render_bwd(self.ws, dL_dimages.data_ptr(), grads.data_ptr(), accumulate, _stream_handle(stream))
        return grads

    def set_sh(self, sh=None, dsh=None, degree=0):
        """View-dependent scattering: sh, dsh cuda float32 [N, 16] (or None);
        applies to the following prepare()/backward() calls."""
        self._sh = (sh, dsh)  # keep the tensors alive while the workspace points at them
        self._sh_state = (sh.data_ptr() if sh is not None else None, dsh.data_ptr() if dsh is not None else None,
                          degree)
        if self.ws is not None:
            L.sdgr_set_sh(self.ws, *self._sh_state)

    def set_densify_stats(self, accum=None, count=None):
        """Bind (or with None, unbind) the densification statistics buffers,
        cuda float32 [N]; every following backward() adds |dL/du_I| and 1 per
        (view, Gaussian) with image-plane weight."""
        self._dens = (accum, count)
        self._dens_state = (accum.data_ptr() if accum is not None else None,
                            count.data_ptr() if count is not None else None)
        if self.ws is not None:
            L.sdgr_set_densify_stats(self.ws, *self._dens_state)

    def set_schedule(self, name):
        """Raster launch policy: 'tiles' (one CTA per tile), 'ordered' (one
        CTA per non-empty tile, longest list first) or 'persistent' (resident
        CTAs pulling the ordered list).  Applies to the following forward /
        backward calls."""
        if name not in L.SCHEDULES:
            raise ValueError(f"unknown schedule {name!r}")
        self.schedule = name
        if self.ws is not None:
            L.sdgr_set_schedule(self.ws, L.SCHEDULES[name])

    def set_stage_batch(self, kernel, records):
        """Gaussian records a CTA of raster kernel `kernel` ('intensity_fwd',
        'splat_fwd', 'splat_bwd' or 'intensity_bwd') stages per batch; one of
        L.sdgr_stage_batch_options(kernel), or 0 / None for the default.
        Applies to the following forward / backward calls; the results do not
        depend on it."""
        if kernel not in L.RASTER_KERNELS:
            raise ValueError(f"unknown raster kernel {kernel!r}")
        records = int(records or 0)
        if records and records not in L.sdgr_stage_batch_options(kernel):
            raise ValueError(f"{kernel} has no staging batch of {records} records")
        if records:
            self.stage_batch[kernel] = records
        else:
            self.stage_batch.pop(kernel, None)
        if self.ws is not None:
            L.sdgr_set_stage_batch(self.ws, kernel, records)

    def count_pairs(self, stream=None):
        """In-cutoff (pixel, Gaussian) pairs (computation plane, imaging plane)
        of the current lists; synchronous."""
        return L.sdgr_count_pairs(self.ws, _stream_handle(stream))

    def profile(self, enable=True):
        L.sdgr_profile_enable(self.ws, enable)

    def profile_read(self, reset=True):
        return L.sdgr_profile_read(self.ws, reset)

    def status(self):
        return L.sdgr_read_status(self.ws)

    def view_gauss(self):
        return sum(self.scene_offsets[v.get("scene", 0) + 1] - self.scene_offsets[v.get("scene", 0)]
                   for v in self.views)


class StaleRendererError(RuntimeError):
    """The renderer of an SDGRRender node was prepared again (other
    parameters or views) before that node's backward ran."""


class SDGRRender(torch.autograd.Function):
    """images (flat, views concatenated) = SDGR(params); backward = the
    hand-written adjoint of Section II-B (dL/dS from autograd, then the
    splat, intensity and projection adjoints in libsdgr.so).

    The sorted lists and per-ray end state the adjoint needs stay in the
    renderer's workspace (per-tile visibility is recomputed, not stored), so
    the renderer must not be prepared again between this forward and its
    backward: a generation count taken at the forward is checked in the
    backward, which raises StaleRendererError instead of differentiating
    another scene.  params are saved, so autograd's version check refuses a
    backward after they were modified in place (e.g. by an optimiser step)."""

    @staticmethod
    def forward(ctx, params, renderer, views, scene_offsets=None):
        renderer.prepare(params.detach().contiguous(), views, scene_offsets)
        images = renderer.forward()
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        ctx.save_for_backward(params)
        return images

    @staticmethod
    def backward(ctx, dL_dimages):
        ctx.saved_tensors  # raises if params changed in place since the forward
        r = ctx.renderer
        if r.generation != ctx.generation:
            raise StaleRendererError("SDGRRender: the renderer was prepared again (generation %d, forward at %d); "
                                     "run backward before the next forward on the same renderer, or use one "
                                     "renderer per graph" % (r.generation, ctx.generation))
        grads = r.backward(dL_dimages.contiguous())
        return grads, None, None, None


def render(params, views, scene_offsets=None, renderer=None, **cfg):
    """Plain forward: returns the list of [NR, NA] images."""
    r = renderer or Renderer(**cfg)
    r.prepare(params.contiguous(), views, scene_offsets)
    return split_images(r.forward(), views)


def l1_loss(images, targets, dL_dimages=None, loss=None, stream=None):
    n = images.numel()
    if dL_dimages is None:
        dL_dimages = torch.empty_like(images)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=images.device)
    L.sdgr_l1_loss(images.data_ptr(), targets.data_ptr(), n, dL_dimages.data_ptr(), loss.data_ptr(),
                   _stream_handle(stream))
    return loss, dL_dimages


def adam_step(params, grads, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15, stream=None):
    L.sdgr_adam_step(params.data_ptr(), grads.data_ptr(), m.data_ptr(), v.data_ptr(), params.shape[0], lr, b1, b2,
                     eps, step, _stream_handle(stream))


def params_tensor(params_np, device=None):
    """float32 [N, 12] device tensor from a NumPy parameter array."""
    t = torch.as_tensor(params_np, dtype=torch.float32)
    return t.to(device or torch.device("cuda")).contiguous()
