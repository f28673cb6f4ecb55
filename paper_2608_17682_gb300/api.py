"""PyTorch-facing API over libvt.so.

PyTorch supplies device memory and the current stream; every step of the
rendering path runs in the library's CUDA kernels. ``VTRender`` is the
``torch.autograd.Function``: its forward calls vt_render_fwd and saves only
the output colours (no per-ray cell lists); its backward calls vt_render_bwd,
which re-traverses each ray (recomputation in place of storing the walk).
"""
from __future__ import annotations

import ctypes

import torch

from . import _vt
from ._vt import VT_BF16, VT_F16, VT_F32, VTError  # noqa: F401

_DTYPES = {"f32": VT_F32, "fp32": VT_F32, "f16": VT_F16, "fp16": VT_F16, "bf16": VT_BF16}


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def _dev_f32(x, device):
    return torch.as_tensor(x, dtype=torch.float32, device=device).contiguous()


def _arr(t, name, shape, dtype=torch.float32, optional=False):
    """Checks a tensor the library reads or writes through a raw pointer: a
    C-contiguous CUDA tensor of `dtype` and `shape`. A wrong one would make the
    kernels read or write outside it, so it is rejected before any call."""
    if t is None:
        if optional:
            return
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


class Scene:
    """A Voronoi scene resident on the GPU (library-owned, Morton-ordered)."""

    def __init__(self, sites, sigma, tex, adj_offsets, adj_indices, tex_dtype="f32", device="cuda",
                 keep_order=False, tex_vd=None, half_offsets=False):
        device = torch.device(device)
        self.device = device
        sites = _dev_f32(sites, device)
        sigma = _dev_f32(sigma, device)
        tex = _dev_f32(tex, device)
        tvd = None if tex_vd is None else _dev_f32(tex_vd, device)
        if tvd is not None and tvd.shape != tex.shape:
            raise ValueError("tex_vd must have the shape of tex")
        self.has_tex_vd = tvd is not None
        off = torch.as_tensor(adj_offsets, dtype=torch.int64, device=device).contiguous()
        idx = torch.as_tensor(adj_indices, dtype=torch.int32, device=device).contiguous()
        n = sites.shape[0]
        if sites.shape != (n, 3) or sigma.shape != (n,) or tex.dim() != 4 or tex.shape[0] != n \
                or tex.shape[1] != tex.shape[2] or tex.shape[3] != 3 or off.shape != (n + 1,):
            raise ValueError("bad scene shapes")
        self.n, self.R = n, tex.shape[1]
        self.tex_dtype = _DTYPES[tex_dtype] if isinstance(tex_dtype, str) else int(tex_dtype)
        desc = _vt.vt_scene_desc(n, self.R, self.tex_dtype, sites.data_ptr(), sigma.data_ptr(), tex.data_ptr(),
                                 off.data_ptr(), idx.data_ptr(),
                                 (_vt.VT_SCENE_KEEP_ORDER if keep_order else 0)
                                 | (_vt.VT_SCENE_HALF_OFFSETS if half_offsets else 0), _ptr(tvd))
        with torch.cuda.device(device):
            self.handle = _vt.vt_scene_create(desc, _stream())
        self.n_edges = _vt.vt_scene_info(self.handle)[3]

    @classmethod
    def from_workload(cls, sc, tex_dtype="f32", device="cuda", keep_order=False, tex_vd=None, half_offsets=False):
        return cls(sc.sites, sc.sigma, sc.tex, sc.offsets, sc.indices, tex_dtype=tex_dtype, device=device,
                   keep_order=keep_order, tex_vd=tex_vd, half_offsets=half_offsets)

    def update(self, sites=None, sigma=None, tex=None, tex_vd=None):
        keep = [None if x is None else _dev_f32(x, self.device) for x in (sites, sigma, tex, tex_vd)]
        n, R = self.n, self.R
        for x, name, shape in zip(keep, ("sites", "sigma", "tex", "tex_vd"),
                                  ((n, 3), (n,), (n, R, R, 3), (n, R, R, 3))):
            _arr(x, name, shape, optional=True)
        if keep[3] is not None and not self.has_tex_vd:
            raise ValueError("tex_vd given for a scene built without one")
        _vt.vt_scene_update(self.handle, *[_ptr(x) for x in keep], _stream())

    def permutation(self):
        """perm [N] int32 on the device: perm[k] = user id of the scene's cell k."""
        perm = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _vt.vt_scene_permutation(self.handle, perm.data_ptr(), _stream())
        return perm

    def get_error(self):
        """(status, fp64_rechecks) since the last call; synchronises the stream."""
        return _vt.vt_scene_get_error(self.handle, _stream())

    def close(self):
        if getattr(self, "handle", None):
            _vt.vt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(t_near=0.0, t_far=20.0, use_clip_box=False, clip_lo=(0, 0, 0), clip_hi=(1, 1, 1), T_eps=1e-4,
                skip_weight=0.0, bg=(1, 1, 1), img_w=0, img_h=0, n_images=0, max_steps=0, image_sizes=None,
                appearance=0):
    """Render parameters. image_sizes: optional list of (w, h) per image for
    launches whose images differ in size (e.g. pinhole and 4-sample thin-lens
    views in one launch)."""
    p = _vt.vt_render_params()
    p.t_near, p.t_far, p.use_clip_box = t_near, t_far, int(bool(use_clip_box))
    p.clip_lo[:] = list(clip_lo)
    p.clip_hi[:] = list(clip_hi)
    p.T_eps, p.skip_weight = T_eps, skip_weight
    p.bg[:] = list(bg)
    p.img_w, p.img_h, p.n_images, p.max_steps = img_w, img_h, n_images, max_steps
    p.appearance = int(appearance)
    if image_sizes is not None:
        arr = (ctypes.c_int32 * (2 * len(image_sizes)))(*[int(v) for wh in image_sizes for v in wh])
        p._image_sizes_keepalive = arr  # the struct holds a raw pointer to it
        p.image_sizes = ctypes.cast(arr, ctypes.c_void_p)
        p.n_images = len(image_sizes)
    return p


def camera_struct(cam) -> _vt.vt_camera:
    """vt_camera from a workloads.Camera-like object."""
    c = _vt.vt_camera()
    c.kind, c.w, c.h = cam.kind, cam.w, cam.h
    c.eye[:] = list(cam.eye)
    c.fwd[:] = list(cam.fwd)
    c.up[:] = list(cam.up)
    c.fov_y, c.fisheye_fov = cam.fov_y, cam.fisheye_fov
    c.rs_velocity[:] = list(cam.rs_velocity)
    c.lens_radius, c.focus_dist, c.lens_samples, c.seed = cam.lens_radius, cam.focus_dist, cam.lens_samples, cam.seed
    return c


def generate_rays(cameras, device="cuda", out=None):
    """Rays of all cameras, in order [camera][row][col][lens sample]."""
    cs = [camera_struct(c) for c in cameras]
    n = sum(_vt.vt_camera_n_rays(c) for c in cs)
    if out is None:
        o = torch.empty(n, 3, device=device)
        d = torch.empty(n, 3, device=device)
        t = torch.empty(n, device=device)
    else:
        o, d, t = out
        _arr(o, "o", (n, 3))
        _arr(d, "d", (n, 3))
        _arr(t, "time", (n,))
    _vt.vt_generate_rays(cs, o.data_ptr(), d.data_ptr(), t.data_ptr(), _stream())
    return o, d, t


def render_fwd(scene: Scene, o, d, params, time=None, out=None, want_steps=True, residual=None, dist=None):
    """Forward render; returns (rgb, T, steps). If `residual` is a [n,3] tensor
    it receives C - rgb (the float-float colour's rounding residual) for an
    exact backward. If `dist` is a [n,3] tensor it receives the distortion
    loss per ray (column 0, Eq. 2) and the two totals the backward needs."""
    n = o.shape[0]
    _arr(o, "o", (n, 3))
    _arr(d, "d", (n, 3))
    _arr(time, "time", (n,), optional=True)
    _arr(residual, "residual", (n, 3), optional=True)
    _arr(dist, "dist", (n, 3), optional=True)
    if out is None:
        rgb = torch.empty(n, 3, device=o.device)
        T = torch.empty(n, device=o.device)
        steps = torch.empty(n, dtype=torch.int32, device=o.device) if want_steps else None
    else:
        rgb, T, steps = out
    _arr(rgb, "rgb", (n, 3))
    _arr(T, "T", (n,), optional=True)
    _arr(steps, "steps", (n,), dtype=torch.int32, optional=True)
    _vt.vt_render_fwd(scene.handle, n, o.data_ptr(), d.data_ptr(), _ptr(time), params, rgb.data_ptr(), _ptr(T),
                      _ptr(steps), _ptr(residual), _ptr(dist), _stream())
    return rgb, T, steps


def render_bwd(scene: Scene, o, d, params, rgb, grad_rgb, time=None, out=None, need=(True, True, True),
               residual=None, tex_vd_out=None, dist=None, grad_dist=None):
    """Backward render: (grad_sites, grad_sigma, grad_tex); the gradient of the
    view-dependent texture (appearance 1) is written to `tex_vd_out` if given.
    With `grad_dist` ([n], dL/dL_dist per ray) the distortion loss is included;
    `dist` is then the forward's `dist` output."""
    dev = o.device
    n, N, R = o.shape[0], scene.n, scene.R
    if out is None:
        gs = torch.empty(N, 3, device=dev) if need[0] else None
        gsig = torch.empty(N, device=dev) if need[1] else None
        gt = torch.empty(N, R, R, 3, device=dev) if need[2] else None
    else:
        gs, gsig, gt = out
    grad_rgb = grad_rgb.contiguous()
    if grad_dist is not None:
        grad_dist = grad_dist.contiguous()
    for t, name, shape, opt in ((o, "o", (n, 3), False), (d, "d", (n, 3), False), (rgb, "rgb", (n, 3), False),
                                (grad_rgb, "grad_rgb", (n, 3), False), (time, "time", (n,), True),
                                (residual, "residual", (n, 3), True), (dist, "dist", (n, 3), True),
                                (grad_dist, "grad_dist", (n,), True), (gs, "grad_sites", (N, 3), True),
                                (gsig, "grad_sigma", (N,), True), (gt, "grad_tex", (N, R, R, 3), True),
                                (tex_vd_out, "tex_vd_out", (N, R, R, 3), True)):
        _arr(t, name, shape, optional=opt)
    _vt.vt_render_bwd(scene.handle, n, o.data_ptr(), d.data_ptr(), _ptr(time), params, rgb.data_ptr(),
                      _ptr(residual), _ptr(dist), grad_rgb.data_ptr(), _ptr(grad_dist), _ptr(gs),
                      _ptr(gsig), _ptr(gt), _ptr(tex_vd_out), _stream())
    return gs, gsig, gt


class _DeviceView:
    """A scene-owned device array seen through __cuda_array_interface__, so
    that torch can wrap it without a copy (the scene keeps ownership)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def render_bwd_scene_order(scene: Scene, o, d, params, rgb, grad_rgb, time=None, residual=None, dist=None,
                           grad_dist=None):
    """Backward render with the gradients left in the scene's cell order:
    returns (grad_cell [N,4] = (dL/ds, dL/dsigma), grad_tex [N,R,R,4] RGBA,
    grad_tex_vd [N,R,R,4] or None), torch views of scene-owned memory valid
    until the next backward call on the scene. Cell k is the user's site
    scene.permutation()[k]."""
    n, N, R = o.shape[0], scene.n, scene.R
    grad_rgb = grad_rgb.contiguous()
    for t, name, shape, opt in ((o, "o", (n, 3), False), (d, "d", (n, 3), False), (rgb, "rgb", (n, 3), False),
                                (grad_rgb, "grad_rgb", (n, 3), False), (time, "time", (n,), True),
                                (residual, "residual", (n, 3), True), (dist, "dist", (n, 3), True),
                                (grad_dist, "grad_dist", (n,), True)):
        _arr(t, name, shape, optional=opt)
    gc, gt, gv = _vt.vt_render_bwd_scene_order(scene.handle, n, o.data_ptr(), d.data_ptr(), _ptr(time), params,
                                               rgb.data_ptr(), _ptr(residual), _ptr(dist), grad_rgb.data_ptr(),
                                               _ptr(grad_dist), scene.has_tex_vd, _stream())
    dev = o.device
    cell = torch.as_tensor(_DeviceView(gc, (N, 4)), device=dev)
    tex = torch.as_tensor(_DeviceView(gt, (N, R, R, 4)), device=dev)
    vd = torch.as_tensor(_DeviceView(gv, (N, R, R, 4)), device=dev) if gv else None
    return cell, tex, vd


def trace_cells(scene: Scene, o, d, params, max_cells=512):
    n = o.shape[0]
    _arr(o, "o", (n, 3))
    _arr(d, "d", (n, 3))
    cells = torch.full((n, max_cells), -1, dtype=torch.int32, device=o.device)
    t_exit = torch.full((n, max_cells), float("nan"), device=o.device)
    n_cells = torch.empty(n, dtype=torch.int32, device=o.device)
    _vt.vt_trace_cells(scene.handle, n, o.data_ptr(), d.data_ptr(), params, max_cells, cells.data_ptr(),
                       t_exit.data_ptr(), n_cells.data_ptr(), _stream())
    return cells, t_exit, n_cells


def l2_loss(rgb, target):
    n = rgb.shape[0]
    target = target.contiguous()
    _arr(rgb, "rgb", (n, 3))
    _arr(target, "target", (n, 3))
    grad = torch.empty(n, 3, device=rgb.device)
    loss = torch.empty(1, device=rgb.device)
    _vt.vt_l2_loss(n, rgb.data_ptr(), target.data_ptr(), grad.data_ptr(), loss.data_ptr(), _stream())
    return loss, grad


def average_samples(rgb_rays, spp):
    if spp < 1 or rgb_rays.shape[0] % spp:
        raise ValueError("the ray count must be a multiple of spp >= 1")
    n_px = rgb_rays.shape[0] // spp
    _arr(rgb_rays, "rgb_rays", (n_px * spp, 3))
    out = torch.empty(n_px, 3, device=rgb_rays.device)
    _vt.vt_average_samples(n_px, spp, rgb_rays.data_ptr(), out.data_ptr(), _stream())
    return out


def sigma_from_rho(rho):
    """sigma = exp(rho) (Sec. 5.4) on the GPU."""
    rho = rho.contiguous()
    _arr(rho, "rho", tuple(rho.shape))
    out = torch.empty_like(rho)
    _vt.vt_sigma_from_rho(rho.numel(), rho.data_ptr(), out.data_ptr(), _stream())
    return out


def sigma_from_rho_bwd(sigma, grad_sigma):
    """dL/drho = dL/dsigma * sigma (Eq. 4) on the GPU."""
    sigma, grad_sigma = sigma.contiguous(), grad_sigma.contiguous()
    _arr(sigma, "sigma", tuple(sigma.shape))
    _arr(grad_sigma, "grad_sigma", tuple(sigma.shape))
    out = torch.empty_like(sigma)
    _vt.vt_sigma_from_rho_bwd(sigma.numel(), sigma.data_ptr(), grad_sigma.data_ptr(), out.data_ptr(), _stream())
    return out


class SigmaFromRho(torch.autograd.Function):
    """sigma = exp(rho) with the adjoint of Eq. 4."""

    @staticmethod
    def forward(ctx, rho):
        sigma = sigma_from_rho(rho)
        ctx.save_for_backward(sigma)
        return sigma

    @staticmethod
    def backward(ctx, grad_sigma):
        (sigma,) = ctx.saved_tensors
        return sigma_from_rho_bwd(sigma, grad_sigma)


def average_samples_bwd(grad_px, spp):
    grad_px = grad_px.contiguous()
    _arr(grad_px, "grad_px", (grad_px.shape[0], 3))
    out = torch.empty(grad_px.shape[0] * spp, 3, device=grad_px.device)
    _vt.vt_average_samples_bwd(grad_px.shape[0], spp, grad_px.data_ptr(), out.data_ptr(), _stream())
    return out


class VTRender(torch.autograd.Function):
    """Differentiable render of rays (o, d) through a Scene.

    The scene's sites / sigma / tex (/ tex_vd for appearance 1) tensors are
    passed so that autograd knows which leaves receive gradients; the Scene
    must hold their current values (call scene.update after changing them)."""

    @staticmethod
    def forward(ctx, sites, sigma, tex, tex_vd, o, d, scene, params, with_dist=False):
        res = torch.empty(o.shape[0], 3, device=o.device)
        dist = torch.empty(o.shape[0], 3, device=o.device) if with_dist else None
        rgb, _, _ = render_fwd(scene, o, d, params, want_steps=False, residual=res, dist=dist)
        ctx.scene, ctx.params, ctx.with_dist = scene, params, with_dist
        ctx.save_for_backward(o, d, rgb, res, dist)
        if with_dist:
            return rgb, dist[:, 0].contiguous()
        return rgb

    @staticmethod
    def backward(ctx, grad_rgb, grad_dist=None):
        o, d, rgb, res, dist = ctx.saved_tensors
        need = ctx.needs_input_grad[:3]
        gvd = None
        if ctx.needs_input_grad[3] and ctx.scene.has_tex_vd:
            gvd = torch.empty(ctx.scene.n, ctx.scene.R, ctx.scene.R, 3, device=o.device)
        gs, gsig, gt = render_bwd(ctx.scene, o, d, ctx.params, rgb, grad_rgb, need=need, residual=res,
                                  tex_vd_out=gvd, dist=dist, grad_dist=grad_dist if ctx.with_dist else None)
        return gs, gsig, gt, gvd, None, None, None, None, None


def render(sites, sigma, tex, o, d, scene: Scene, params, tex_vd=None, with_dist=False):
    """Differentiable render; returns rgb, or (rgb, L_dist per ray) with
    with_dist=True (distortion loss of Sec. 5.3, Eq. 2)."""
    return VTRender.apply(sites, sigma, tex, tex_vd, o, d, scene, params, with_dist)
