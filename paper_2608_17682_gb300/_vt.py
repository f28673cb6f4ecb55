"""ctypes binding of libvt.so: one Python function per C-ABI entry point, same
names, argument marshalling only (every step of the rendering path runs in
the library's CUDA kernels). Tensors are passed as raw device pointers and
the caller's current CUDA stream.

Importing this module loads libvt.so and raises if it is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("VT_LIB_PATH") or os.path.join(HERE, "libvt.so")

VT_OK, VT_ERR_INVALID_ARG, VT_ERR_CUDA, VT_ERR_OOM, VT_ERR_MAX_STEPS, VT_ERR_CAPACITY, VT_ERR_UNSUPPORTED = range(7)
VT_F32, VT_F16, VT_BF16 = 0, 1, 2
VT_CAM_PINHOLE, VT_CAM_FISHEYE_EQUIDIST, VT_CAM_ROLLING_SHUTTER, VT_CAM_THIN_LENS, VT_CAM_MOTION_BLUR = 0, 1, 2, 3, 4

# every symbol include/vt.h declares
EXPORTS = ["vt_render_params_default", "vt_scene_create", "vt_scene_update", "vt_scene_destroy", "vt_scene_info",
           "vt_scene_get_error", "vt_camera_n_rays", "vt_generate_rays", "vt_render_fwd", "vt_render_bwd",
           "vt_render_bwd_static", "vt_render_bwd_scene_order", "vt_scene_permutation", "vt_trace_cells", "vt_l2_loss", "vt_average_samples", "vt_average_samples_bwd", "vt_sigma_from_rho",
           "vt_sigma_from_rho_bwd", "vt_sample_rays", "vt_smooth_l1_loss", "vt_texture_regularizers", "vt_adam_step",
           "vt_adam_step_tex_scene_order", "vt_adam_step_cells_scene_order", "vt_kernel_launches", "vt_stream_read", "vt_status_str"]


class VTError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)}")


class vt_scene_desc(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("tex_res", C.c_int32), ("tex_dtype", C.c_int32), ("sites", C.c_void_p),
                ("sigma", C.c_void_p), ("tex", C.c_void_p), ("adj_offsets", C.c_void_p),
                ("adj_indices", C.c_void_p), ("flags", C.c_int32), ("tex_vd", C.c_void_p)]


VT_SCENE_KEEP_ORDER = 1
VT_SCENE_HALF_OFFSETS = 2


class vt_render_params(C.Structure):
    _fields_ = [("t_near", C.c_float), ("t_far", C.c_float), ("use_clip_box", C.c_int32),
                ("clip_lo", C.c_float * 3), ("clip_hi", C.c_float * 3), ("T_eps", C.c_float),
                ("skip_weight", C.c_float), ("bg", C.c_float * 3), ("img_w", C.c_int32), ("img_h", C.c_int32),
                ("n_images", C.c_int32), ("max_steps", C.c_int32), ("image_sizes", C.c_void_p),
                ("appearance", C.c_int32), ("walk_events", C.c_void_p * 2)]


class vt_camera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("w", C.c_int32), ("h", C.c_int32), ("eye", C.c_float * 3),
                ("fwd", C.c_float * 3), ("up", C.c_float * 3), ("fov_y", C.c_float), ("fisheye_fov", C.c_float),
                ("rs_velocity", C.c_float * 3), ("lens_radius", C.c_float), ("focus_dist", C.c_float),
                ("lens_samples", C.c_int32), ("seed", C.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(nvcc for sm_103a); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
    sig = {
        "vt_render_params_default": ([P], None),
        "vt_scene_create": ([P, P, P], C.c_int),
        "vt_scene_update": ([P, P, P, P, P, P], C.c_int),
        "vt_scene_destroy": ([P], None),
        "vt_scene_info": ([P, P, P, P, P], C.c_int),
        "vt_scene_get_error": ([P, P, P], C.c_int),
        "vt_camera_n_rays": ([P], I64),
        "vt_generate_rays": ([P, I32, P, P, P, P], C.c_int),
        "vt_render_fwd": ([P, I64, P, P, P, P, P, P, P, P, P, P], C.c_int),
        "vt_render_bwd": ([P, I64, P, P, P, P, P, P, P, P, P, P, P, P, P, P], C.c_int),
        "vt_render_bwd_static": ([P, I64, P, P, P, P, P, P, P, P, P, P], C.c_int),
        "vt_render_bwd_scene_order": ([P, I64, P, P, P, P, P, P, P, P, P, P, P, P, P], C.c_int),
        "vt_scene_permutation": ([P, P, P], C.c_int),
        "vt_trace_cells": ([P, I64, P, P, P, I32, P, P, P, P], C.c_int),
        "vt_l2_loss": ([I64, P, P, P, P, P], C.c_int),
        "vt_average_samples": ([I64, I32, P, P, P], C.c_int),
        "vt_average_samples_bwd": ([I64, I32, P, P, P], C.c_int),
        "vt_sigma_from_rho": ([I64, P, P, P], C.c_int),
        "vt_sigma_from_rho_bwd": ([I64, P, P, P, P], C.c_int),
        "vt_sample_rays": ([I64, P, P, P, I64, C.c_uint64, P, P, P, P, P], C.c_int),
        "vt_smooth_l1_loss": ([I64, P, P, C.c_float, P, P, P], C.c_int),
        "vt_texture_regularizers": ([I64, I32, P, P, C.c_float, C.c_float, P, P, P, P], C.c_int),
        "vt_adam_step": ([I64, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, I64, P], C.c_int),
        "vt_adam_step_tex_scene_order": ([I64, I32, P, P, P, P, P, I32, C.c_float, C.c_float, C.c_float, C.c_float,
                                          C.c_float, I64, P, P], C.c_int),
        "vt_adam_step_cells_scene_order": ([I64, P, P, P, P, P, P, P, P, P, C.c_float, C.c_float, C.c_float,
                                            C.c_float, C.c_float, I64, P], C.c_int),
        "vt_kernel_launches": ([], C.c_uint64),
        "vt_stream_read": ([P, I64, I32, P, P], C.c_int),
        "vt_status_str": ([C.c_int], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def status_str(s: int) -> str:
    return lib.vt_status_str(int(s)).decode()


def check(status: int, what: str):
    if status != VT_OK:
        raise VTError(status, what)


# ---------------------------------------------------------------- thin wrappers (same names as the C ABI)

def vt_render_params_default() -> vt_render_params:
    p = vt_render_params()
    lib.vt_render_params_default(C.byref(p))
    return p


def vt_scene_create(desc: vt_scene_desc, stream: int) -> int:
    h = C.c_void_p()
    check(lib.vt_scene_create(C.byref(desc), C.c_void_p(stream), C.byref(h)), "vt_scene_create")
    return h.value


def vt_scene_update(scene: int, sites: int, sigma: int, tex: int, tex_vd: int, stream: int):
    check(lib.vt_scene_update(C.c_void_p(scene), C.c_void_p(sites), C.c_void_p(sigma), C.c_void_p(tex),
                              C.c_void_p(tex_vd), C.c_void_p(stream)), "vt_scene_update")


def vt_scene_destroy(scene: int):
    lib.vt_scene_destroy(C.c_void_p(scene))


def vt_scene_info(scene: int):
    n, R, dt, E = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
    check(lib.vt_scene_info(C.c_void_p(scene), C.byref(n), C.byref(R), C.byref(dt), C.byref(E)), "vt_scene_info")
    return n.value, R.value, dt.value, E.value


def vt_scene_get_error(scene: int, stream: int):
    """Returns (status, n_fp64_rechecks); does not raise."""
    n = C.c_int64()
    st = lib.vt_scene_get_error(C.c_void_p(scene), C.c_void_p(stream), C.byref(n))
    return st, n.value


def vt_camera_n_rays(cam: vt_camera) -> int:
    return lib.vt_camera_n_rays(C.byref(cam))


def vt_generate_rays(cams, o: int, d: int, time: int, stream: int):
    arr = (vt_camera * len(cams))(*cams)
    check(lib.vt_generate_rays(arr, len(cams), C.c_void_p(o), C.c_void_p(d), C.c_void_p(time), C.c_void_p(stream)),
          "vt_generate_rays")


def vt_render_fwd(scene: int, n_rays: int, o: int, d: int, time: int, params: vt_render_params, rgb: int, T: int,
                  steps: int, rgb_residual: int, dist: int, stream: int):
    check(lib.vt_render_fwd(C.c_void_p(scene), n_rays, C.c_void_p(o), C.c_void_p(d), C.c_void_p(time),
                            C.byref(params), C.c_void_p(rgb), C.c_void_p(T), C.c_void_p(steps),
                            C.c_void_p(rgb_residual), C.c_void_p(dist), C.c_void_p(stream)), "vt_render_fwd")


def vt_render_bwd(scene: int, n_rays: int, o: int, d: int, time: int, params: vt_render_params, rgb: int,
                  rgb_residual: int, dist: int, grad_rgb: int, grad_dist: int, grad_sites: int, grad_sigma: int,
                  grad_tex: int, grad_tex_vd: int, stream: int):
    check(lib.vt_render_bwd(C.c_void_p(scene), n_rays, C.c_void_p(o), C.c_void_p(d), C.c_void_p(time),
                            C.byref(params), C.c_void_p(rgb), C.c_void_p(rgb_residual), C.c_void_p(dist),
                            C.c_void_p(grad_rgb), C.c_void_p(grad_dist), C.c_void_p(grad_sites),
                            C.c_void_p(grad_sigma), C.c_void_p(grad_tex), C.c_void_p(grad_tex_vd),
                            C.c_void_p(stream)), "vt_render_bwd")


def vt_render_bwd_static(scene: int, n_rays: int, o: int, d: int, time: int, params: vt_render_params, rgb: int,
                         grad_rgb: int, grad_sites: int, grad_sigma: int, grad_tex: int, stream: int):
    """Allocation-free backward (fixed 32 MiB library scratch); raises VTError
    with VT_ERR_CAPACITY for scenes that need more."""
    check(lib.vt_render_bwd_static(C.c_void_p(scene), n_rays, C.c_void_p(o), C.c_void_p(d), C.c_void_p(time),
                                   C.byref(params), C.c_void_p(rgb), C.c_void_p(grad_rgb), C.c_void_p(grad_sites),
                                   C.c_void_p(grad_sigma), C.c_void_p(grad_tex), C.c_void_p(stream)),
          "vt_render_bwd_static")


def vt_render_bwd_scene_order(scene: int, n_rays: int, o: int, d: int, time: int, params: vt_render_params,
                              rgb: int, rgb_residual: int, dist: int, grad_rgb: int, grad_dist: int, want_vd: bool,
                              stream: int):
    """Returns the device addresses (grad_cell, grad_tex, grad_tex_vd or 0) of
    the scene-owned, scene-order gradients."""
    gc, gt, gv = C.c_void_p(), C.c_void_p(), C.c_void_p()
    check(lib.vt_render_bwd_scene_order(C.c_void_p(scene), n_rays, C.c_void_p(o), C.c_void_p(d), C.c_void_p(time),
                                        C.byref(params), C.c_void_p(rgb), C.c_void_p(rgb_residual), C.c_void_p(dist),
                                        C.c_void_p(grad_rgb), C.c_void_p(grad_dist), C.byref(gc), C.byref(gt),
                                        C.byref(gv) if want_vd else None, C.c_void_p(stream)),
          "vt_render_bwd_scene_order")
    return gc.value or 0, gt.value or 0, gv.value or 0


def vt_scene_permutation(scene: int, perm: int, stream: int):
    check(lib.vt_scene_permutation(C.c_void_p(scene), C.c_void_p(perm), C.c_void_p(stream)), "vt_scene_permutation")


def vt_trace_cells(scene: int, n_rays: int, o: int, d: int, params: vt_render_params, max_cells: int, cells: int,
                   t_exit: int, n_cells: int, stream: int):
    check(lib.vt_trace_cells(C.c_void_p(scene), n_rays, C.c_void_p(o), C.c_void_p(d), C.byref(params), max_cells,
                             C.c_void_p(cells), C.c_void_p(t_exit), C.c_void_p(n_cells), C.c_void_p(stream)),
          "vt_trace_cells")


def vt_l2_loss(n: int, rgb: int, target: int, grad: int, loss: int, stream: int):
    check(lib.vt_l2_loss(n, C.c_void_p(rgb), C.c_void_p(target), C.c_void_p(grad), C.c_void_p(loss),
                         C.c_void_p(stream)), "vt_l2_loss")


def vt_average_samples(n_pixels: int, spp: int, rgb_rays: int, rgb_px: int, stream: int):
    check(lib.vt_average_samples(n_pixels, spp, C.c_void_p(rgb_rays), C.c_void_p(rgb_px), C.c_void_p(stream)),
          "vt_average_samples")


def vt_average_samples_bwd(n_pixels: int, spp: int, grad_px: int, grad_rays: int, stream: int):
    check(lib.vt_average_samples_bwd(n_pixels, spp, C.c_void_p(grad_px), C.c_void_p(grad_rays),
                                     C.c_void_p(stream)), "vt_average_samples_bwd")


def vt_sigma_from_rho(n: int, rho: int, sigma: int, stream: int):
    check(lib.vt_sigma_from_rho(n, C.c_void_p(rho), C.c_void_p(sigma), C.c_void_p(stream)), "vt_sigma_from_rho")


def vt_sigma_from_rho_bwd(n: int, sigma: int, grad_sigma: int, grad_rho: int, stream: int):
    check(lib.vt_sigma_from_rho_bwd(n, C.c_void_p(sigma), C.c_void_p(grad_sigma), C.c_void_p(grad_rho),
                                    C.c_void_p(stream)), "vt_sigma_from_rho_bwd")


def vt_sample_rays(n_pool: int, o_pool: int, d_pool: int, y_pool: int, n: int, seed: int, o: int, d: int, y: int,
                   idx: int, stream: int):
    check(lib.vt_sample_rays(n_pool, C.c_void_p(o_pool), C.c_void_p(d_pool), C.c_void_p(y_pool), n, seed,
                             C.c_void_p(o), C.c_void_p(d), C.c_void_p(y), C.c_void_p(idx), C.c_void_p(stream)),
          "vt_sample_rays")


def vt_smooth_l1_loss(n: int, rgb: int, target: int, beta: float, grad: int, loss: int, stream: int):
    check(lib.vt_smooth_l1_loss(n, C.c_void_p(rgb), C.c_void_p(target), beta, C.c_void_p(grad), C.c_void_p(loss),
                                C.c_void_p(stream)), "vt_smooth_l1_loss")


def vt_texture_regularizers(n_cells: int, tex_res: int, tex: int, tex_vd: int, lambda_vd: float, lambda_mean: float,
                            grad_tex: int, grad_tex_vd: int, loss: int, stream: int):
    check(lib.vt_texture_regularizers(n_cells, tex_res, C.c_void_p(tex), C.c_void_p(tex_vd), lambda_vd, lambda_mean,
                                      C.c_void_p(grad_tex), C.c_void_p(grad_tex_vd), C.c_void_p(loss),
                                      C.c_void_p(stream)), "vt_texture_regularizers")


def vt_adam_step(n: int, param: int, grad: int, m: int, v: int, lr: float, beta1: float, beta2: float, eps: float,
                 step: int, stream: int):
    check(lib.vt_adam_step(n, C.c_void_p(param), C.c_void_p(grad), C.c_void_p(m), C.c_void_p(v), lr, beta1, beta2,
                           eps, step, C.c_void_p(stream)), "vt_adam_step")


def vt_kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib.vt_kernel_launches())


def vt_stream_read(buf: int, nbytes: int, reps: int, sink: int, stream: int):
    check(lib.vt_stream_read(C.c_void_p(buf), nbytes, reps, C.c_void_p(sink), C.c_void_p(stream)), "vt_stream_read")


def vt_adam_step_tex_scene_order(n_cells: int, tex_res: int, perm: int, grad_tex_scene: int, tex: int, m: int, v: int,
                                 regularizer: int, lam: float, lr: float, beta1: float, beta2: float, eps: float,
                                 step: int, loss: int, stream: int):
    check(lib.vt_adam_step_tex_scene_order(n_cells, tex_res, C.c_void_p(perm), C.c_void_p(grad_tex_scene),
                                           C.c_void_p(tex), C.c_void_p(m), C.c_void_p(v), regularizer, lam, lr, beta1,
                                           beta2, eps, step, C.c_void_p(loss), C.c_void_p(stream)),
          "vt_adam_step_tex_scene_order")


def vt_adam_step_cells_scene_order(n_cells: int, perm: int, grad_cell_scene: int, sites: int, rho: int, sigma: int,
                                   m_sites: int, v_sites: int, m_rho: int, v_rho: int, lr_sites: float, lr_rho: float,
                                   beta1: float, beta2: float, eps: float, step: int, stream: int):
    check(lib.vt_adam_step_cells_scene_order(n_cells, C.c_void_p(perm), C.c_void_p(grad_cell_scene),
                                             C.c_void_p(sites), C.c_void_p(rho), C.c_void_p(sigma),
                                             C.c_void_p(m_sites), C.c_void_p(v_sites), C.c_void_p(m_rho),
                                             C.c_void_p(v_rho), lr_sites, lr_rho, beta1, beta2, eps, step,
                                             C.c_void_p(stream)),
          "vt_adam_step_cells_scene_order")
