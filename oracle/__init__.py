"""ctypes wrapper of the FP64 CPU oracle (``vt_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
bench.py's oracle leg (cpu_baseline with its accuracy check, and the reference
arm). The product library never imports it.
All inputs are promoted to float64 before the call (FP32 -> FP64 is exact).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vt_oracle.c")
_LIB = os.path.join(_HERE, "libvt_oracle.so")

F_NEAR_EDGE, F_NEAR_ORIGIN, F_NEAR_CLIP, F_T_AMBIG, F_SKIP_AMBIG, F_MAX_STEPS, F_BAD_RAY = 1, 2, 4, 8, 16, 32, 64
BAND_FLAGS = F_NEAR_EDGE | F_NEAR_ORIGIN | F_NEAR_CLIP | F_T_AMBIG | F_SKIP_AMBIG


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        # -ffp-contract=off: no fused multiply-adds, so the arithmetic is the
        # source's as written, on x86 and Arm alike
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-D_GNU_SOURCE", "-fPIC", "-shared", _SRC,
                               "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("t_near", C.c_double), ("t_far", C.c_double), ("use_clip_box", C.c_int32),
                ("clip_lo", C.c_double * 3), ("clip_hi", C.c_double * 3), ("T_eps", C.c_double),
                ("skip_weight", C.c_double), ("bg", C.c_double * 3), ("max_steps", C.c_int32),
                ("band_eps", C.c_double), ("appearance", C.c_int32)]


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sites", C.c_void_p), ("sigma", C.c_void_p), ("tex", C.c_void_p),
                ("R", C.c_int32), ("off", C.c_void_p), ("idx", C.c_void_p), ("tex_vd", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("w", C.c_int32), ("h", C.c_int32), ("eye", C.c_double * 3),
                ("fwd", C.c_double * 3), ("up", C.c_double * 3), ("fov_y", C.c_double),
                ("fisheye_fov", C.c_double), ("rs_velocity", C.c_double * 3), ("lens_radius", C.c_double),
                ("focus_dist", C.c_double), ("lens_samples", C.c_int32), ("seed", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # VT_ORACLE_LIB points the wrapper at another build of this source:
        # the mutation tests load deliberately broken copies through it
        _lib = C.CDLL(os.environ.get("VT_ORACLE_LIB") or build())
        L = _lib
        L.vto_oct.argtypes = [C.c_void_p, C.c_void_p]
        L.vto_bilinear_taps.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.vto_bilinear_taps.restype = None
        L.vto_nearest.argtypes = [C.c_int64, C.c_void_p, C.c_void_p]
        L.vto_nearest.restype = C.c_int64
        L.vto_render.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.vto_trace.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.vto_segments.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64] + [C.c_void_p] * 7
        L.vto_segments.restype = C.c_int64
        L.vto_render_bwd.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.vto_render_bwd_dist.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.vto_distortion.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int]
        L.vto_raygen.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.vto_camera_rays.argtypes = [C.c_void_p]
        L.vto_camera_rays.restype = C.c_int64
        L.vto_uniform.argtypes = [C.c_uint64, C.c_uint64]
        L.vto_uniform.restype = C.c_double
        L.vto_mix64.argtypes = [C.c_uint64]
        L.vto_mix64.restype = C.c_uint64
        L.vto_concentric.argtypes = [C.c_double, C.c_double, C.c_void_p]
        L.vto_concentric.restype = None
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleScene:
    """FP64 copy of a scene (sites, sigma, textures [N,R,R,3], CSR; optional
    view-dependent logit textures tex_vd for appearance mode 1)."""

    def __init__(self, sites, sigma, tex, offsets, indices, tex_vd=None):
        self.sites = _f64(sites).reshape(-1, 3)
        self.sigma = _f64(sigma).reshape(-1)
        self.tex = _f64(tex)
        self.R = int(self.tex.shape[1])
        self.off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.idx = np.ascontiguousarray(np.asarray(indices, dtype=np.int32))
        self.n = len(self.sites)
        self.tex_vd = None if tex_vd is None else _f64(tex_vd)
        self._s = _Scene(self.n, _ptr(self.sites), _ptr(self.sigma), _ptr(self.tex), self.R, _ptr(self.off),
                         _ptr(self.idx), _ptr(self.tex_vd))

    @classmethod
    def from_workload_scene(cls, sc):
        return cls(sc.sites, sc.sigma, sc.tex, sc.offsets, sc.indices)


def make_params(t_near=0.0, t_far=20.0, use_clip_box=False, clip_lo=(0, 0, 0), clip_hi=(1, 1, 1), T_eps=1e-4,
                skip_weight=0.0, bg=(1, 1, 1), max_steps=1 << 20, band_eps=1e-6, appearance=0):
    return _Params(t_near, t_far, int(bool(use_clip_box)), (C.c_double * 3)(*clip_lo), (C.c_double * 3)(*clip_hi),
                   T_eps, skip_weight, (C.c_double * 3)(*bg), max_steps, band_eps, int(appearance))


def _threads(n):
    return n if n else (os.cpu_count() or 1)


def render(sc: OracleScene, o, d, params=None, n_threads=0, **kw):
    """FP64 render: returns rgb [R,3], T [R], steps [R] int32, flags [R] int32."""
    p = params if params is not None else make_params(**kw)
    o, d = _f64(o).reshape(-1, 3), _f64(d).reshape(-1, 3)
    n = len(o)
    rgb = np.zeros((n, 3))
    T = np.zeros(n)
    steps = np.zeros(n, np.int32)
    flags = np.zeros(n, np.int32)
    st = lib().vto_render(C.byref(sc._s), n, _ptr(o), _ptr(d), C.byref(p), _ptr(rgb), _ptr(T), _ptr(steps),
                          _ptr(flags), _threads(n_threads))
    if st:
        raise RuntimeError(f"oracle render failed: {st}")
    return rgb, T, steps, flags


def trace(sc: OracleScene, o, d, max_cells=512, params=None, n_threads=0, **kw):
    """Visited cells (walk order), exit t per cell, cell counts, flags."""
    p = params if params is not None else make_params(**kw)
    o, d = _f64(o).reshape(-1, 3), _f64(d).reshape(-1, 3)
    n = len(o)
    cells = np.full((n, max_cells), -1, np.int32)
    t_out = np.full((n, max_cells), np.nan)
    n_cells = np.zeros(n, np.int32)
    flags = np.zeros(n, np.int32)
    st = lib().vto_trace(C.byref(sc._s), n, _ptr(o), _ptr(d), C.byref(p), max_cells, _ptr(cells), _ptr(t_out),
                         _ptr(n_cells), _ptr(flags), _threads(n_threads))
    if st:
        raise RuntimeError(f"oracle trace failed: {st}")
    return cells, t_out, n_cells, flags


def segments(sc: OracleScene, o, d, cap=4096, params=None, **kw):
    """Segment list of one ray as a dict of arrays."""
    p = params if params is not None else make_params(**kw)
    o, d = _f64(o).reshape(3), _f64(d).reshape(3)
    out = dict(cell=np.zeros(cap, np.int64), a=np.zeros(cap), b=np.zeros(cap), delta=np.zeros(cap),
               composited=np.zeros(cap, np.int32), T_before=np.zeros(cap), alpha=np.zeros(cap))
    n = lib().vto_segments(C.byref(sc._s), _ptr(o), _ptr(d), C.byref(p), cap, _ptr(out["cell"]), _ptr(out["a"]),
                           _ptr(out["b"]), _ptr(out["delta"]), _ptr(out["composited"]), _ptr(out["T_before"]),
                           _ptr(out["alpha"]))
    if n < 0:
        raise RuntimeError("oracle segments failed")
    m = min(n, cap)
    return {k: v[:m] for k, v in out.items()}


def render_bwd(sc: OracleScene, o, d, grad_rgb, params=None, n_threads=0, grad_dist=None, **kw):
    """FP64 gradients (sites [N,3], sigma [N], tex [N,R,R,3]) for dL/dC and,
    if grad_dist [R] is given, dL/dL_dist per ray (distortion loss, Eq. 2);
    a fourth array (tex_vd gradient) is returned when the scene has tex_vd."""
    p = params if params is not None else make_params(**kw)
    o, d, g = _f64(o).reshape(-1, 3), _f64(d).reshape(-1, 3), _f64(grad_rgb).reshape(-1, 3)
    gd = None if grad_dist is None else _f64(grad_dist).reshape(-1)
    gs = np.zeros((sc.n, 3))
    gsig = np.zeros(sc.n)
    gt = np.zeros(sc.tex.shape)
    gtv = None if sc.tex_vd is None else np.zeros(sc.tex.shape)
    st = lib().vto_render_bwd_dist(C.byref(sc._s), len(o), _ptr(o), _ptr(d), C.byref(p), _ptr(g), _ptr(gd), _ptr(gs),
                                   _ptr(gsig), _ptr(gt), _ptr(gtv), _threads(n_threads))
    if st:
        raise RuntimeError(f"oracle bwd failed: {st}")
    return (gs, gsig, gt) if gtv is None else (gs, gsig, gt, gtv)


def distortion(sc: OracleScene, o, d, params=None, n_threads=0, **kw):
    """Per-ray distortion loss L_dist [R] (Eq. 2) over the composited intervals."""
    p = params if params is not None else make_params(**kw)
    o, d = _f64(o).reshape(-1, 3), _f64(d).reshape(-1, 3)
    L = np.zeros(len(o))
    st = lib().vto_distortion(C.byref(sc._s), len(o), _ptr(o), _ptr(d), C.byref(p), _ptr(L), _threads(n_threads))
    if st:
        raise RuntimeError(f"oracle distortion failed: {st}")
    return L


def density_from_log(rho):
    """sigma = exp(rho) (Sec. 5.4, scale-invariant density)."""
    return np.exp(_f64(rho))


def density_log_bwd(sigma, grad_sigma):
    """dL/drho = dL/dsigma * sigma (Eq. 4)."""
    return _f64(grad_sigma) * _f64(sigma)


def octahedral(d):
    d = _f64(d).reshape(3)
    uv = np.zeros(2)
    if lib().vto_oct(_ptr(d), _ptr(uv)):
        raise ValueError("zero direction")
    return uv


def bilinear_taps(R, u, v):
    idx = np.zeros(4, np.int64)
    w = np.zeros(4)
    lib().vto_bilinear_taps(R, u, v, _ptr(idx), _ptr(w))
    return idx, w


def nearest(sites, q):
    s = _f64(sites).reshape(-1, 3)
    q = _f64(q).reshape(3)
    return int(lib().vto_nearest(len(s), _ptr(s), _ptr(q)))


def _camera_struct(cam):
    return _Camera(cam.kind, cam.w, cam.h, (C.c_double * 3)(*cam.eye), (C.c_double * 3)(*cam.fwd),
                   (C.c_double * 3)(*cam.up), cam.fov_y, cam.fisheye_fov, (C.c_double * 3)(*cam.rs_velocity),
                   cam.lens_radius, cam.focus_dist, cam.lens_samples, cam.seed)


def raygen(cam):
    """FP64 rays of one camera: o [n,3], d [n,3], time [n]."""
    cs = _camera_struct(cam)
    n = lib().vto_camera_rays(C.byref(cs))
    o = np.zeros((n, 3))
    d = np.zeros((n, 3))
    t = np.zeros(n)
    if lib().vto_raygen(C.byref(cs), _ptr(o), _ptr(d), _ptr(t)):
        raise ValueError("bad camera")
    return o, d, t


def uniform(seed, counter):
    return lib().vto_uniform(seed, counter)


def concentric(a, b):
    out = np.zeros(2)
    lib().vto_concentric(a, b, _ptr(out))
    return out


def mix64(z):
    return int(lib().vto_mix64(z))
