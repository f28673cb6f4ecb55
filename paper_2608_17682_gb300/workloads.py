"""Seeded synthetic inputs for the Voronoi ray-traversal renderer.

This module produces input data only: site positions, densities, textures,
the Delaunay adjacency (computed by scipy/Qhull on the host), camera poses and
jittered ray bundles. It holds none of the renderer's arithmetic and is the
one module that both the CUDA path's tests/benchmark and the CPU oracle draw
their inputs from.

The scene recipes stand in for the paper's Mip-NeRF 360 captures (Sec. 6.1),
which are not available here:

* ``tiny``: 2,000 sites uniform in the unit cube, sigma ~ lognormal(0, 1.5),
  4x4 RGB textures U[0,1], one 64x64 pinhole camera at distance 2.5 from the
  cube centre, rays clipped to the unit cube.
* ``surface``: a surface-concentrated cloud -- 70% of the sites within +-0.01
  of 40 seeded noisy spheres and planes, 20% uniform in [-1,1]^3, 10% on a
  background shell of radius U[4,8]. Surface cells get sigma ~ lognormal(3,1),
  the rest lognormal(-2,1). This mimics the bimodal, surface-concentrated
  opacity the paper trains towards (Sec. 5.3).

Seeds: scene 1000+k, camera jitter 2000+k, target image 3000+k, lens samples
4000+k for workload k.
"""
from __future__ import annotations

import hashlib
import math
import os
import tempfile
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# sites, densities, textures


def uniform_sites(n: int, rng: np.random.Generator, lo=0.0, hi=1.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)


def _sin_sum(rng, k=3):
    f = rng.integers(1, 7, size=k).astype(np.float64)
    g = rng.integers(1, 7, size=k).astype(np.float64)
    ph = rng.uniform(0, 2 * np.pi, size=k)
    ps = rng.uniform(0, 2 * np.pi, size=k)

    def h(a, b):
        out = np.zeros_like(a)
        for m in range(k):
            out += np.sin(f[m] * a + ph[m]) * np.sin(g[m] * b + ps[m])
        return out

    return h


def _sphere_points(n, rng):
    c = rng.uniform(-0.7, 0.7, size=3)
    r0 = rng.uniform(0.1, 0.4)
    noise = _sin_sum(rng)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    theta = np.arccos(np.clip(v[:, 2], -1, 1))
    phi = np.arctan2(v[:, 1], v[:, 0])
    r = r0 * (1.0 + 0.05 * noise(theta, phi))
    p = c + v * r[:, None]
    p += v * rng.uniform(-0.01, 0.01, size=(n, 1))
    return p


def _plane_points(n, rng):
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    off = rng.uniform(-0.5, 0.5)
    a = np.cross(nrm, [1.0, 0.0, 0.0] if abs(nrm[0]) < 0.9 else [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(nrm, a)
    noise = _sin_sum(rng)
    out = np.empty((0, 3))
    while len(out) < n:
        m = 2 * (n - len(out)) + 64
        uv = rng.uniform(-math.sqrt(3), math.sqrt(3), size=(m, 2))
        hgt = 0.03 * noise(2.0 * uv[:, 0], 2.0 * uv[:, 1])
        p = off * nrm + uv[:, :1] * a + uv[:, 1:] * b + (hgt[:, None] + rng.uniform(-0.01, 0.01, size=(m, 1))) * nrm
        p = p[np.all(np.abs(p) <= 1.0, axis=1)]
        out = np.concatenate([out, p])
    return out[:n]


def surface_sites(n: int, rng: np.random.Generator):
    """70% near 40 noisy surfaces, 20% uniform in [-1,1]^3, 10% shell r~U[4,8].

    Returns (sites float32 [n,3], is_surface bool [n])."""
    n_surf = int(round(0.7 * n))
    n_unif = int(round(0.2 * n))
    n_shell = n - n_surf - n_unif
    per = np.full(40, n_surf // 40)
    per[: n_surf - per.sum()] += 1
    parts = []
    for s in range(40):
        parts.append(_sphere_points(per[s], rng) if s < 20 else _plane_points(per[s], rng))
    surf = np.concatenate(parts)
    unif = rng.uniform(-1.0, 1.0, size=(n_unif, 3))
    v = rng.normal(size=(n_shell, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    shell = v * rng.uniform(4.0, 8.0, size=(n_shell, 1))
    pts = np.concatenate([surf, unif, shell]).astype(np.float32)
    is_surf = np.zeros(n, dtype=bool)
    is_surf[:n_surf] = True
    perm = rng.permutation(n)
    return np.ascontiguousarray(pts[perm]), is_surf[perm]


def dedupe(sites: np.ndarray) -> np.ndarray:
    """Drop exact duplicate FP32 sites (keeps the first occurrence, in order)."""
    _, first = np.unique(sites, axis=0, return_index=True)
    if len(first) == len(sites):
        return sites
    return np.ascontiguousarray(sites[np.sort(first)])


def textures(n: int, R: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(0.0, 1.0, size=(n, R, R, 3)).astype(np.float32)


# --------------------------------------------------------------------------
# Delaunay adjacency (host, scipy / Qhull)


def _cache_dir():
    return os.environ.get("VT_CACHE_DIR", os.path.join(tempfile.gettempdir(), "vt_delaunay_cache"))


def delaunay_csr(sites: np.ndarray, cache: bool = True):
    """CSR Delaunay adjacency of the sites: offsets int64 [n+1], indices int32.

    Qhull runs on the float64 promotion of the FP32 sites. Raises if Qhull
    left any site out of the triangulation (duplicates / coplanar points).
    Results for more than 100k sites are cached on local disk, keyed by a hash
    of the site array, so that a test run and a benchmark on the same machine
    triangulate a large scene once."""
    from scipy.spatial import Delaunay

    sites = np.ascontiguousarray(sites, dtype=np.float32)
    path = None
    if cache and len(sites) > 100_000:
        key = hashlib.sha1(sites.tobytes()).hexdigest()[:20]
        path = os.path.join(_cache_dir(), f"{key}_{len(sites)}.npz")
        if os.path.exists(path):
            try:
                z = np.load(path)
                return z["offsets"], z["indices"]
            except Exception:
                pass
    tri = Delaunay(sites.astype(np.float64))
    if len(tri.coplanar):
        raise ValueError(f"{len(tri.coplanar)} sites left out of the Delaunay triangulation")
    indptr, indices = tri.vertex_neighbor_vertices
    off, idx = indptr.astype(np.int64), indices.astype(np.int32)
    if path:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.npz"
            np.savez(tmp, offsets=off, indices=idx)
            os.replace(tmp, path)
        except OSError:
            pass
    return off, idx


# --------------------------------------------------------------------------
# cameras and rays


def orbit_eye(target, radius, az_deg, el_deg):
    az, el = math.radians(az_deg), math.radians(el_deg)
    v = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return np.asarray(target, dtype=np.float64) + radius * v


@dataclass
class Camera:
    """Camera description, mirrored by the C ABI's ``vt_camera``.

    kind: 0 pinhole, 1 equidistant fisheye, 2 rolling shutter, 3 thin lens,
    4 motion blur (lens_samples time samples per pixel)."""

    kind: int
    w: int
    h: int
    eye: tuple
    fwd: tuple
    up: tuple = (0.0, 0.0, 1.0)
    fov_y: float = math.radians(60.0)
    fisheye_fov: float = math.pi
    rs_velocity: tuple = (0.0, 0.0, 0.0)
    lens_radius: float = 0.0
    focus_dist: float = 1.0
    lens_samples: int = 1
    seed: int = 0

    @property
    def spp(self):
        return self.lens_samples if self.kind in (3, 4) else 1

    @property
    def n_rays(self):
        return self.w * self.h * self.spp


def look_at_camera(kind, w, h, eye, target, **kw) -> Camera:
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    return Camera(kind=kind, w=w, h=h, eye=tuple(float(x) for x in eye), fwd=tuple(float(x) for x in fwd), **kw)


def frustum_rays(eye, target, w, h, rng: np.random.Generator, fov_y=math.radians(60.0), up=(0.0, 0.0, 1.0),
                 origin_jitter=0.0):
    """Jittered ray bundle shaped like a camera's: one ray per pixel of a w x h
    grid, through a uniformly random point of that pixel on a frustum of
    vertical field of view fov_y, from eye (+ optional uniform origin jitter in
    a cube of half-size origin_jitter). Returns float32 o, d of shape [h*w, 3]
    in row-major pixel order; d is unit length."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    ty = math.tan(0.5 * fov_y)
    tx = ty * w / h
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    jx = rng.uniform(0.0, 1.0, size=(h, w))
    jy = rng.uniform(0.0, 1.0, size=(h, w))
    px = (2.0 * (xs + jx) / w - 1.0) * tx
    py = (1.0 - 2.0 * (ys + jy) / h) * ty
    d = f[None, None, :] + px[..., None] * r + py[..., None] * u
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    o = np.broadcast_to(eye, d.shape).copy()
    if origin_jitter > 0:
        o += rng.uniform(-origin_jitter, origin_jitter, size=o.shape)
    d = d.reshape(-1, 3).astype(np.float32)
    # re-normalise after rounding so |d| is 1 to FP32 precision
    d = (d / np.linalg.norm(d.astype(np.float64), axis=1, keepdims=True)).astype(np.float32)
    return np.ascontiguousarray(o.reshape(-1, 3).astype(np.float32)), np.ascontiguousarray(d)


def wide_rays(eye, target, n, rng: np.random.Generator, half_angle=math.radians(107.0), origin_radius=0.0,
              up=(0.0, 0.0, 1.0)):
    """n rays with directions uniform over the spherical cap of the given
    half-angle around eye->target, origins uniform on a disk of origin_radius
    around eye (perpendicular to the axis). Rays are ordered by a coarse
    (azimuth, polar) grid cell so that consecutive rays are close, and are
    returned as float32 o, d of shape [n,3] (d unit length)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    z = rng.uniform(math.cos(half_angle), 1.0, size=n)
    phi = rng.uniform(0.0, 2 * math.pi, size=n)
    st = np.sqrt(np.maximum(0.0, 1 - z * z))
    d = z[:, None] * f + (st * np.cos(phi))[:, None] * r + (st * np.sin(phi))[:, None] * u
    rad = origin_radius * np.sqrt(rng.uniform(0, 1, size=n))
    ang = rng.uniform(0, 2 * math.pi, size=n)
    o = eye + (rad * np.cos(ang))[:, None] * r + (rad * np.sin(ang))[:, None] * u
    order = np.lexsort((z, np.floor(phi / (2 * math.pi) * 64), np.floor((1 - z) * 32)))
    o, d = o[order], d[order]
    d = d.astype(np.float32)
    d = (d / np.linalg.norm(d.astype(np.float64), axis=1, keepdims=True)).astype(np.float32)
    return np.ascontiguousarray(o.astype(np.float32)), np.ascontiguousarray(d)


# --------------------------------------------------------------------------
# workloads


@dataclass
class Scene:
    sites: np.ndarray  # float32 [N,3]
    sigma: np.ndarray  # float32 [N]
    tex: np.ndarray  # float32 [N,R,R,3]
    offsets: np.ndarray  # int64 [N+1]
    indices: np.ndarray  # int32 [E]

    @property
    def n(self):
        return len(self.sites)

    @property
    def R(self):
        return self.tex.shape[1]


@dataclass
class Workload:
    name: str
    scene: Scene
    cameras: list
    params: dict = field(default_factory=dict)
    seed: int = 0


def make_scene(kind: str, n: int, R: int, seed: int) -> Scene:
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        sites = dedupe(uniform_sites(n, rng))
        sigma = np.exp(rng.normal(0.0, 1.5, size=len(sites))).astype(np.float32)
    elif kind == "surface":
        sites, is_surf = surface_sites(n, rng)
        keep_n = len(sites)
        sites = dedupe(sites)
        if len(sites) != keep_n:
            raise ValueError("duplicate sites in the surface cloud")
        sigma = np.where(is_surf, np.exp(rng.normal(3.0, 1.0, size=n)), np.exp(rng.normal(-2.0, 1.0, size=n)))
        sigma = sigma.astype(np.float32)
    else:
        raise ValueError(kind)
    tex = textures(len(sites), R, rng)
    off, idx = delaunay_csr(sites)
    return Scene(sites, sigma, tex, off, idx)


def crop_scene(sites_all, sigma_all, tex_all, lo, hi) -> Scene:
    """Sub-scene of the sites inside the box [lo,hi]^3, with its own Delaunay."""
    m = np.all((sites_all >= lo) & (sites_all <= hi), axis=1)
    s = np.ascontiguousarray(sites_all[m])
    off, idx = delaunay_csr(s)
    return Scene(s, np.ascontiguousarray(sigma_all[m]), np.ascontiguousarray(tex_all[m]), off, idx)


def surface_crop(n_max: int = 1000, side: float = 0.3, R: int = 8, seed: int = 1003) -> Scene:
    """About n_max sites of the surface-concentrated distribution (generated
    at 1M sites) inside a side^3 box centred on a surface site, with sigma by
    the same rule, fresh U[0,1] textures and their own Delaunay graph -- the
    small scene of the gradient finite-difference checks."""
    rng = np.random.default_rng(seed)
    pts, surf = surface_sites(1_000_000, rng)
    sigma = np.where(surf, np.exp(rng.normal(3.0, 1.0, size=len(pts))), np.exp(rng.normal(-2.0, 1.0, size=len(pts))))
    c = pts[np.nonzero(surf & (np.abs(pts).max(axis=1) < 0.5))[0][0]].astype(np.float64)
    m = np.all(np.abs(pts - c) <= side / 2, axis=1)
    idx = np.nonzero(m)[0]
    if len(idx) > n_max:
        idx = np.sort(rng.choice(idx, size=n_max, replace=False))
    sites = np.ascontiguousarray(pts[idx])
    off, ind = delaunay_csr(sites, cache=False)
    tex = textures(len(sites), R, rng)
    return Scene(sites, sigma[idx].astype(np.float32), tex, off, ind)


def default_params(**kw):
    p = dict(t_near=0.0, t_far=20.0, use_clip_box=False, clip_lo=(0.0, 0.0, 0.0), clip_hi=(1.0, 1.0, 1.0),
             T_eps=1e-4, skip_weight=0.0, bg=(1.0, 1.0, 1.0))
    p.update(kw)
    return p


WORKLOADS = {
    # name: (scene kind, sites, texture res, cameras spec)
    "tiny": ("uniform", 2_000, 4),
    "fwd500k": ("surface", 500_000, 4),
    "diff1m": ("surface", 1_000_000, 8),
    "prec3m": ("surface", 3_000_000, 8),
    "mixed3m": ("surface", 3_000_000, 8),
}
WORKLOAD_INDEX = {"tiny": 1, "fwd500k": 2, "diff1m": 3, "prec3m": 4, "mixed3m": 5}


def workload_cameras(name: str, w=1280, h=832):
    k = WORKLOAD_INDEX[name]
    if name == "tiny":
        c = np.array([0.5, 0.5, 0.5])
        return [look_at_camera(0, 64, 64, orbit_eye(c, 2.5, 30.0, 20.0), c)]
    o = np.zeros(3)
    if name == "fwd500k":
        return [look_at_camera(0, w, h, orbit_eye(o, 3.0, 30.0, 20.0), o)]
    if name in ("diff1m", "prec3m"):
        return [look_at_camera(0, w, h, orbit_eye(o, 3.0, az, 20.0), o) for az in (0.0, 90.0, 180.0, 270.0)]
    cams = []
    for q in range(16):
        eye = orbit_eye(o, 3.0, 22.5 * q, 20.0)
        if q < 4:
            cams.append(look_at_camera(0, w, h, eye, o))
        elif q < 8:
            cams.append(look_at_camera(1, w, h, eye, o, fisheye_fov=math.pi))
        elif q < 12:
            # linear motion of 0.05 units per frame along the camera's right axis
            f = -eye / np.linalg.norm(eye)
            r = np.cross(f, (0.0, 0.0, 1.0))
            r /= np.linalg.norm(r)
            cams.append(look_at_camera(2, w, h, eye, o, rs_velocity=tuple(float(x) for x in 0.05 * r)))
        else:
            cams.append(look_at_camera(3, w, h, eye, o, lens_radius=0.01, focus_dist=3.0, lens_samples=4,
                                       seed=4000 + k * 100 + q))
    return cams


def workload_params(name: str):
    if name == "tiny":
        return default_params(t_far=1e3, use_clip_box=True)
    return default_params()


def make_workload(name: str, n_sites: int | None = None, w=1280, h=832) -> Workload:
    kind, n, R = WORKLOADS[name]
    k = WORKLOAD_INDEX[name]
    sc = make_scene(kind, n if n_sites is None else n_sites, R, 1000 + k)
    return Workload(name, sc, workload_cameras(name, w, h), workload_params(name), seed=k)


def workload_rays(wl: Workload, jitter=True):
    """Jittered frustum rays for each pinhole-type camera of the workload,
    concatenated in camera order (seed 2000+k)."""
    rng = np.random.default_rng(2000 + wl.seed)
    os_, ds = [], []
    for c in wl.cameras:
        tgt = np.asarray(c.eye) + np.asarray(c.fwd)
        o, d = frustum_rays(c.eye, tgt, c.w, c.h, rng, fov_y=c.fov_y, up=c.up)
        os_.append(o)
        ds.append(d)
    return np.concatenate(os_), np.concatenate(ds)


def target_image(n_pixels: int, seed: int) -> np.ndarray:
    return np.random.default_rng(3000 + seed).uniform(0.0, 1.0, size=(n_pixels, 3)).astype(np.float32)
