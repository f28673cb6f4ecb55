"""Multi-view training loop on the GPU renderer (Sec. 5.3-5.5 and the
appendix's training settings).

Each iteration:
  sigma = exp(rho)                                  (Sec. 5.4)
  rays  = stratified sample of the training cameras' rays and pixels
  L     = SmoothL1(C, Y) + l_dist mean L_dist + l_vd L_vd + l_mean L_mean   (Eq. 5)
  Adam on sites, rho and both texture maps, with the learning-rate schedules
  of the appendix (cosine decays, density warm-up, site freeze, quadratic ramp
  of the view-dependent rate), and a Delaunay refresh every `refresh_every`
  iterations because the sites move (the appendix's periodic update).

Every array operation of the step runs in libvt kernels (apart from zeroing
the regulariser's loss scalar); torch holds the tensors. By default the
backward leaves the gradients in the scene's cell order and fused Adam steps
consume them (no user-order gradient arrays). The Delaunay refresh runs on the
host (scipy), outside the kernels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _vt, api
from . import workloads as W


@dataclass
class TrainConfig:
    iters: int = 20_000
    rays_per_iter: int = 1 << 20
    lr_sites: tuple = (2e-4, 5e-6)
    sites_frac: float = 0.9  # site positions follow the cosine schedule, then stay fixed
    lr_density: tuple = (1e-1, 1e-2)
    density_warmup_frac: float = 0.1
    lr_tex: tuple = (2e-2, 5e-4)
    vd_ramp_frac: float = 0.2  # quadratic ramp of the view-dependent rate (0: none)
    lambda_dist: float = 2e-3
    lambda_vd: float = 1e-2
    lambda_mean: float = 5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    smooth_l1_beta: float = 1e-2
    refresh_every: int = 500
    seed: int = 0
    # gradients left in the scene's cell order and consumed by fused Adam
    # steps (regularisers and Eq. 4 included); False: user-order gradients,
    # then separate regulariser, density-chain and Adam kernels
    scene_order_grads: bool = True


def cosine(lr0, lr1, t):
    """lr1 + (lr0 - lr1) (1 + cos(pi t)) / 2 for t in [0, 1]."""
    t = min(max(t, 0.0), 1.0)
    return lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * t))


def learning_rates(cfg: TrainConfig, it: int) -> dict:
    """Learning rates at iteration `it` (0-based) of cfg.iters."""
    n = max(1, cfg.iters)
    f = it / n
    s_end = cfg.sites_frac
    lr_s = cosine(*cfg.lr_sites, f / s_end) if f < s_end else 0.0
    w = cfg.density_warmup_frac
    if f < w:
        lr_d = cfg.lr_density[0] * (it + 1) / max(1.0, w * n)
    else:
        lr_d = cosine(*cfg.lr_density, (f - w) / max(1e-12, 1.0 - w))
    lr_t = cosine(*cfg.lr_tex, f)
    ramp = 1.0 if cfg.vd_ramp_frac <= 0 else min(1.0, f / cfg.vd_ramp_frac) ** 2
    return {"sites": lr_s, "rho": lr_d, "tex": lr_t, "tex_vd": lr_t * ramp}


class Trainer:
    """Optimises (sites, rho, tex, tex_vd) of a Voronoi scene against images.

    cams: list of workloads.Camera; images: [sum of camera rays, 3] target
    colours in the cameras' ray order (torch, on `device`)."""

    def __init__(self, sites, rho, tex, tex_vd, cams, images, render_params: dict, cfg: TrainConfig,
                 device="cuda", offsets=None, indices=None):
        self.cfg = cfg
        self.dev = torch.device(device)
        f = lambda x: torch.as_tensor(np.asarray(x, np.float32), device=self.dev).contiguous()  # noqa: E731
        self.p = {"sites": f(sites), "rho": f(rho), "tex": f(tex), "tex_vd": f(tex_vd)}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.sigma = api.sigma_from_rho(self.p["rho"])
        self.rparams = api.make_params(**render_params, appearance=1)
        self.n_pool = sum(c.n_rays for c in cams)
        self.o_pool, self.d_pool, _ = api.generate_rays(cams)
        self.y_pool = images.contiguous()
        assert self.y_pool.shape == (self.n_pool, 3)
        B = min(cfg.rays_per_iter, self.n_pool)
        self.B = B
        self.o = torch.empty(B, 3, device=self.dev)
        self.d = torch.empty(B, 3, device=self.dev)
        self.y = torch.empty(B, 3, device=self.dev)
        self.rgb = torch.empty(B, 3, device=self.dev)
        self.res = torch.empty(B, 3, device=self.dev)
        self.dist = torch.empty(B, 3, device=self.dev)
        self.grad_rgb = torch.empty(B, 3, device=self.dev)
        self.gdist = torch.full((B,), cfg.lambda_dist / B, device=self.dev)
        self.loss = torch.empty(1, device=self.dev)
        self.reg = torch.empty(1, device=self.dev)
        n, R = self.p["tex"].shape[0], self.p["tex"].shape[1]
        self.R = R
        if not cfg.scene_order_grads:  # user-order gradient arrays of the unfused path
            self.g = {"sites": torch.empty(n, 3, device=self.dev), "rho": torch.empty(n, device=self.dev),
                      "tex": torch.empty(n, R, R, 3, device=self.dev),
                      "tex_vd": torch.empty(n, R, R, 3, device=self.dev)}
            self.gsig = torch.empty(n, device=self.dev)
        self.it = 0
        self.refreshes = 0
        self.scene = None
        self._build_scene(offsets, indices)

    # ------------------------------------------------------------------ topology
    def _build_scene(self, offsets=None, indices=None):
        if offsets is None:
            offsets, indices = W.delaunay_csr(self.p["sites"].cpu().numpy(), cache=False)
        if self.scene is not None:
            self.scene.close()
        self.scene = api.Scene(self.p["sites"], self.sigma, self.p["tex"], offsets, indices, tex_dtype="f32",
                               device=self.dev, tex_vd=self.p["tex_vd"])
        self.perm = self.scene.permutation()  # scene cell k = user cell perm[k]
        self.n_edges = len(indices)

    def refresh(self):
        """Recompute the Delaunay graph of the current sites (host) and rebuild
        the scene; optimiser state is kept (it is in site order)."""
        self._build_scene()
        self.refreshes += 1

    # ------------------------------------------------------------------ one iteration
    def step(self, sync_loss=False):
        cfg, s = self.cfg, _vt
        st = api._stream()
        if self.it > 0 and cfg.refresh_every > 0 and self.it % cfg.refresh_every == 0:
            self.refresh()
        _vt.vt_sigma_from_rho(self.sigma.numel(), self.p["rho"].data_ptr(), self.sigma.data_ptr(), st)
        self.scene.update(sites=self.p["sites"], sigma=self.sigma, tex=self.p["tex"], tex_vd=self.p["tex_vd"])
        s.vt_sample_rays(self.n_pool, self.o_pool.data_ptr(), self.d_pool.data_ptr(), self.y_pool.data_ptr(), self.B,
                         cfg.seed * 1_000_003 + self.it, self.o.data_ptr(), self.d.data_ptr(), self.y.data_ptr(),
                         0, st)
        api.render_fwd(self.scene, self.o, self.d, self.rparams, out=(self.rgb, None, None), residual=self.res,
                       dist=self.dist)
        s.vt_smooth_l1_loss(self.B, self.rgb.data_ptr(), self.y.data_ptr(), cfg.smooth_l1_beta,
                            self.grad_rgb.data_ptr(), self.loss.data_ptr(), st)
        if cfg.scene_order_grads:
            self._fused_update(st)
            if sync_loss:
                return self.loss.item(), self.reg.item(), self.dist[:, 0].mean().item()
            return None
        api.render_bwd(self.scene, self.o, self.d, self.rparams, self.rgb, self.grad_rgb,
                       out=(self.g["sites"], self.gsig, self.g["tex"]), residual=self.res, dist=self.dist,
                       grad_dist=self.gdist, tex_vd_out=self.g["tex_vd"])
        n = self.p["tex"].shape[0]
        s.vt_texture_regularizers(n, self.R, self.p["tex"].data_ptr(), self.p["tex_vd"].data_ptr(), cfg.lambda_vd,
                                  cfg.lambda_mean, self.g["tex"].data_ptr(), self.g["tex_vd"].data_ptr(),
                                  self.reg.data_ptr(), st)
        s.vt_sigma_from_rho_bwd(n, self.sigma.data_ptr(), self.gsig.data_ptr(), self.g["rho"].data_ptr(), st)
        lrs = learning_rates(cfg, self.it)
        self.it += 1
        for k in ("sites", "rho", "tex", "tex_vd"):
            if lrs[k] == 0.0:
                continue
            s.vt_adam_step(self.p[k].numel(), self.p[k].data_ptr(), self.g[k].data_ptr(), self.m[k].data_ptr(),
                           self.v[k].data_ptr(), lrs[k], cfg.beta1, cfg.beta2, cfg.eps, self.it, st)
        if sync_loss:
            return self.loss.item(), self.reg.item(), self.dist[:, 0].mean().item()
        return None

    def _fused_update(self, st):
        """Backward with the gradients left in scene order, then one fused Adam
        step per texture map (with its regulariser) and one for sites and
        densities (with Eq. 4): no user-order gradient arrays are written."""
        cfg, s = self.cfg, _vt
        gc, gt, gv = api.render_bwd_scene_order(self.scene, self.o, self.d, self.rparams, self.rgb, self.grad_rgb,
                                                residual=self.res, dist=self.dist, grad_dist=self.gdist)
        lrs = learning_rates(cfg, self.it)
        self.it += 1
        n = self.p["tex"].shape[0]
        self.reg.zero_()  # the two texture steps add their regulariser losses
        for k, g, reg, lam in (("tex", gt, 0, cfg.lambda_mean), ("tex_vd", gv, 1, cfg.lambda_vd)):
            s.vt_adam_step_tex_scene_order(n, self.R, self.perm.data_ptr(), g.data_ptr(), self.p[k].data_ptr(),
                                           self.m[k].data_ptr(), self.v[k].data_ptr(), reg, lam, lrs[k], cfg.beta1,
                                           cfg.beta2, cfg.eps, self.it, self.reg.data_ptr(), st)
        s.vt_adam_step_cells_scene_order(n, self.perm.data_ptr(), gc.data_ptr(), self.p["sites"].data_ptr(),
                                         self.p["rho"].data_ptr(), self.sigma.data_ptr(), self.m["sites"].data_ptr(),
                                         self.v["sites"].data_ptr(), self.m["rho"].data_ptr(),
                                         self.v["rho"].data_ptr(), lrs["sites"], lrs["rho"], cfg.beta1, cfg.beta2,
                                         cfg.eps, self.it, st)

    def render(self, cams):
        """Render full images of `cams` with the current parameters."""
        _vt.vt_sigma_from_rho(self.sigma.numel(), self.p["rho"].data_ptr(), self.sigma.data_ptr(), api._stream())
        self.scene.update(sites=self.p["sites"], sigma=self.sigma, tex=self.p["tex"], tex_vd=self.p["tex_vd"])
        o, d, _ = api.generate_rays(cams)
        return api.render_fwd(self.scene, o, d, self.rparams)[0]


def synthetic_problem(n_sites=20_000, n_cams=8, w=96, h=64, tex_res=4, seed=0, device="cuda"):
    """A ground-truth Voronoi scene (surface-concentrated sites, paper
    appearance model with random logit textures), its renders from n_cams
    orbit cameras as the training images, and an initial guess: sites jittered
    by N(0, 1e-2) (the appendix's perturbation), a constant low density, grey
    view-independent texture (logit 0) and zero view-dependent texture.
    Returns (init dict, cams, images, render_params, gt dict)."""
    rng = np.random.default_rng(seed)
    sc = W.make_scene("surface", n_sites, tex_res, 7000 + seed)
    tvi = rng.normal(0.0, 1.5, size=sc.tex.shape).astype(np.float32)
    tvd = rng.normal(0.0, 0.3, size=sc.tex.shape).astype(np.float32)
    centre = np.zeros(3)
    cams = [W.look_at_camera(0, w, h, W.orbit_eye(centre, 3.0, 360.0 * k / n_cams, 15.0 + 10.0 * (k % 3)), centre)
            for k in range(n_cams)]
    rp = dict(W.default_params())
    gt = api.Scene(sc.sites, sc.sigma, tvi, sc.offsets, sc.indices, tex_dtype="f32", device=device, tex_vd=tvd)
    o, d, _ = api.generate_rays(cams)
    images = api.render_fwd(gt, o, d, api.make_params(**rp, appearance=1))[0]
    gt.close()
    init = {"sites": (sc.sites + rng.normal(0.0, 1e-2, size=sc.sites.shape)).astype(np.float32),
            "rho": np.full(sc.n, math.log(max(1e-3, float(np.median(sc.sigma)) * 0.1)), np.float32),
            "tex": np.zeros_like(tvi), "tex_vd": np.zeros_like(tvd)}
    return init, cams, images, rp, {"sites": sc.sites, "sigma": sc.sigma, "tex": tvi, "tex_vd": tvd}
