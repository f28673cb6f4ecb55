"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Bars: cell sequences bit-exact for rays outside the degenerate band (the
oracle flags rays that pass within 1e-6 of another face, start within 1e-6
of a face, cross near t_near'/t_far', or sit within 1e-4 relative of the
T / skip thresholds); images within 1e-4 max abs per channel (FP32 textures);
gradients within |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max|g_ref|).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
import parity_log  # noqa: E402
from paper_2608_17682_gb300 import workloads as W  # noqa: E402
from paper_2608_17682_gb300 import api  # noqa: E402

DEV = "cuda"
IMG_TOL = 1e-4
GRAD_REL = 1e-3


def gpu_params(p, **kw):
    q = dict(p)
    q.update(kw)
    return api.make_params(**q)


def oracle_params(p, **kw):
    q = {k: v for k, v in p.items() if k not in ("img_w", "img_h", "n_images", "max_steps")}
    q.update({k: v for k, v in kw.items() if k not in ("img_w", "img_h", "n_images")})
    return O.make_params(**q)


def to_dev(*a):
    return [torch.as_tensor(x, device=DEV).contiguous() for x in a]


def seeded(*shape, seed, normal=True):
    """Seeded random FP32 tensor on the device, drawn on the CPU so that it is
    the same on every machine."""
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(*shape, generator=g) if normal else torch.rand(*shape, generator=g)
    return x.to(DEV)


def fwd_res(scene, to, td, P):
    """Forward render that also returns the colour residual for the backward."""
    res = torch.empty(to.shape[0], 3, device=DEV)
    rgb = api.render_fwd(scene, to, td, P, residual=res)[0]
    return rgb, res


def compare_sequences(gc, gn, oc, on, flags, name=None):
    """Cell sequences equal for every unflagged ray; returns (#checked,
    #flagged-mismatch). With `name`, the counts go to the run's parity report."""
    ok = (flags & O.BAND_FLAGS) == 0
    same = (gn == on) & np.all(gc == oc, axis=1)
    bad = ok & ~same
    n_ok, n_band_diff = int(ok.sum()), int((~ok & ~same).sum())
    if name:
        parity_log.record(name, rays=len(flags), band=int((~ok).sum()), band_seq_mismatch=n_band_diff,
                          unflagged_seq_mismatch=int(bad.sum()))
    assert not bad.any(), f"{bad.sum()} unflagged rays differ, first {np.nonzero(bad)[0][:5]}"
    return n_ok, n_band_diff


def image_report(name, rgb, orgb, flags):
    """Image error against the oracle inside and outside the degenerate band
    (reported; the bars are asserted by the caller)."""
    ok = (flags & O.BAND_FLAGS) == 0
    err = np.abs(np.asarray(rgb, np.float64) - orgb)
    parity_log.record(name, rays=len(flags), band=int((~ok).sum()),
                      max_err=float(err[ok].max()) if ok.any() else 0.0,
                      max_err_band=float(err[~ok].max()) if (~ok).any() else 0.0,
                      rmse=float(np.sqrt(np.mean(err[ok] ** 2))) if ok.any() else 0.0)


def grad_close(g, ref, name):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = 1e-3 * np.abs(ref).max()
    tol = GRAD_REL * np.maximum(np.abs(ref), floor)
    err = np.abs(g - ref)
    bad = err > tol
    if bad.any():
        rel = err / np.maximum(np.abs(ref), floor)
        worst = np.argsort(rel, axis=None)[::-1][:5]
        detail = "; ".join(f"idx {np.unravel_index(i, ref.shape)} ref {ref.flat[i]:.6g} got {g.flat[i]:.6g}"
                           for i in worst)
        raise AssertionError(f"{name}: {bad.sum()} / {bad.size} entries off; worst rel {rel.max():.3g}; "
                             f"max|ref| {np.abs(ref).max():.4g}; {detail}")


# ---------------------------------------------------------------- fixtures

@pytest.fixture(scope="module")
def tiny():
    wl = W.make_workload("tiny")
    o, d = W.workload_rays(wl)
    return wl, O.OracleScene.from_workload_scene(wl.scene), o, d


@pytest.fixture(scope="module")
def medium():
    """50k-site surface-concentrated scene (several hundred tiles, ragged image)."""
    sc = W.make_scene("surface", 50_000, 8, 77)
    cams = [W.look_at_camera(0, 203, 121, W.orbit_eye(np.zeros(3), 3.0, az, 20.0), np.zeros(3))
            for az in (30.0, 210.0)]
    rng = np.random.default_rng(78)
    os_, ds = [], []
    for c in cams:
        o, d = W.frustum_rays(c.eye, np.zeros(3), c.w, c.h, rng)
        os_.append(o)
        ds.append(d)
    return sc, O.OracleScene.from_workload_scene(sc), np.concatenate(os_), np.concatenate(ds), cams


# ---------------------------------------------------------------- forward

@pytest.mark.parametrize("layout", ["image", "1d"])
def test_tiny_forward_parity(tiny, layout):
    wl, osc, o, d = tiny
    scene = api.Scene.from_workload(wl.scene)
    img = dict(img_w=64, img_h=64, n_images=1) if layout == "image" else {}
    P = gpu_params(wl.params, **img)
    to, td = to_dev(o, d)
    rgb, T, steps = api.render_fwd(scene, to, td, P)
    cells, t_exit, n_cells = api.trace_cells(scene, to, td, P, max_cells=256)
    assert scene.get_error()[0] == 0
    orgb, oT, osteps, flags = O.render(osc, o, d, params=oracle_params(wl.params))
    oc, ot, on, _ = O.trace(osc, o, d, max_cells=256, params=oracle_params(wl.params))
    ok = (flags & O.BAND_FLAGS) == 0
    assert ok.mean() > 0.95
    compare_sequences(cells.cpu().numpy(), n_cells.cpu().numpy(), oc, on, flags, name=f"tiny forward ({layout})")
    image_report(f"tiny forward image ({layout})", rgb.cpu().numpy(), orgb, flags)
    assert np.array_equal(steps.cpu().numpy()[ok], osteps[ok])
    assert np.abs(rgb.cpu().numpy()[ok] - orgb[ok]).max() <= IMG_TOL
    assert np.abs(T.cpu().numpy()[ok] - oT[ok]).max() <= IMG_TOL
    te = t_exit.cpu().numpy()
    m = np.isfinite(ot) & ok[:, None] & (np.arange(256)[None] < on[:, None])
    assert np.abs(te[m] - ot[m]).max() <= 1e-5 * max(1.0, np.abs(ot[m]).max())


def test_medium_forward_parity_ragged_tiles(medium):
    sc, osc, o, d, cams = medium
    scene = api.Scene.from_workload(sc)
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2)
    to, td = to_dev(o, d)
    rgb, T, steps = api.render_fwd(scene, to, td, P)
    cells, _, n_cells = api.trace_cells(scene, to, td, P, max_cells=400)
    assert scene.get_error()[0] == 0
    orgb, oT, osteps, flags = O.render(osc, o, d, params=oracle_params(base))
    oc, _, on, _ = O.trace(osc, o, d, max_cells=400, params=oracle_params(base))
    n_ok, n_flag_diff = compare_sequences(cells.cpu().numpy(), n_cells.cpu().numpy(), oc, on, flags,
                                          name="50k-site forward, ragged tiles")
    image_report("50k-site forward image", rgb.cpu().numpy(), orgb, flags)
    ok = (flags & O.BAND_FLAGS) == 0
    assert n_ok > 0.95 * len(o)
    assert np.abs(rgb.cpu().numpy()[ok] - orgb[ok]).max() <= IMG_TOL
    assert np.array_equal(steps.cpu().numpy()[ok], osteps[ok])


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_half_precision_textures(medium, dtype):
    sc, osc, o, d, cams = medium
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2)
    scene = api.Scene.from_workload(sc, tex_dtype=dtype)
    to, td = to_dev(o, d)
    rgb = api.render_fwd(scene, to, td, P)[0].cpu().numpy()
    # (ii) oracle on the dequantised textures: kernel error only
    tq = torch.as_tensor(sc.tex).to(torch.float16 if dtype == "f16" else torch.bfloat16).float().numpy()
    osq = O.OracleScene(sc.sites, sc.sigma, tq, sc.offsets, sc.indices)
    orgb_q, _, _, flags = O.render(osq, o, d, params=oracle_params(base))
    ok = (flags & O.BAND_FLAGS) == 0
    image_report(f"50k-site {dtype} textures vs dequantised", rgb, orgb_q, flags)
    assert np.abs(rgb[ok] - orgb_q[ok]).max() <= IMG_TOL
    # (i) oracle on the FP32 textures: total error, RMSE <= 2e-3
    orgb, _, _, _ = O.render(osc, o, d, params=oracle_params(base))
    image_report(f"50k-site {dtype} textures vs FP32 textures", rgb, orgb, flags)
    rmse = math.sqrt(np.mean((rgb[ok] - orgb[ok]) ** 2))
    assert rmse <= 2e-3, rmse


def test_exactly_representable_f16_texture_is_exact(tiny):
    wl, osc, o, d = tiny
    sc = wl.scene
    tex = np.round(sc.tex * 16) / 16  # k/16 values are exact in FP16 and BF16
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1)
    to, td = to_dev(o, d)
    a = api.render_fwd(api.Scene(sc.sites, sc.sigma, tex, sc.offsets, sc.indices, tex_dtype="f32"), to, td, P)[0]
    b = api.render_fwd(api.Scene(sc.sites, sc.sigma, tex, sc.offsets, sc.indices, tex_dtype="f16"), to, td, P)[0]
    assert torch.equal(a, b)


def test_skip_weight_rule(tiny):
    wl, osc, o, d = tiny
    scene = api.Scene.from_workload(wl.scene)
    P = gpu_params(wl.params, skip_weight=1e-2, img_w=64, img_h=64, n_images=1)
    to, td = to_dev(o, d)
    rgb = api.render_fwd(scene, to, td, P)[0].cpu().numpy()
    orgb, _, _, flags = O.render(osc, o, d, params=oracle_params(wl.params, skip_weight=1e-2))
    ok = (flags & O.BAND_FLAGS) == 0
    assert np.abs(rgb[ok] - orgb[ok]).max() <= IMG_TOL


# ---------------------------------------------------------------- backward

def test_tiny_backward_parity(tiny):
    wl, osc, o, d = tiny
    sc = wl.scene
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1)
    _, _, _, flags = O.render(osc, o, d, params=oracle_params(wl.params))
    ok = (flags & O.BAND_FLAGS) == 0
    Y = W.target_image(len(o), 1)
    g = np.random.default_rng(5).normal(size=(len(o), 3)) * ok[:, None]  # flagged rays carry no gradient
    scene = api.Scene.from_workload(sc)
    to, td, tg = to_dev(o, d, g.astype(np.float32))
    rgb, res = fwd_res(scene, to, td, P)
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, tg, residual=res)
    assert scene.get_error()[0] == 0
    ogs, ogsig, ogt = O.render_bwd(osc, o, d, g.astype(np.float32).astype(np.float64),
                                   params=oracle_params(wl.params))
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gt.cpu().numpy(), ogt, "tex")
    grad_close(gs.cpu().numpy(), ogs, "sites")
    del Y


def test_medium_backward_parity(medium):
    sc, osc, o, d, cams = medium
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2)
    _, _, _, flags = O.render(osc, o, d, params=oracle_params(base))
    ok = (flags & O.BAND_FLAGS) == 0
    g = (np.random.default_rng(6).normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    scene = api.Scene.from_workload(sc)
    to, td, tg = to_dev(o, d, g)
    rgb, res = fwd_res(scene, to, td, P)
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, tg, residual=res)
    ogs, ogsig, ogt = O.render_bwd(osc, o, d, g.astype(np.float64), params=oracle_params(base))
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gt.cpu().numpy(), ogt, "tex")
    grad_close(gs.cpu().numpy(), ogs, "sites")


def test_chunked_gradients_sum(medium):
    """Rays split into chunks (one per data-parallel replica): the sum of the
    chunk gradients equals the gradient of all rays at once."""
    sc, osc, o, d, cams = medium
    P1 = gpu_params(W.default_params())
    scene = api.Scene.from_workload(sc)
    to, td = to_dev(o, d)
    g = seeded(len(o), 3, seed=101)
    rgb = api.render_fwd(scene, to, td, P1)[0]
    full = api.render_bwd(scene, to, td, P1, rgb, g)
    acc = [torch.zeros_like(x) for x in full]
    for sl in (slice(0, 9000), slice(9000, 30000), slice(30000, len(o))):
        part = api.render_bwd(scene, to[sl].contiguous(), td[sl].contiguous(), P1, rgb[sl].contiguous(),
                              g[sl].contiguous())
        for a, p in zip(acc, part):
            a += p
    for a, f in zip(acc, full):
        scale = f.abs().max().item()
        assert (a - f).abs().max().item() <= 1e-4 * scale


def test_autograd_function(tiny):
    wl, osc, o, d = tiny
    sc = wl.scene
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1)
    scene = api.Scene.from_workload(sc)
    sites = torch.tensor(sc.sites, device=DEV, requires_grad=True)
    sigma = torch.tensor(sc.sigma, device=DEV, requires_grad=True)
    tex = torch.tensor(sc.tex, device=DEV, requires_grad=True)
    to, td = to_dev(o, d)
    Y = torch.as_tensor(W.target_image(len(o), 1), device=DEV)
    rgb = api.render(sites, sigma, tex, to, td, scene, P)
    loss = ((rgb - Y) ** 2).mean()
    loss.backward()
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb.detach(), 2 * (rgb.detach() - Y) / rgb.numel())
    assert torch.allclose(sites.grad, gs, rtol=1e-5, atol=1e-9)
    assert torch.allclose(sigma.grad, gsig, rtol=1e-5, atol=1e-9)
    assert torch.allclose(tex.grad, gt, rtol=1e-5, atol=1e-9)


def test_l2_loss_kernel(tiny):
    wl, osc, o, d = tiny
    rgb = seeded(4096, 3, seed=102, normal=False)
    Y = seeded(4096, 3, seed=103, normal=False)
    loss, grad = api.l2_loss(rgb, Y)
    r64 = (rgb.double() - Y.double())
    assert abs(loss.item() - (r64 ** 2).mean().item()) < 1e-6
    assert torch.allclose(grad.double(), 2 * r64 / r64.numel(), rtol=1e-6, atol=1e-12)


# ---------------------------------------------------------------- ray generation

@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_raygen_parity(kind):
    eye = W.orbit_eye(np.zeros(3), 3.0, 67.5, 20.0)
    kw = {}
    if kind == 2:
        kw = dict(rs_velocity=(0.05, -0.02, 0.0))
    if kind == 3:
        kw = dict(lens_radius=0.01, focus_dist=3.0, lens_samples=4, seed=4242)
    if kind == 4:
        kw = dict(rs_velocity=(0.03, 0.01, -0.02), lens_samples=3, seed=99)
    cam = W.look_at_camera(kind, 130, 83, eye, np.zeros(3), **kw)
    o, d, t = api.generate_rays([cam, cam])
    oo, od, ot = O.raygen(cam)
    oo, od, ot = np.concatenate([oo, oo]), np.concatenate([od, od]), np.concatenate([ot, ot])
    assert np.abs(o.cpu().numpy() - oo).max() <= 4e-7 * 3.0
    assert np.abs(d.cpu().numpy() - od).max() <= 4e-6
    assert np.abs(t.cpu().numpy() - ot).max() <= 1e-7


def test_average_samples():
    x = seeded(40, 3, seed=104, normal=False)
    y = api.average_samples(x, 4)
    assert torch.allclose(y, x.view(10, 4, 3).mean(1), atol=1e-7)
    g = seeded(10, 3, seed=105, normal=False)
    gx = api.average_samples_bwd(g, 4)
    assert torch.allclose(gx, g.repeat_interleave(4, 0) / 4, atol=1e-7)


# ---------------------------------------------------------------- edge cases

def test_empty_and_missing_rays(tiny):
    wl, osc, o, d = tiny
    scene = api.Scene.from_workload(wl.scene)
    P = gpu_params(wl.params)
    e = torch.empty(0, 3, device=DEV)
    rgb, T, s = api.render_fwd(scene, e, e, P)
    assert rgb.shape == (0, 3)
    # rays pointing away from the clip box: background, T = 1, no steps
    o2 = torch.tensor([[2.0, 2.0, 2.0]] * 5, device=DEV)
    d2 = torch.tensor([[1.0, 0.0, 0.0]] * 5, device=DEV)
    rgb, T, s = api.render_fwd(scene, o2, d2, P)
    assert torch.all(rgb == 1) and torch.all(T == 1) and torch.all(s == 0)
    # their backward and an empty backward give exactly zero gradients
    for oo, dd, cc in ((o2, d2, rgb), (e, e, torch.empty(0, 3, device=DEV))):
        gs, gsig, gt = api.render_bwd(scene, oo, dd, P, cc, torch.ones_like(cc))
        assert scene.get_error()[0] == 0
        assert gs.abs().max().item() == 0 and gsig.abs().max().item() == 0 and gt.abs().max().item() == 0


def test_grazing_planes_take_the_fp64_recheck(tiny):
    """Rays nearly parallel to a bisector plane of the cell they start near
    (|n.d| from 1e-8 to 9e-7 of |n||d|, origins 1e-5 to 1e-4 off the plane):
    their exit decisions go through the FP64 recheck of grazing planes (the
    library counts the rechecks), and cells, steps and colours still match
    the oracle outside the degenerate band."""
    wl, osc, o_, d_ = tiny
    sc = wl.scene
    rng = np.random.default_rng(31)
    os_, ds = [], []
    for _ in range(3000):
        i = int(rng.integers(sc.n))
        nb = sc.indices[sc.offsets[i]:sc.offsets[i + 1]]
        j = int(rng.choice(nb))
        si, sj = sc.sites[i].astype(np.float64), sc.sites[j].astype(np.float64)
        nh = (sj - si) / np.linalg.norm(sj - si)
        t1 = np.cross(nh, rng.normal(size=3))
        t1 /= np.linalg.norm(t1)
        h = rng.choice([1e-5, 3e-5, 1e-4])
        eps = rng.choice([1e-8, 3e-7, 9e-7])
        os_.append(0.5 * (si + sj) - h * nh - 0.02 * t1)
        d = t1 + eps * nh
        ds.append(d / np.linalg.norm(d))
    o = np.asarray(os_, np.float32)
    d = np.asarray(ds, np.float32)
    scene = api.Scene.from_workload(sc)
    P = gpu_params(wl.params)
    to, td = to_dev(o, d)
    rgb, T, steps = api.render_fwd(scene, to, td, P)
    cells, _, n_cells = api.trace_cells(scene, to, td, P, max_cells=256)
    st, n_fp64 = scene.get_error()
    assert st == 0 and n_fp64 > 0
    op = oracle_params(wl.params)
    orgb, oT, osteps, flags = O.render(osc, o, d, params=op)
    oc, _, on, _ = O.trace(osc, o, d, max_cells=256, params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    assert ok.mean() > 0.5
    compare_sequences(cells.cpu().numpy(), n_cells.cpu().numpy(), oc, on, flags, name="grazing rays")
    image_report("grazing rays image", rgb.cpu().numpy(), orgb, flags)
    assert np.array_equal(steps.cpu().numpy()[ok], osteps[ok])
    assert np.abs(rgb.cpu().numpy()[ok] - orgb[ok]).max() <= IMG_TOL
    parity_log.record("grazing rays FP64 rechecks", rechecks=int(n_fp64))


def test_single_site_scene_closed_form():
    c = np.array([0.2, 0.5, 0.9], np.float32)
    tex = np.broadcast_to(c, (1, 4, 4, 3)).copy()
    scene = api.Scene(np.array([[0.1, 0.2, 0.3]], np.float32), np.array([1.7], np.float32), tex,
                      np.array([0, 0]), np.zeros(0, np.int32))
    rng = np.random.default_rng(3)
    o = rng.uniform(-2, 2, size=(64, 3)).astype(np.float32)
    d = rng.normal(size=(64, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    P = api.make_params(t_near=0.2, t_far=1.5, T_eps=0.0)
    rgb = api.render_fwd(scene, *to_dev(o, d), P)[0].cpu().numpy()
    L = 1.3
    ref = (1 - np.exp(-1.7 * L)) * c + np.exp(-1.7 * L)
    assert np.abs(rgb - ref).max() <= 1e-6


def test_max_steps_and_capacity_errors(tiny):
    wl, osc, o, d = tiny
    scene = api.Scene.from_workload(wl.scene)
    to, td = to_dev(o, d)
    api.render_fwd(scene, to, td, gpu_params(wl.params, max_steps=4))
    assert scene.get_error()[0] == api._vt.VT_ERR_MAX_STEPS
    api.trace_cells(scene, to, td, gpu_params(wl.params), max_cells=2)
    assert scene.get_error()[0] == api._vt.VT_ERR_CAPACITY
    api.render_fwd(scene, to, td, gpu_params(wl.params))
    assert scene.get_error()[0] == 0
    bad = td.clone()
    bad[7] = 0
    rgb = api.render_fwd(scene, to, bad, gpu_params(wl.params))[0]
    assert scene.get_error()[0] == api._vt.VT_ERR_INVALID_ARG
    assert torch.all(rgb[7] == 0)


def test_create_rejects_malformed_inputs():
    sc = W.make_scene("uniform", 300, 4, 9)
    good = dict(sites=sc.sites, sigma=sc.sigma, tex=sc.tex, adj_offsets=sc.offsets, adj_indices=sc.indices)
    api.Scene(**good).close()

    def rejects(**kw):
        args = dict(good)
        args.update(kw)
        with pytest.raises(api._vt.VTError) as e:
            api.Scene(**args)
        assert e.value.status == api._vt.VT_ERR_INVALID_ARG

    s = sc.sites.copy()
    s[5, 1] = np.nan
    rejects(sites=s)
    g = sc.sigma.copy()
    g[3] = -1
    rejects(sigma=g)
    idx = sc.indices.copy()
    idx[10] = 300  # out of range
    rejects(adj_indices=idx)
    idx = sc.indices.copy()
    row0 = idx[sc.offsets[0]:sc.offsets[1]]
    idx[sc.offsets[0]] = 0  # self loop in row 0
    rejects(adj_indices=idx)
    idx = sc.indices.copy()
    j = idx[sc.offsets[0]]
    idx[sc.offsets[0]] = [k for k in range(1, 300) if k not in row0][0]  # asymmetric
    rejects(adj_indices=idx)
    del j


def test_scene_update_matches_fresh_scene(tiny):
    wl, osc, o, d = tiny
    sc = wl.scene
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1)
    to, td = to_dev(o, d)
    scene = api.Scene.from_workload(sc)
    rng = np.random.default_rng(4)
    sites2 = (sc.sites + rng.normal(0, 1e-4, size=sc.sites.shape)).astype(np.float32)
    sig2 = (sc.sigma * 1.5).astype(np.float32)
    tex2 = rng.uniform(0, 1, size=sc.tex.shape).astype(np.float32)
    scene.update(sites2, sig2, tex2)
    a = api.render_fwd(scene, to, td, P)[0]
    fresh = api.Scene(sites2, sig2, tex2, sc.offsets, sc.indices)
    b = api.render_fwd(fresh, to, td, P)[0]
    assert torch.equal(a, b)


def test_wide_angle_moving_origin_rays(medium):
    """Rays shaped like the mixed-camera workload: directions up to 107 deg
    off-axis (fisheye corners) and origins spread over a 0.05 disk (lens /
    rolling-shutter motion), 1-D layout, uneven lengths."""
    sc, osc, o_, d_, cams = medium
    o, d = W.wide_rays(W.orbit_eye(np.zeros(3), 3.0, 100.0, 20.0), np.zeros(3), 20000,
                       np.random.default_rng(79), origin_radius=0.05)
    base = W.default_params()
    scene = api.Scene.from_workload(sc, tex_dtype="f16")
    to, td = to_dev(o, d)
    res = torch.empty(to.shape[0], 3, device=DEV)
    rgb, T, steps = api.render_fwd(scene, to, td, gpu_params(base), residual=res)
    cells, _, n_cells = api.trace_cells(scene, to, td, gpu_params(base), max_cells=400)
    assert scene.get_error()[0] == 0
    tq = torch.as_tensor(sc.tex).half().float().numpy()
    osq = O.OracleScene(sc.sites, sc.sigma, tq, sc.offsets, sc.indices)
    orgb, _, osteps, flags = O.render(osq, o, d, params=oracle_params(base))
    oc, _, on, _ = O.trace(osq, o, d, max_cells=400, params=oracle_params(base))
    compare_sequences(cells.cpu().numpy(), n_cells.cpu().numpy(), oc, on, flags, name="wide-angle moving origins")
    image_report("wide-angle moving origins image", rgb.cpu().numpy(), orgb, flags)
    ok = (flags & O.BAND_FLAGS) == 0
    assert np.abs(rgb.cpu().numpy()[ok] - orgb[ok]).max() <= IMG_TOL
    assert np.array_equal(steps.cpu().numpy()[ok], osteps[ok])
    g = (np.random.default_rng(80).normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    gs, gsig, gt = api.render_bwd(scene, to, td, gpu_params(base), rgb, torch.as_tensor(g, device=DEV), residual=res)
    ogs, ogsig, ogt = O.render_bwd(osq, o, d, g.astype(np.float64), params=oracle_params(base))
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gt.cpu().numpy(), ogt, "tex")
    grad_close(gs.cpu().numpy(), ogs, "sites")


def test_image_table_layout_matches_1d(medium):
    """Images of different sizes in one launch (image table, 4x8 tiles per
    image, one anchor per image) give the same per-ray results as 1-D order."""
    sc, osc, o_, d_, cams = medium
    base = W.default_params()
    sizes = [(64, 64), (203, 31), (40, 8), (13, 5)]
    rng = np.random.default_rng(81)
    os_, ds = [], []
    for k, (w, h) in enumerate(sizes):
        eye = W.orbit_eye(np.zeros(3), 3.0, 40.0 * k, 20.0)
        o, d = W.frustum_rays(eye, np.zeros(3), w, h, rng, origin_jitter=0.002 * k)
        os_.append(o)
        ds.append(d)
    to, td = to_dev(np.concatenate(os_), np.concatenate(ds))
    scene = api.Scene.from_workload(sc, tex_dtype="f16")
    a = api.render_fwd(scene, to, td, gpu_params(base, image_sizes=sizes))
    b = api.render_fwd(scene, to, td, gpu_params(base))
    assert scene.get_error()[0] == 0
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    g = seeded(to.shape[0], 3, seed=106)
    ga = api.render_bwd(scene, to, td, gpu_params(base, image_sizes=sizes), a[0], g)
    gb = api.render_bwd(scene, to, td, gpu_params(base), b[0], g)
    for x, y in zip(ga, gb):
        assert (x - y).abs().max().item() <= 1e-5 * max(1.0, y.abs().max().item())


def test_mixed_cameras_one_launch(medium):
    """Pinhole, fisheye, rolling-shutter, thin-lens and motion-blur views
    generated on the GPU and rendered in one launch; per-ray results equal a 1-D launch, and
    the 4-sample thin-lens pixels average correctly."""
    sc, osc, o_, d_, cams = medium
    o0 = np.zeros(3)
    mk = [W.look_at_camera(0, 48, 32, W.orbit_eye(o0, 3.0, 10, 20), o0),
          W.look_at_camera(1, 48, 32, W.orbit_eye(o0, 3.0, 100, 20), o0),
          W.look_at_camera(2, 48, 32, W.orbit_eye(o0, 3.0, 190, 20), o0, rs_velocity=(0.05, 0.0, 0.0)),
          W.look_at_camera(3, 48, 32, W.orbit_eye(o0, 3.0, 280, 20), o0, lens_radius=0.01, focus_dist=3.0,
                           lens_samples=4, seed=7),
          W.look_at_camera(4, 48, 32, W.orbit_eye(o0, 3.0, 330, 20), o0, rs_velocity=(0.0, 0.02, 0.01),
                           lens_samples=2, seed=8)]
    o, d, t = api.generate_rays(mk)
    sizes = [(48 * c.spp, 32) for c in mk]
    base = W.default_params()
    scene = api.Scene.from_workload(sc)
    a = api.render_fwd(scene, o, d, gpu_params(base, image_sizes=sizes), time=t)
    b = api.render_fwd(scene, o, d, gpu_params(base))
    assert scene.get_error()[0] == 0
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2])
    n_px = 48 * 32
    lens = a[0][3 * n_px:7 * n_px]
    px = api.average_samples(lens.contiguous(), 4)
    assert torch.allclose(px, lens.view(n_px, 4, 3).mean(1), atol=1e-6)


def mixed_camera_rays(cams):
    """FP32 rays of each camera from the oracle's ray generation (its own
    pins fix it; the GPU's ray generation is compared with it separately), so
    that both sides walk the same input rays."""
    os_, ds = [], []
    for c in cams:
        o, d, _ = O.raygen(c)
        os_.append(o.astype(np.float32))
        ds.append(d.astype(np.float32))
    return np.concatenate(os_), np.concatenate(ds)


def mixed_launch_against_oracle(name, sc, cams, sel_px, seed, tex_dtype="f16"):
    """The launch path of the mixed-camera workload against the oracle: all
    cameras' rays in one image-table launch (one anchor per image; thin-lens,
    rolling-shutter and motion-blur origins reach their start cells by
    descent from the anchor), lens/time samples averaged per pixel by
    vt_average_samples, and the backward through vt_average_samples_bwd.
    `sel_px[k]` are the pixels of camera k the oracle computes: cells (exact
    outside the band), colours, pixel averages, gradients."""
    o, d = mixed_camera_rays(cams)
    sizes = [(c.w * c.spp, c.h) for c in cams]
    base = W.default_params()
    P = gpu_params(base, image_sizes=sizes)
    scene = api.Scene.from_workload(sc, tex_dtype=tex_dtype)
    to, td = to_dev(o, d)
    res = torch.empty(len(o), 3, device=DEV)
    rgb, T, steps = api.render_fwd(scene, to, td, P, residual=res)
    assert scene.get_error()[0] == 0
    # the sampled rays: every lens / time sample of each selected pixel
    first = np.cumsum([0] + [c.n_rays for c in cams])
    sel = np.concatenate([first[k] + (np.asarray(px)[:, None] * c.spp + np.arange(c.spp)[None]).ravel()
                          for k, (c, px) in enumerate(zip(cams, sel_px))])
    tq = sc.tex if tex_dtype == "f32" else torch.as_tensor(sc.tex).half().float().numpy()
    osq = O.OracleScene(sc.sites, sc.sigma, tq, sc.offsets, sc.indices)
    op = oracle_params(base)
    orgb, oT, osteps, flags = O.render(osq, o[sel], d[sel], params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    assert ok.mean() > 0.95
    g_rgb = rgb.cpu().numpy()[sel]
    image_report(name + " image", g_rgb, orgb, flags)
    assert np.abs(g_rgb[ok] - orgb[ok]).max() <= IMG_TOL
    assert np.abs(T.cpu().numpy()[sel][ok] - oT[ok]).max() <= IMG_TOL
    assert np.array_equal(steps.cpu().numpy()[sel][ok], osteps[ok])
    cells, _, n_cells = api.trace_cells(scene, to[sel].contiguous(), td[sel].contiguous(), gpu_params(base),
                                        max_cells=512)
    oc, _, on, _ = O.trace(osq, o[sel], d[sel], max_cells=512, params=op)
    compare_sequences(cells.cpu().numpy(), n_cells.cpu().numpy(), oc, on, flags, name=name)
    # pixel averages of the multi-sample cameras; a pixel is checked when all
    # its samples are outside the band
    rng = np.random.default_rng(seed)
    g_px_all, g_ray_o = [], np.zeros((len(sel), 3))
    pos = 0
    for k, (c, px) in enumerate(zip(cams, sel_px)):
        m = len(px) * c.spp
        ok_px = ok[pos:pos + m].reshape(len(px), c.spp).all(1)
        g_px = np.zeros((c.n_rays // c.spp, 3), np.float32)
        g_px[np.asarray(px)[ok_px]] = rng.normal(size=(ok_px.sum(), 3))
        if c.spp > 1:
            blk = rgb[first[k]:first[k + 1]].contiguous()
            avg = api.average_samples(blk, c.spp).cpu().numpy()[np.asarray(px)]
            o_avg = orgb[pos:pos + m].reshape(len(px), c.spp, 3).mean(1)
            assert np.abs(avg[ok_px] - o_avg[ok_px]).max() <= IMG_TOL
        # dL/d(sample colour) = dL/d(pixel) / spp: the adjoint of the mean
        g_ray_o[pos:pos + m] = np.repeat(g_px[np.asarray(px)].astype(np.float64), c.spp, axis=0) / c.spp
        g_px_all.append(torch.as_tensor(g_px, device=DEV))
        pos += m
    g_dev = torch.cat([api.average_samples_bwd(gp, c.spp) if c.spp > 1 else gp
                       for gp, c in zip(g_px_all, cams)]).contiguous()
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, g_dev, residual=res)
    assert scene.get_error()[0] == 0
    ogs, ogsig, ogt = O.render_bwd(osq, o[sel], d[sel], g_ray_o, params=op)
    grad_close(gsig.cpu().numpy(), ogsig, name + " sigma")
    grad_close(gs.cpu().numpy(), ogs, name + " sites")
    gt = gt.cpu().numpy()
    touched = np.nonzero(np.abs(ogt).reshape(len(ogt), -1).max(1) > 0)[0]
    grad_close(gt[touched], ogt[touched], name + " tex")
    rest = np.setdiff1d(np.arange(len(ogt)), touched)
    assert np.abs(gt.reshape(len(ogt), -1)[rest]).max() == 0


def test_mixed_cameras_image_table_against_oracle(medium):
    """Pinhole, equidistant fisheye, rolling shutter, thin lens (4 lens
    samples) and motion blur (2 time samples) in one image-table launch on the
    50k-site scene, every ray against the oracle."""
    sc, osc, o_, d_, cams_ = medium
    o0 = np.zeros(3)
    cams = [W.look_at_camera(0, 48, 32, W.orbit_eye(o0, 3.0, 10, 20), o0),
            W.look_at_camera(1, 48, 32, W.orbit_eye(o0, 3.0, 100, 20), o0, fisheye_fov=math.pi),
            W.look_at_camera(2, 48, 32, W.orbit_eye(o0, 3.0, 190, 20), o0, rs_velocity=(0.05, 0.0, 0.0)),
            W.look_at_camera(3, 48, 32, W.orbit_eye(o0, 3.0, 280, 20), o0, lens_radius=0.01, focus_dist=3.0,
                             lens_samples=4, seed=7),
            W.look_at_camera(4, 48, 32, W.orbit_eye(o0, 3.0, 330, 20), o0, rs_velocity=(0.0, 0.02, 0.01),
                             lens_samples=2, seed=8)]
    mixed_launch_against_oracle("50k-site mixed cameras", sc, cams, [np.arange(48 * 32)] * len(cams), seed=91)


def test_keep_order_scene_gives_identical_results(medium):
    """Cell storage order (Morton vs user order) changes memory locality only:
    every decision and value is the same."""
    sc, osc, o, d, cams = medium
    P = gpu_params(W.default_params(), img_w=203, img_h=121, n_images=2)
    to, td = to_dev(o, d)
    a = api.render_fwd(api.Scene.from_workload(sc), to, td, P)
    b = api.render_fwd(api.Scene.from_workload(sc, keep_order=True), to, td, P)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_gradients_vs_finite_differences_on_surface_crop():
    """GPU (FP32) gradients on the 1,000-site crop against FP64 central finite
    differences of the oracle's forward pass, at 1e-3 relative."""
    from test_oracle_pins import crop_setup, fd_crop
    sc, o, d, Y, params = crop_setup()
    res, (gs_o, gsig_o, gt_o) = fd_crop(sc, o, d, Y, params)
    scene = api.Scene.from_workload(sc)
    P = gpu_params(params, img_w=32, img_h=32, n_images=1)
    to, td = to_dev(o.astype(np.float32), d.astype(np.float32))
    rgb, resid = fwd_res(scene, to, td, P)
    # dL/dC from the oracle's colours, so both sides differentiate the same L
    osc = O.OracleScene.from_workload_scene(sc)
    orgb = O.render(osc, o, d, params=O.make_params(**params))[0]
    g = torch.as_tensor((orgb - Y).astype(np.float32), device=DEV)
    gs, gsig, gt = [x.cpu().numpy() for x in api.render_bwd(scene, to, td, P, rgb, g, residual=resid)]
    got = {"sigma": gsig, "tex": gt, "sites": gs}
    floors = {"sigma": 1e-3 * np.abs(gsig_o).max(), "tex": 1e-3 * np.abs(gt_o).max(),
              "sites": 1e-3 * np.abs(gs_o).max()}
    for kind, idx, fd, an in res:
        v = got[kind][idx]
        assert abs(v - fd) <= GRAD_REL * max(abs(fd), floors[kind]), (kind, idx, v, fd)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_paper_appearance_model(medium, dtype):
    """Appearance 1 (Sec. 5.1-5.2): c = sigmoid(T_vi(oct(surface direction)) +
    T_vd(oct(-d))). Forward images and the gradients of sites, sigma and both
    textures against the oracle; rays start in big empty cells, so the
    exit-point rule of the origin cell is exercised too."""
    sc, osc_, o, d, cams = medium
    rng = np.random.default_rng(90)
    tvi = rng.normal(0.0, 1.5, size=sc.tex.shape).astype(np.float32)
    tvd = rng.normal(0.0, 0.5, size=sc.tex.shape).astype(np.float32)
    if dtype == "f16":  # the oracle sees the stored (rounded) values
        tvi_o, tvd_o = [torch.as_tensor(x).half().float().numpy() for x in (tvi, tvd)]
    else:
        tvi_o, tvd_o = tvi, tvd
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2, appearance=1)
    scene = api.Scene(sc.sites, sc.sigma, tvi, sc.offsets, sc.indices, tex_dtype=dtype, tex_vd=tvd)
    to, td = to_dev(o, d)
    rgb, res = fwd_res(scene, to, td, P)
    assert scene.get_error()[0] == 0
    osc = O.OracleScene(sc.sites, sc.sigma, tvi_o, sc.offsets, sc.indices, tex_vd=tvd_o)
    op = O.make_params(**base, appearance=1)
    orgb, _, _, flags = O.render(osc, o, d, params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    assert ok.mean() > 0.95
    assert np.abs(rgb.cpu().numpy()[ok] - orgb[ok]).max() <= IMG_TOL
    g = (rng.normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    gvd = torch.empty(sc.n, sc.R, sc.R, 3, device=DEV)
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, torch.as_tensor(g, device=DEV), residual=res,
                                  tex_vd_out=gvd)
    ogs, ogsig, ogt, ogvd = O.render_bwd(osc, o, d, g.astype(np.float64), params=op)
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gt.cpu().numpy(), ogt, "tex_vi")
    grad_close(gvd.cpu().numpy(), ogvd, "tex_vd")
    grad_close(gs.cpu().numpy(), ogs, "sites")


def test_paper_appearance_autograd_and_rejections(tiny):
    wl, osc, o, d = tiny
    sc = wl.scene
    tvd = np.zeros_like(sc.tex)
    scene = api.Scene.from_workload(sc, tex_vd=tvd)
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1, appearance=1)
    sites = torch.tensor(sc.sites, device=DEV, requires_grad=True)
    sigma = torch.tensor(sc.sigma, device=DEV, requires_grad=True)
    tex = torch.tensor(sc.tex, device=DEV, requires_grad=True)
    tex_vd = torch.tensor(tvd, device=DEV, requires_grad=True)
    to, td = to_dev(o, d)
    rgb = api.render(sites, sigma, tex, to, td, scene, P, tex_vd=tex_vd)
    rgb.sum().backward()
    assert tex_vd.grad is not None and torch.isfinite(tex_vd.grad).all()
    assert (tex_vd.grad.abs().sum() > 0).item()
    # appearance 1 needs a scene with a view-dependent texture
    plain = api.Scene.from_workload(sc)
    with pytest.raises(api._vt.VTError):
        api.render_fwd(plain, to, td, P)


# ---------------------------------------------------------------- distortion loss (Eq. 2), sigma = exp(rho)

DIST_TOL = 2e-5  # |L_gpu - L_ref| <= DIST_TOL * max(L_ref, 1e-3 max L_ref): FP32 sums of positive terms


@pytest.mark.parametrize("which", ["tiny", "medium"])
def test_distortion_forward_parity(which, tiny, medium):
    if which == "tiny":
        wl, osc, o, d = tiny
        sc, base, img = wl.scene, wl.params, dict(img_w=64, img_h=64, n_images=1)
    else:
        sc, osc, o, d, _ = medium
        base, img = W.default_params(), dict(img_w=203, img_h=121, n_images=2)
    scene = api.Scene.from_workload(sc)
    to, td = to_dev(o, d)
    dist = torch.empty(len(o), 3, device=DEV)
    rgb, _, _ = api.render_fwd(scene, to, td, gpu_params(base, **img), dist=dist)
    plain = api.render_fwd(scene, to, td, gpu_params(base, **img))[0]
    assert torch.equal(rgb, plain)  # the loss does not change the image
    assert scene.get_error()[0] == 0
    _, oT, _, flags = O.render(osc, o, d, params=oracle_params(base))
    ok = (flags & O.BAND_FLAGS) == 0
    L = O.distortion(osc, o, d, params=oracle_params(base))
    got = dist[:, 0].cpu().numpy().astype(np.float64)
    tol = DIST_TOL * np.maximum(L, 1e-3 * L.max())
    assert np.all(np.abs(got - L)[ok] <= tol[ok]), np.abs(got - L)[ok].max()
    hit = ok & (oT < 1)  # rays that composite at least one interval
    assert hit.sum() > 500 and np.all(L[hit] > 0)
    assert np.all(got >= 0)


@pytest.mark.parametrize("appearance", [0, 1])
def test_distortion_backward_parity(tiny, appearance):
    wl, osc, o, d = tiny
    sc = wl.scene
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1, appearance=appearance)
    if appearance:
        tvd = np.random.default_rng(21).normal(0, 0.5, size=sc.tex.shape).astype(np.float32)
        osc = O.OracleScene(sc.sites, sc.sigma, sc.tex, sc.offsets, sc.indices, tex_vd=tvd)
        scene = api.Scene(sc.sites, sc.sigma, sc.tex, sc.offsets, sc.indices, tex_vd=tvd)
    else:
        scene = api.Scene.from_workload(sc)
    op = oracle_params(wl.params, appearance=appearance)
    _, _, _, flags = O.render(osc, o, d, params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    rng = np.random.default_rng(22)
    g = (rng.normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    gd = (rng.uniform(0.5, 2.0, size=len(o)) * ok).astype(np.float32)
    to, td, tg, tgd = to_dev(o, d, g, gd)
    res = torch.empty(len(o), 3, device=DEV)
    dist = torch.empty(len(o), 3, device=DEV)
    rgb = api.render_fwd(scene, to, td, P, residual=res, dist=dist)[0]
    tvo = torch.empty_like(torch.as_tensor(sc.tex, device=DEV)) if appearance else None
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, tg, residual=res, dist=dist, grad_dist=tgd,
                                  tex_vd_out=tvo)
    assert scene.get_error()[0] == 0
    ref = O.render_bwd(osc, o, d, g.astype(np.float64), params=op, grad_dist=gd.astype(np.float64))
    grad_close(gsig.cpu().numpy(), ref[1], "sigma")
    grad_close(gt.cpu().numpy(), ref[2], "tex")
    grad_close(gs.cpu().numpy(), ref[0], "sites")
    if appearance:
        grad_close(tvo.cpu().numpy(), ref[3], "tex_vd")
    # distortion only (no colour gradient)
    z = torch.zeros_like(tg)
    gs2, gsig2, gt2 = api.render_bwd(scene, to, td, P, rgb, z, residual=res, dist=dist, grad_dist=tgd)
    ref2 = O.render_bwd(osc, o, d, np.zeros((len(o), 3)), params=op, grad_dist=gd.astype(np.float64))
    grad_close(gsig2.cpu().numpy(), ref2[1], "sigma (distortion only)")
    grad_close(gs2.cpu().numpy(), ref2[0], "sites (distortion only)")
    assert gt2.abs().max().item() == 0.0


def test_distortion_medium_backward_parity(medium):
    sc, osc, o, d, cams = medium
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2)
    _, _, _, flags = O.render(osc, o, d, params=oracle_params(base))
    ok = (flags & O.BAND_FLAGS) == 0
    rng = np.random.default_rng(23)
    g = (rng.normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    gd = (rng.uniform(0.0, 1.0, size=len(o)) * ok).astype(np.float32)
    scene = api.Scene.from_workload(sc)
    to, td, tg, tgd = to_dev(o, d, g, gd)
    res = torch.empty(len(o), 3, device=DEV)
    dist = torch.empty(len(o), 3, device=DEV)
    rgb = api.render_fwd(scene, to, td, P, residual=res, dist=dist)[0]
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, tg, residual=res, dist=dist, grad_dist=tgd)
    ogs, ogsig, ogt = O.render_bwd(osc, o, d, g.astype(np.float64), params=oracle_params(base),
                                   grad_dist=gd.astype(np.float64))
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gt.cpu().numpy(), ogt, "tex")
    grad_close(gs.cpu().numpy(), ogs, "sites")


def test_distortion_autograd_and_rho(tiny):
    """Training-style use: sigma = exp(rho) on the GPU, render with the
    distortion loss, torch autograd through both; equals the explicit calls."""
    wl, osc, o, d = tiny
    sc = wl.scene
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1)
    scene = api.Scene.from_workload(sc)
    rho = torch.log(torch.tensor(sc.sigma, device=DEV)).requires_grad_(True)
    sites = torch.tensor(sc.sites, device=DEV, requires_grad=True)
    tex = torch.tensor(sc.tex, device=DEV, requires_grad=True)
    sigma = api.SigmaFromRho.apply(rho)
    assert torch.allclose(sigma, torch.exp(rho.detach()), rtol=2e-7, atol=0)
    scene.update(sigma=sigma.detach())
    to, td = to_dev(o, d)
    Y = torch.as_tensor(W.target_image(len(o), 1), device=DEV)
    rgb, Ld = api.render(sites, sigma, tex, to, td, scene, P, with_dist=True)
    lam = 0.01
    loss = ((rgb - Y) ** 2).mean() + lam * Ld.mean()
    loss.backward()
    res = torch.empty(len(o), 3, device=DEV)
    dist = torch.empty(len(o), 3, device=DEV)
    rgb2 = api.render_fwd(scene, to, td, P, residual=res, dist=dist)[0]
    assert torch.equal(rgb2, rgb.detach()) and torch.equal(dist[:, 0], Ld.detach())
    gd = torch.full((len(o),), lam / len(o), device=DEV)
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb2, 2 * (rgb2 - Y) / rgb2.numel(), residual=res, dist=dist,
                                  grad_dist=gd)
    assert torch.allclose(sites.grad, gs, rtol=1e-5, atol=1e-9)
    assert torch.allclose(tex.grad, gt, rtol=1e-5, atol=1e-9)
    assert torch.allclose(rho.grad, gsig * sigma.detach(), rtol=1e-5, atol=1e-12)  # Eq. 4


def test_distortion_rejects_negative_t_near(tiny):
    wl, osc, o, d = tiny
    scene = api.Scene.from_workload(wl.scene)
    to, td = to_dev(o[:10], d[:10])
    dist = torch.empty(10, 3, device=DEV)
    with pytest.raises(api.VTError):
        api.render_fwd(scene, to, td, gpu_params(wl.params, t_near=-0.5), dist=dist)
    rgb = api.render_fwd(scene, to, td, gpu_params(wl.params))[0]
    with pytest.raises(api.VTError):  # grad_dist without the forward's totals
        api.render_bwd(scene, to, td, gpu_params(wl.params), rgb, torch.zeros_like(rgb),
                       grad_dist=torch.ones(10, device=DEV))


# ---------------------------------------------------------------- FP16 neighbour offsets (Sec. 5.6 inference variant)

def test_half_offsets_forward_against_exact_walk(medium):
    """FP16 offsets move each plane by about |n| 2^-11, so rays that pass
    close to a Voronoi edge may take another cell; the rest keep the exact
    sequence. Reports the mismatch count; bounds it and the image error."""
    sc, osc, o, d, cams = medium
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2)
    to, td = to_dev(o, d)
    half = api.Scene.from_workload(sc, half_offsets=True)
    full = api.Scene.from_workload(sc)
    rgb_h = api.render_fwd(half, to, td, P)[0].cpu().numpy()
    rgb_f = api.render_fwd(full, to, td, P)[0].cpu().numpy()
    ch, _, nh = api.trace_cells(half, to, td, P, max_cells=256)
    assert half.get_error()[0] == 0
    orgb, _, _, flags = O.render(osc, o, d, params=oracle_params(base))
    oc, _, on, _ = O.trace(osc, o, d, max_cells=256, params=oracle_params(base))
    ok = (flags & O.BAND_FLAGS) == 0
    same = (nh.cpu().numpy() == on) & np.all(ch.cpu().numpy() == oc, axis=1)
    frac = same[ok].mean()
    rmse_h = float(np.sqrt(np.mean((rgb_h - orgb) ** 2)))
    rmse_f = float(np.sqrt(np.mean((rgb_f[ok] - orgb[ok]) ** 2)))
    parity_log.record("50k-site FP16 neighbour offsets (not exact by design)", rays=len(o),
                      unflagged_seq_differ=int((~same & ok).sum()), rmse=rmse_h, rmse_exact_offsets=rmse_f)
    assert frac >= 0.9 and rmse_h <= 5e-3
    # forward only
    with pytest.raises(api.VTError):
        api.render_bwd(half, to, td, P, torch.as_tensor(rgb_h, device=DEV), torch.zeros(len(o), 3, device=DEV))
    with pytest.raises(api.VTError):
        api.render_fwd(half, to, td, P, dist=torch.empty(len(o), 3, device=DEV))


def test_backward_scratch_is_clean_between_calls(medium):
    """The backward leaves its texel scratch zeroed for the next call (only the
    cells it touched are rewritten): repeated calls with other rays, other
    gradients and skipped outputs give the results of a fresh scene."""
    sc, osc, o, d, cams = medium
    P = gpu_params(W.default_params())
    to, td = to_dev(o, d)
    g = seeded(len(o), 3, seed=107)
    used = api.Scene.from_workload(sc)
    rgb = api.render_fwd(used, to, td, P)[0]
    # dirty the scratch: a call without texel output, then one on half the rays
    api.render_bwd(used, to, td, P, rgb, g * 3.0, need=(True, True, False))
    h = len(o) // 2
    api.render_bwd(used, to[:h].contiguous(), td[:h].contiguous(), P, rgb[:h].contiguous(), g[:h].contiguous())
    a = api.render_bwd(used, to[h:].contiguous(), td[h:].contiguous(), P, rgb[h:].contiguous(), g[h:].contiguous())
    fresh = api.Scene.from_workload(sc)
    b = api.render_bwd(fresh, to[h:].contiguous(), td[h:].contiguous(), P, rgb[h:].contiguous(), g[h:].contiguous())
    for x, y in zip(a, b):
        assert (x - y).abs().max().item() <= 1e-5 * max(1.0, y.abs().max().item())
    # untouched texels are exactly zero
    touched = b[2].abs().reshape(sc.n, -1).max(1).values > 0
    assert a[2].reshape(sc.n, -1)[~touched].abs().max().item() == 0.0


def _scene_order_to_user(scene, gc, gt):
    """Scene-order gradients (float4 cells, RGBA texels) in user order, as the
    outputs of vt_render_bwd."""
    perm = scene.permutation().long()
    gs = torch.empty(scene.n, 3, device=DEV)
    gsig = torch.empty(scene.n, device=DEV)
    gtu = torch.empty(scene.n, scene.R, scene.R, 3, device=DEV)
    gs[perm] = gc[:, :3]
    gsig[perm] = gc[:, 3]
    gtu[perm] = gt[..., :3]
    return gs, gsig, gtu


def test_scene_order_backward_against_oracle(medium):
    """vt_render_bwd_scene_order: the gradients left in the scene's cell order
    (no permute), mapped back with vt_scene_permutation, against the oracle;
    repeated calls and a following vt_render_bwd see clean scratch."""
    sc, osc, o, d, cams = medium
    base = W.default_params()
    P = gpu_params(base, img_w=203, img_h=121, n_images=2)
    _, _, _, flags = O.render(osc, o, d, params=oracle_params(base))
    ok = (flags & O.BAND_FLAGS) == 0
    rng = np.random.default_rng(24)
    g = (rng.normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    scene = api.Scene.from_workload(sc)
    to, td, tg = to_dev(o, d, g)
    rgb, res = fwd_res(scene, to, td, P)
    gc, gt, gv = api.render_bwd_scene_order(scene, to, td, P, rgb, tg, residual=res)
    assert gv is None and gc.shape == (sc.n, 4) and gt.shape == (sc.n, sc.R, sc.R, 4)
    assert scene.get_error()[0] == 0
    assert gt[..., 3].abs().max().item() == 0.0
    gs, gsig, gtu = [x.cpu().numpy() for x in _scene_order_to_user(scene, gc, gt)]
    ogs, ogsig, ogt = O.render_bwd(osc, o, d, g.astype(np.float64), params=oracle_params(base))
    grad_close(gsig, ogsig, "sigma")
    grad_close(gtu, ogt, "tex")
    grad_close(gs, ogs, "sites")
    # a second scene-order call with other gradients, then the user-order call:
    # both equal a fresh scene's user-order backward
    g2 = seeded(len(o), 3, seed=108)
    gc2, gt2, _ = api.render_bwd_scene_order(scene, to, td, P, rgb, g2, residual=res)
    second = _scene_order_to_user(scene, gc2, gt2)
    third = api.render_bwd(scene, to, td, P, rgb, g2, residual=res)
    fresh = api.render_bwd(api.Scene.from_workload(sc), to, td, P, rgb, g2, residual=res)
    for a, b, f in zip(second, third, fresh):
        scale = max(1.0, f.abs().max().item())
        assert (a - f).abs().max().item() <= 1e-5 * scale
        assert (b - f).abs().max().item() <= 1e-5 * scale


def test_scene_order_backward_paper_appearance(tiny):
    """The scene-order backward with the paper's appearance model and the
    distortion loss equals vt_render_bwd mapped to scene order, both maps."""
    wl, osc, o, d = tiny
    sc = wl.scene
    tvd = np.random.default_rng(25).normal(0, 0.5, size=sc.tex.shape).astype(np.float32)
    scene = api.Scene(sc.sites, sc.sigma, sc.tex, sc.offsets, sc.indices, tex_vd=tvd)
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1, appearance=1)
    to, td = to_dev(o, d)
    res = torch.empty(len(o), 3, device=DEV)
    dist = torch.empty(len(o), 3, device=DEV)
    rgb = api.render_fwd(scene, to, td, P, residual=res, dist=dist)[0]
    g = seeded(len(o), 3, seed=109)
    gd = seeded(len(o), seed=110, normal=False)
    vd_ref = torch.empty(sc.n, sc.R, sc.R, 3, device=DEV)
    ref = api.render_bwd(scene, to, td, P, rgb, g, residual=res, dist=dist, grad_dist=gd, tex_vd_out=vd_ref)
    gc, gt, gv = api.render_bwd_scene_order(scene, to, td, P, rgb, g, residual=res, dist=dist, grad_dist=gd)
    got = _scene_order_to_user(scene, gc, gt)
    perm = scene.permutation().long()
    vd = torch.empty_like(vd_ref)
    vd[perm] = gv[..., :3]
    for a, b in zip(list(got) + [vd], list(ref) + [vd_ref]):
        assert (a - b).abs().max().item() <= 1e-5 * max(1.0, b.abs().max().item())


def test_cuda_path_matches_stored_golden_values():
    """The CUDA path against the stored oracle values of tests/golden (no
    oracle run): cells and step counts exact, colours within 1e-4."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny_rays.json")))
    wl = W.make_workload("tiny")
    o, d = W.workload_rays(wl)
    sel = np.array([r["index"] for r in g["rays"]])
    scene = api.Scene.from_workload(wl.scene)
    P = gpu_params(wl.params)
    to, td = to_dev(o[sel], d[sel])
    dist = torch.empty(len(sel), 3, device=DEV)
    rgb, T, steps = api.render_fwd(scene, to, td, P, dist=dist)
    cells, t_exit, n_cells = api.trace_cells(scene, to, td, P, max_cells=64)
    rgb, T, steps, dist = rgb.cpu().numpy(), T.cpu().numpy(), steps.cpu().numpy(), dist.cpu().numpy()
    cells, t_exit, n_cells = cells.cpu().numpy(), t_exit.cpu().numpy(), n_cells.cpu().numpy()
    for k, r in enumerate(g["rays"]):
        assert r["flags"] == 0
        n = len(r["cells"])
        assert steps[k] == r["steps"] and n_cells[k] == n and list(cells[k, :n]) == r["cells"]
        assert np.abs(rgb[k] - np.array(r["rgb"])).max() <= IMG_TOL and abs(T[k] - r["T"]) <= IMG_TOL
        assert abs(dist[k, 0] - r["L_dist"]) <= 2e-5 * max(r["L_dist"], 1e-3)
        te = np.array([np.inf if t is None else t for t in r["t_exit"]])
        fin = np.isfinite(te)
        assert np.all(np.abs(t_exit[k, :n][fin] - te[fin]) <= 1e-5 * np.maximum(1.0, np.abs(te[fin])))


def test_walk_events_time_the_kernel(medium):
    """vt_render_params.walk_events: the library records the pair around the
    walk kernel; the interval lies inside the whole call's interval."""
    sc, osc, o, d, cams = medium
    P = gpu_params(W.default_params(), img_w=203, img_h=121, n_images=2)
    to, td = to_dev(o, d)
    scene = api.Scene.from_workload(sc)
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev[1:3]:
        e.record(st)  # create the handles the library records into
    torch.cuda.synchronize()
    P.walk_events[0], P.walk_events[1] = ev[1].cuda_event, ev[2].cuda_event
    ev[0].record(st)
    api.render_fwd(scene, to, td, P)
    ev[3].record(st)
    torch.cuda.synchronize()
    walk, call = ev[1].elapsed_time(ev[2]), ev[0].elapsed_time(ev[3])
    assert 0.0 < walk <= call
    assert ev[0].elapsed_time(ev[1]) >= 0.0 and ev[2].elapsed_time(ev[3]) >= 0.0


def test_measurement_aids(tiny):
    """vt_kernel_launches counts the library's own launches (a forward render:
    anchor search, anchor refinement, walk); vt_stream_read reads a buffer
    and rejects a misaligned pointer or size."""
    from paper_2608_17682_gb300 import _vt
    wl, osc, o, d = tiny
    scene = api.Scene.from_workload(wl.scene)
    to, td = to_dev(o, d)
    P = gpu_params(wl.params, img_w=64, img_h=64, n_images=1)
    api.render_fwd(scene, to, td, P)
    before = _vt.vt_kernel_launches()
    api.render_fwd(scene, to, td, P)
    assert _vt.vt_kernel_launches() - before == 3
    buf = torch.ones(1 << 20, device=DEV)
    sink = torch.zeros(1, device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    _vt.vt_stream_read(buf.data_ptr(), buf.numel() * 4, 3, sink.data_ptr(), st)
    torch.cuda.synchronize()
    assert sink.item() == 0.0  # written only on a value the data never produces
    for ptr, nbytes in ((buf.data_ptr() + 4, 1024), (buf.data_ptr(), 1000)):
        with pytest.raises(api._vt.VTError) as e:
            _vt.vt_stream_read(ptr, nbytes, 1, sink.data_ptr(), st)
        assert e.value.status == api._vt.VT_ERR_INVALID_ARG
