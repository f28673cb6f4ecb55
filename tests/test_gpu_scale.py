"""Full-size parity at the benchmark's scale and launch configuration:
3,000,000 surface-concentrated sites, 8x8 textures, four 1280x832 views
(4,259,840 rays in one launch, image layout, 4x8 tiles) with FP32, FP16 and
BF16 texture storage, and the paper's appearance model with the distortion
loss; the mixed-camera workload (16 cameras, 29,818,880 rays in one
image-table launch). The oracle computes a strided sample of the rays one by
one (every 997th ray of the four views, every 4001st pixel of the mixed
cameras); gradients are compared for a launch over all rays in which only the
sampled rays carry dL/dC. Ray generation of the 16 mixed cameras is compared
with the oracle's ray generation camera by camera.

The 3M-site Delaunay triangulations take a few minutes on the host the first
time; they are cached on local disk for the benchmark.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2608_17682_gb300 import api  # noqa: E402
from paper_2608_17682_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import compare_sequences, grad_close, image_report, IMG_TOL, mixed_launch_against_oracle  # noqa: E402,E501

STRIDE = 997


@pytest.fixture(scope="module")
def big():
    wl = W.make_workload("prec3m")
    o, d = W.workload_rays(wl)
    sel = np.arange(0, len(o), STRIDE)
    return wl, o, d, sel


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_fullsize_forward_and_backward(big, dtype):
    wl, o, d, sel = big
    sc = wl.scene
    c0 = wl.cameras[0]
    P = api.make_params(**wl.params, img_w=c0.w, img_h=c0.h, n_images=len(wl.cameras))
    scene = api.Scene.from_workload(sc, tex_dtype=dtype)
    to = torch.as_tensor(o, device="cuda")
    td = torch.as_tensor(d, device="cuda")
    res = torch.empty(len(o), 3, device="cuda")
    rgb, T, steps = api.render_fwd(scene, to, td, P, residual=res)
    assert scene.get_error()[0] == 0
    q = {"f16": torch.float16, "bf16": torch.bfloat16}
    tex = sc.tex if dtype == "f32" else torch.as_tensor(sc.tex).to(q[dtype]).float().numpy()
    osc = O.OracleScene(sc.sites, sc.sigma, tex, sc.offsets, sc.indices)
    op = O.make_params(**wl.params)
    orgb, oT, osteps, flags = O.render(osc, o[sel], d[sel], params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    assert ok.mean() > 0.95
    g_rgb = rgb.cpu().numpy()[sel]
    image_report(f"3M-site {dtype} textures (oracle on the stored texels)", g_rgb, orgb, flags)
    assert np.abs(g_rgb[ok] - orgb[ok]).max() <= IMG_TOL
    assert np.array_equal(steps.cpu().numpy()[sel][ok], osteps[ok])
    # cell sequences of the sampled rays
    cells, _, n_cells = api.trace_cells(scene, to[sel].contiguous(), td[sel].contiguous(), api.make_params(**wl.params),
                                        max_cells=512)
    oc, _, on, _ = O.trace(osc, o[sel], d[sel], max_cells=512, params=op)
    compare_sequences(cells.cpu().numpy(), n_cells.cpu().numpy(), oc, on, flags, name=f"3M-site {dtype} textures")
    if dtype != "f32":
        # total error against the FP64 oracle on the FP32 textures
        o32 = O.OracleScene.from_workload_scene(sc)
        orgb32 = O.render(o32, o[sel], d[sel], params=op)[0]
        image_report(f"3M-site {dtype} textures vs FP32 textures", g_rgb, orgb32, flags)
        rmse = math.sqrt(np.mean((g_rgb[ok] - orgb32[ok]) ** 2))
        assert rmse <= 2e-3, rmse
    # backward over all rays; only sampled, unflagged rays carry a gradient
    g = np.zeros((len(o), 3), np.float32)
    rng = np.random.default_rng(12)
    g[sel[ok]] = rng.normal(size=(ok.sum(), 3))
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, torch.as_tensor(g, device="cuda"), residual=res)
    assert scene.get_error()[0] == 0
    ogs, ogsig, ogt = O.render_bwd(osc, o[sel], d[sel], g[sel].astype(np.float64), params=op)
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gs.cpu().numpy(), ogs, "sites")
    touched = np.nonzero(np.abs(ogt).reshape(len(ogt), -1).max(1) > 0)[0]
    grad_close(gt.cpu().numpy()[touched], ogt[touched], "tex")
    assert np.abs(gt.cpu().numpy()).reshape(len(ogt), -1).max(1)[np.setdiff1d(np.arange(len(ogt)), touched)].max() == 0


def test_fullsize_paper_appearance_with_distortion(big):
    """The paper's appearance model (Sec. 5.1-5.2) and the distortion loss
    (Eq. 2) fused into the same full-size launch (FP16 textures), sampled
    rays against the oracle: colour, L_dist, and the gradients of
    L = sum g.C + sum gd L_dist."""
    wl, o, d, sel = big
    sc = wl.scene
    c0 = wl.cameras[0]
    rng = np.random.default_rng(5000 + wl.seed)
    tvd = rng.normal(0.0, 0.5, size=sc.tex.shape).astype(np.float32)
    tvi = rng.normal(0.0, 1.5, size=sc.tex.shape).astype(np.float32)
    P = api.make_params(**wl.params, img_w=c0.w, img_h=c0.h, n_images=len(wl.cameras), appearance=1)
    scene = api.Scene(sc.sites, sc.sigma, tvi, sc.offsets, sc.indices, tex_dtype="f16", tex_vd=tvd)
    to = torch.as_tensor(o, device="cuda")
    td = torch.as_tensor(d, device="cuda")
    res = torch.empty(len(o), 3, device="cuda")
    dist = torch.empty(len(o), 3, device="cuda")
    rgb, _, _ = api.render_fwd(scene, to, td, P, residual=res, dist=dist)
    assert scene.get_error()[0] == 0
    q = lambda x: torch.as_tensor(x).half().float().numpy()  # noqa: E731
    osc = O.OracleScene(sc.sites, sc.sigma, q(tvi), sc.offsets, sc.indices, tex_vd=q(tvd))
    op = O.make_params(**wl.params, appearance=1)
    orgb, _, _, flags = O.render(osc, o[sel], d[sel], params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    assert ok.mean() > 0.95
    assert np.abs(rgb.cpu().numpy()[sel][ok] - orgb[ok]).max() <= IMG_TOL
    L = O.distortion(osc, o[sel], d[sel], params=op)
    got = dist[:, 0].cpu().numpy()[sel].astype(np.float64)
    assert np.all(np.abs(got - L)[ok] <= 2e-5 * np.maximum(L, 1e-3 * L.max())[ok])
    g = np.zeros((len(o), 3), np.float32)
    gd = np.zeros(len(o), np.float32)
    g[sel[ok]] = rng.normal(size=(ok.sum(), 3))
    gd[sel[ok]] = rng.uniform(0.5, 2.0, size=ok.sum())
    gvd = torch.empty(sc.n, sc.R, sc.R, 3, device="cuda")
    gs, gsig, gt = api.render_bwd(scene, to, td, P, rgb, torch.as_tensor(g, device="cuda"), residual=res,
                                  dist=dist, grad_dist=torch.as_tensor(gd, device="cuda"), tex_vd_out=gvd)
    assert scene.get_error()[0] == 0
    ogs, ogsig, ogt, ogvd = O.render_bwd(osc, o[sel], d[sel], g[sel].astype(np.float64), params=op,
                                         grad_dist=gd[sel].astype(np.float64))
    grad_close(gsig.cpu().numpy(), ogsig, "sigma")
    grad_close(gs.cpu().numpy(), ogs, "sites")
    touched = np.nonzero(np.abs(ogt).reshape(len(ogt), -1).max(1) > 0)[0]
    grad_close(gt.cpu().numpy()[touched], ogt[touched], "tex")
    touched = np.nonzero(np.abs(ogvd).reshape(len(ogvd), -1).max(1) > 0)[0]
    grad_close(gvd.cpu().numpy()[touched], ogvd[touched], "tex_vd")


def test_fullsize_mixed_camera_raygen():
    cams = W.workload_cameras("mixed3m")
    o, d, t = api.generate_rays(cams)
    assert o.shape[0] == 29_818_880
    base = 0
    for c in cams:
        n = c.n_rays
        oo, od, ot = O.raygen(c)
        go = o[base:base + n].cpu().numpy()
        gd = d[base:base + n].cpu().numpy()
        gt = t[base:base + n].cpu().numpy()
        assert np.abs(go - oo).max() <= 4e-7 * 4.0, c.kind
        assert np.abs(gd - od).max() <= 4e-6, c.kind
        assert np.abs(gt - ot).max() <= 1e-7, c.kind
        base += n


def test_fullsize_mixed_cameras_against_oracle():
    """The mixed-camera workload as the benchmark launches it: 3,000,000 sites
    (FP16 8x8 textures), 4 pinhole, 4 fisheye, 4 rolling-shutter and 4
    thin-lens (4 lens samples) cameras of 1280x832, 29,818,880 rays in one
    image-table launch, forward and backward. Every 4001st pixel of each
    camera (all its lens samples) against the oracle."""
    wl = W.make_workload("mixed3m")
    sel_px = [np.arange(0, c.n_rays // c.spp, 4001) for c in wl.cameras]
    mixed_launch_against_oracle("3M-site mixed cameras", wl.scene, wl.cameras, sel_px, seed=13)
