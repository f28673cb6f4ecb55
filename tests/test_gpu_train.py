"""GPU checks of the training step (Sec. 5.3-5.5, Eq. 5): the helper kernels
against the plain float64 definitions in oracle/training.py, and a short
multi-view optimisation with Delaunay refreshes that must reduce the loss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import training as TR  # noqa: E402
from paper_2608_17682_gb300 import _vt, api  # noqa: E402
from paper_2608_17682_gb300 import train as T  # noqa: E402

DEV = "cuda"


def _st():
    return api._stream()


@pytest.mark.parametrize("n_pool,n", [(10_000, 777), (4096, 4096), (1_000_003, 65_536)])
def test_sample_rays_matches_definition(n_pool, n):
    g = torch.Generator().manual_seed(n)
    o = torch.rand(n_pool, 3, generator=g).to(DEV)
    d = torch.rand(n_pool, 3, generator=g).to(DEV)
    y = torch.rand(n_pool, 3, generator=g).to(DEV)
    oo, dd, yy = (torch.empty(n, 3, device=DEV) for _ in range(3))
    idx = torch.empty(n, dtype=torch.int64, device=DEV)
    _vt.vt_sample_rays(n_pool, o.data_ptr(), d.data_ptr(), y.data_ptr(), n, 99, oo.data_ptr(), dd.data_ptr(),
                       yy.data_ptr(), idx.data_ptr(), _st())
    ref = TR.stratified_indices(n_pool, n, 99)
    assert np.array_equal(idx.cpu().numpy(), ref)
    r = torch.as_tensor(ref, device=DEV)
    assert torch.equal(oo, o[r]) and torch.equal(dd, d[r]) and torch.equal(yy, y[r])


def test_smooth_l1_kernel():
    rng = np.random.default_rng(41)
    a = rng.uniform(0, 1, size=(70_001, 3)).astype(np.float32)
    b = rng.uniform(0, 1, size=(70_001, 3)).astype(np.float32)
    ta, tb = torch.as_tensor(a, device=DEV), torch.as_tensor(b, device=DEV)
    g = torch.empty_like(ta)
    loss = torch.empty(1, device=DEV)
    _vt.vt_smooth_l1_loss(len(a), ta.data_ptr(), tb.data_ptr(), 0.05, g.data_ptr(), loss.data_ptr(), _st())
    L, gr = TR.smooth_l1(a, b, 0.05)
    assert abs(loss.item() - L) <= 1e-6 * L
    assert np.allclose(g.cpu().numpy(), gr, rtol=2e-6, atol=1e-13)


@pytest.mark.parametrize("R", [4, 8])
def test_texture_regularizer_kernel(R):
    rng = np.random.default_rng(42 + R)
    n = 3001
    t = rng.normal(size=(n, R, R, 3)).astype(np.float32)
    v = rng.normal(size=(n, R, R, 3)).astype(np.float32)
    g0 = (1e-6 * rng.normal(size=(n, R, R, 3))).astype(np.float32)  # small enough that the sum keeps the term
    tt, tv = torch.as_tensor(t, device=DEV), torch.as_tensor(v, device=DEV)
    gt, gv = torch.as_tensor(g0, device=DEV).clone(), torch.as_tensor(g0, device=DEV).clone()
    loss = torch.empty(1, device=DEV)
    _vt.vt_texture_regularizers(n, R, tt.data_ptr(), tv.data_ptr(), 0.01, 0.005, gt.data_ptr(), gv.data_ptr(),
                                loss.data_ptr(), _st())
    L, rgt, rgv = TR.texture_regularizers(t, v, 0.01, 0.005)
    assert abs(loss.item() - L) <= 1e-5 * L
    # gradients are added to what the buffers held
    assert np.allclose(gt.cpu().numpy().astype(np.float64) - g0, rgt, rtol=1e-4, atol=1e-12)
    assert np.allclose(gv.cpu().numpy().astype(np.float64) - g0, rgv, rtol=1e-4, atol=1e-12)


def test_adam_kernel():
    rng = np.random.default_rng(43)
    n = 100_003
    p = rng.normal(size=n).astype(np.float32)
    tp = torch.as_tensor(p, device=DEV).clone()
    tm, tv = torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    rp, rm, rv = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for k in range(1, 5):
        g = rng.normal(size=n).astype(np.float32)
        tg = torch.as_tensor(g, device=DEV)
        _vt.vt_adam_step(n, tp.data_ptr(), tg.data_ptr(), tm.data_ptr(), tv.data_ptr(), 1e-2, 0.9, 0.999, 1e-15, k,
                         _st())
        rp, rm, rv = TR.adam(rp, g, rm, rv, 1e-2, 0.9, 0.999, 1e-15, k)
    assert np.abs(tp.cpu().numpy() - rp).max() <= 2e-6


def test_training_reduces_loss_with_delaunay_refresh():
    init, cams, images, rp, gt = T.synthetic_problem(n_sites=4000, n_cams=6, w=64, h=48, tex_res=4, seed=3)
    cfg = T.TrainConfig(iters=120, rays_per_iter=8192, refresh_every=40, vd_ramp_frac=0.0, seed=1)
    tr = T.Trainer(init["sites"], init["rho"], init["tex"], init["tex_vd"], cams, images, rp, cfg)

    def image_mse():
        return float(((tr.render(cams) - images) ** 2).mean().item())

    m0 = image_mse()
    losses = []
    for _ in range(cfg.iters):
        losses.append(tr.step(sync_loss=True)[0])
    st, _ = tr.scene.get_error()
    assert st == 0
    assert tr.refreshes == 2
    m1 = image_mse()
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10]), (losses[:10], losses[-10:])
    assert m1 < 0.5 * m0, (m0, m1)
    assert torch.isfinite(tr.p["sites"]).all() and torch.isfinite(tr.p["rho"]).all()


@pytest.mark.parametrize("reg", [0, 1])
def test_scene_order_texture_adam_matches_definition(reg):
    """vt_adam_step_tex_scene_order: scene-order RGBA gradients mapped to user
    order through the permutation, the regulariser of Eq. 5 (L_mean or L_vd)
    added at the parameters before the step, then Adam — against the float64
    definitions; two steps, the second with another gradient."""
    rng = np.random.default_rng(44 + reg)
    n, R = 2003, 4
    perm = rng.permutation(n).astype(np.int32)
    p = rng.normal(size=(n, R, R, 3)).astype(np.float32)
    tp = torch.as_tensor(p, device=DEV).clone()
    tm, tv = torch.zeros_like(tp), torch.zeros_like(tp)
    rp, rm, rv = p.astype(np.float64), np.zeros(p.shape), np.zeros(p.shape)
    tperm = torch.as_tensor(perm, device=DEV)
    lam, lr = 0.3, 1e-2
    for k in range(1, 3):
        gsc = rng.normal(size=(n, R, R, 4)).astype(np.float32)
        tgsc = torch.as_tensor(gsc, device=DEV)  # referenced until the kernel has run
        loss = torch.zeros(1, device=DEV)
        _vt.vt_adam_step_tex_scene_order(n, R, tperm.data_ptr(), tgsc.data_ptr(), tp.data_ptr(), tm.data_ptr(),
                                         tv.data_ptr(), reg, lam, lr, 0.9, 0.999, 1e-15, k, loss.data_ptr(), _st())
        torch.cuda.synchronize()
        g_user = np.empty(p.shape)
        g_user[perm] = gsc[..., :3]
        if reg == 0:
            L, g_reg, _ = TR.texture_regularizers(rp, np.zeros(p.shape), 0.0, lam)
        else:
            L, _, g_reg = TR.texture_regularizers(np.zeros(p.shape), rp, lam, 0.0)
        assert abs(loss.item() - L) <= 1e-5 * L
        rp, rm, rv = TR.adam(rp, g_user + g_reg, rm, rv, lr, 0.9, 0.999, 1e-15, k)
        assert np.abs(tp.cpu().numpy() - rp).max() <= 2e-6, k


def test_scene_order_cell_adam_matches_definition():
    """vt_adam_step_cells_scene_order: site gradients and dL/drho =
    dL/dsigma * sigma (Eq. 4) from scene-order records, Adam in user order."""
    rng = np.random.default_rng(46)
    n = 5001
    perm = rng.permutation(n).astype(np.int32)
    sites = rng.normal(size=(n, 3)).astype(np.float32)
    rho = rng.normal(size=n).astype(np.float32)
    sigma = np.exp(rho).astype(np.float32)
    gc = rng.normal(size=(n, 4)).astype(np.float32)
    ts, tr_ = torch.as_tensor(sites, device=DEV).clone(), torch.as_tensor(rho, device=DEV).clone()
    z = [torch.zeros(n, 3, device=DEV), torch.zeros(n, 3, device=DEV), torch.zeros(n, device=DEV),
         torch.zeros(n, device=DEV)]
    # every device array the kernel reads stays referenced until it has run
    tperm, tgc, tsig = (torch.as_tensor(x, device=DEV) for x in (perm, gc, sigma))
    _vt.vt_adam_step_cells_scene_order(n, tperm.data_ptr(), tgc.data_ptr(), ts.data_ptr(), tr_.data_ptr(),
                                       tsig.data_ptr(), *[x.data_ptr() for x in z], 2e-3, 5e-2, 0.9, 0.999, 1e-15, 1,
                                       _st())
    torch.cuda.synchronize()
    gs_u = np.empty((n, 3))
    gs_u[perm] = gc[:, :3]
    gr_u = np.empty(n)
    gr_u[perm] = gc[:, 3] * sigma[perm]
    rs = TR.adam(sites, gs_u, np.zeros((n, 3)), np.zeros((n, 3)), 2e-3, 0.9, 0.999, 1e-15, 1)[0]
    rr = TR.adam(rho, gr_u, np.zeros(n), np.zeros(n), 5e-2, 0.9, 0.999, 1e-15, 1)[0]
    assert np.abs(ts.cpu().numpy() - rs).max() <= 2e-6
    assert np.abs(tr_.cpu().numpy() - rr).max() <= 2e-6


def test_fused_training_step_follows_the_unfused_one():
    """The trainer's default step (scene-order gradients into the fused Adam
    steps) against the step built from user-order gradients, separate
    regulariser, Eq. 4 and Adam kernels: the same losses over a few
    iterations and parameters that agree to float rounding."""
    init, cams, images, rp, gt = T.synthetic_problem(n_sites=3000, n_cams=4, w=48, h=32, tex_res=4, seed=5)
    out = {}
    for fused in (True, False):
        cfg = T.TrainConfig(iters=50, rays_per_iter=4096, refresh_every=0, vd_ramp_frac=0.0, seed=2,
                            scene_order_grads=fused)
        tr = T.Trainer(init["sites"], init["rho"], init["tex"], init["tex_vd"], cams, images, rp, cfg)
        out[fused] = ([tr.step(sync_loss=True) for _ in range(4)], {k: v.clone() for k, v in tr.p.items()})
        assert tr.scene.get_error()[0] == 0
    (la, pa), (lb, pb) = out[True], out[False]
    for a, b in zip(la, lb):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-7), (a, b)
    for k in pa:
        diff = (pa[k] - pb[k]).abs()
        scale = (pb[k] - torch.as_tensor(init[k], device=DEV)).abs().max().item()  # size of the updates
        # The gradient atomics sum in a different order on every run, and Adam
        # with eps = 1e-15 steps by about the learning rate whatever the
        # gradient's size, so a cell whose few rays' gradients nearly cancel
        # (textures start at zero, so L_mean adds nothing at first) can step
        # the other way in one run: all but a handful of cells agree to
        # rounding, and no entry moves by more than the updates themselves.
        off_cells = (diff.reshape(diff.shape[0], -1) > 1e-3 * scale + 1e-6).any(dim=1).float().mean().item()
        assert off_cells <= 3e-3 and diff.max().item() <= scale, (k, off_cells, diff.max().item(), scale)
