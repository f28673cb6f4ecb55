"""The allocation-free backward entry point, vt_render_bwd_static.

It exists for callers that may not allocate device memory during a step --
cudaMalloc can synchronise the device and bypasses an application's own
memory pool -- and accumulates into a fixed 32 MiB array inside libvt.so
instead of scratch allocated on first use. Called through the C ABI, its
gradients must match vt_render_bwd's within the gradient tolerance of the
parity tests, on two calls in a row (the shared array keeps the previous
call's contents, so the second call checks that it is cleared).

This file is named to be collected last: a run that stops at the first
failure has then already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2608_17682_gb300 import _vt, api  # noqa: E402
from paper_2608_17682_gb300 import workloads as W  # noqa: E402

GRAD_REL = 1e-3


def _close(a, ref, name):
    a = a.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    floor = 1e-3 * np.abs(ref).max()
    rel = np.abs(a - ref) / np.maximum(np.abs(ref), floor)
    assert rel.max() <= GRAD_REL, f"{name}: worst relative error {rel.max():.3g}"


def _static_bwd(scene, o, d, params, rgb, g):
    gs = torch.full((scene.n, 3), float("nan"), device="cuda")
    gsig = torch.full((scene.n,), float("nan"), device="cuda")
    gt = torch.full((scene.n, scene.R, scene.R, 3), float("nan"), device="cuda")
    _vt.vt_render_bwd_static(scene.handle, o.shape[0], o.data_ptr(), d.data_ptr(), 0, params, rgb.data_ptr(),
                             g.data_ptr(), gs.data_ptr(), gsig.data_ptr(), gt.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    return gs, gsig, gt


def test_static_backward_matches_allocating_backward_twice():
    wl = W.make_workload("tiny")
    o, d = W.workload_rays(wl)
    P = api.make_params(**wl.params, img_w=64, img_h=64, n_images=1)
    scene = api.Scene.from_workload(wl.scene)
    to = torch.as_tensor(o, device="cuda")
    td = torch.as_tensor(d, device="cuda")
    rgb = api.render_fwd(scene, to, td, P)[0]
    for call in range(2):
        g = torch.randn(len(o), 3, device="cuda", generator=torch.Generator("cuda").manual_seed(call))
        ref = api.render_bwd(scene, to, td, P, rgb, g)
        got = _static_bwd(scene, to, td, P, rgb, g)
        assert scene.get_error()[0] == 0
        for name, a, b in zip(("sites", "sigma", "tex"), got, ref):
            assert torch.isfinite(a).all()
            _close(a, b, f"call {call} {name}")


def test_static_backward_matches_the_oracle():
    """The same entry point against the FP64 oracle directly, on the rays
    outside the degenerate band (the others carry no gradient)."""
    import oracle as O

    wl = W.make_workload("tiny")
    o, d = W.workload_rays(wl)
    osc = O.OracleScene.from_workload_scene(wl.scene)
    op = O.make_params(**wl.params)
    flags = O.render(osc, o, d, params=op)[3]
    ok = (flags & O.BAND_FLAGS) == 0
    g = (np.random.default_rng(7).normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    P = api.make_params(**wl.params, img_w=64, img_h=64, n_images=1)
    scene = api.Scene.from_workload(wl.scene)
    to = torch.as_tensor(o, device="cuda")
    td = torch.as_tensor(d, device="cuda")
    rgb = api.render_fwd(scene, to, td, P)[0]
    got = _static_bwd(scene, to, td, P, rgb, torch.as_tensor(g, device="cuda"))
    assert scene.get_error()[0] == 0
    ref = O.render_bwd(osc, o, d, g.astype(np.float64), params=op)
    for name, a, b in zip(("sites", "sigma", "tex"), got, ref):
        _close(a, torch.as_tensor(b), f"oracle {name}")


def test_static_backward_rejects_scene_beyond_capacity():
    # 40,000 sites with 8x8 textures need 40,000 * 65 * 16 bytes > 32 MiB
    sc = W.make_scene("uniform", 40_000, 8, 31)
    scene = api.Scene.from_workload(sc)
    o = torch.zeros(4, 3, device="cuda")
    d = torch.tensor([[1.0, 0.0, 0.0]] * 4, device="cuda")
    P = api.make_params()
    rgb = api.render_fwd(scene, o, d, P)[0]
    g = torch.ones(4, 3, device="cuda")
    gs = torch.full((scene.n, 3), float("nan"), device="cuda")
    gsig = torch.full((scene.n,), float("nan"), device="cuda")
    gt = torch.full((scene.n, scene.R, scene.R, 3), float("nan"), device="cuda")
    with pytest.raises(_vt.VTError) as e:
        _vt.vt_render_bwd_static(scene.handle, o.shape[0], o.data_ptr(), d.data_ptr(), 0, P, rgb.data_ptr(),
                                 g.data_ptr(), gs.data_ptr(), gsig.data_ptr(), gt.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert e.value.status == _vt.VT_ERR_CAPACITY
    # a rejected call writes nothing
    torch.cuda.synchronize()
    assert torch.isnan(gs).all() and torch.isnan(gsig).all() and torch.isnan(gt).all()
