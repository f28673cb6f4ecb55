"""Host-side checks that need no GPU: the C-ABI library loads and exports every
symbol include/vt.h declares, host argument validation, workload inputs."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def vt():
    from paper_2608_17682_gb300 import build
    build.build()
    from paper_2608_17682_gb300 import _vt
    return _vt


def test_header_matches_binding_list(vt):
    assert _declared() == sorted(vt.EXPORTS)


def test_library_exports_every_declared_symbol(vt):
    out = subprocess.run(["nm", "-D", "--defined-only", vt.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in _declared() if s not in syms]
    assert not missing, missing
    for s in _declared():
        assert hasattr(vt.lib, s)


def test_status_strings_and_defaults(vt):
    assert vt.status_str(0) == "VT_OK"
    assert vt.status_str(4) == "VT_ERR_MAX_STEPS"
    p = vt.vt_render_params_default()
    assert p.t_near == 0 and p.t_far == 20 and abs(p.T_eps - 1e-4) < 1e-10 and list(p.bg) == [1, 1, 1]
    assert p.skip_weight == 0 and p.img_w == 0 and p.max_steps == 0


def test_host_argument_validation(vt):
    import ctypes as C
    out = C.c_void_p(123)
    assert vt.lib.vt_scene_create(None, None, C.byref(out)) == vt.VT_ERR_INVALID_ARG
    assert out.value is None
    d = vt.vt_scene_desc(0, 4, 0, 0, 0, 0, 0, 0, 0)
    assert vt.lib.vt_scene_create(C.byref(d), None, C.byref(out)) == vt.VT_ERR_INVALID_ARG
    d = vt.vt_scene_desc(10, 1, 0, 8, 8, 8, 8, 8, 0)  # tex_res < 2
    assert vt.lib.vt_scene_create(C.byref(d), None, C.byref(out)) == vt.VT_ERR_INVALID_ARG
    d = vt.vt_scene_desc(10, 4, 7, 8, 8, 8, 8, 8, 0)  # bad dtype
    assert vt.lib.vt_scene_create(C.byref(d), None, C.byref(out)) == vt.VT_ERR_INVALID_ARG
    cam = vt.vt_camera()
    cam.kind, cam.w, cam.h = 3, 4, 4
    cam.fwd[:] = [1, 0, 0]
    cam.up[:] = [0, 0, 1]
    cam.lens_samples = 3  # not a square
    arr = (vt.vt_camera * 1)(cam)
    assert vt.lib.vt_generate_rays(arr, 1, C.c_void_p(8), C.c_void_p(8), None, None) == vt.VT_ERR_INVALID_ARG
    cam.lens_samples = 4
    assert vt.vt_camera_n_rays(cam) == 64
    assert vt.lib.vt_render_fwd(None, 1, None, None, None, None, None, None, None, None, None,
                                None) == vt.VT_ERR_INVALID_ARG
    assert vt.lib.vt_sigma_from_rho(-1, None, None, None) == vt.VT_ERR_INVALID_ARG
    assert vt.lib.vt_sigma_from_rho_bwd(3, None, None, None, None) == vt.VT_ERR_INVALID_ARG
    cam.kind, cam.lens_samples = 4, 0  # motion blur needs >= 1 time sample
    arr = (vt.vt_camera * 1)(cam)
    assert vt.lib.vt_generate_rays(arr, 1, C.c_void_p(8), C.c_void_p(8), None, None) == vt.VT_ERR_INVALID_ARG
    assert vt.lib.vt_l2_loss(-1, None, None, None, None, None) == vt.VT_ERR_INVALID_ARG
    assert vt.lib.vt_average_samples(4, 0, None, None, None) == vt.VT_ERR_INVALID_ARG


def test_workload_csr_is_a_valid_delaunay_graph():
    from paper_2608_17682_gb300 import workloads as W
    sc = W.make_scene("uniform", 3000, 4, 5)
    off, idx = sc.offsets, sc.indices
    n = sc.n
    assert off[0] == 0 and off[-1] == len(idx) and np.all(np.diff(off) > 0)
    rows = np.repeat(np.arange(n), np.diff(off))
    assert np.all(idx != rows) and idx.min() >= 0 and idx.max() < n
    e = set(zip(rows.tolist(), idx.tolist()))
    assert all((j, i) in e for i, j in e)
    assert 13 < len(idx) / n < 17  # mean Delaunay degree of a random 3-D point set is about 15.5


def test_surface_workload_recipe():
    from paper_2608_17682_gb300 import workloads as W
    rng = np.random.default_rng(0)
    pts, surf = W.surface_sites(20000, rng)
    r = np.linalg.norm(pts.astype(np.float64), axis=1)
    assert abs(surf.mean() - 0.7) < 1e-3
    shell = r > 3.9
    assert abs(shell.mean() - 0.1) < 1e-3 and r[shell].max() <= 8.0 + 1e-5
    inner = ~surf & ~shell
    assert np.all(np.abs(pts[inner]) <= 1.0)


def test_camera_set_of_mixed_workload():
    from paper_2608_17682_gb300 import workloads as W
    cams = W.workload_cameras("mixed3m")
    assert [c.kind for c in cams] == [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4
    assert sum(c.n_rays for c in cams) == 29_818_880
    cams = W.workload_cameras("prec3m")
    assert sum(c.n_rays for c in cams) == 4 * 1280 * 832


def test_learning_rate_schedules():
    """The appendix's schedules: cosine decays, linear density warm-up over the
    first 10%, sites fixed for the last 10%, quadratic view-dependent ramp."""
    from paper_2608_17682_gb300 import train as T

    cfg = T.TrainConfig(iters=20_000)
    a = T.learning_rates(cfg, 0)
    assert abs(a["sites"] - 2e-4) < 1e-12 and abs(a["tex"] - 2e-2) < 1e-12
    assert a["tex_vd"] == 0.0  # quadratic ramp starts at zero
    assert abs(T.learning_rates(cfg, 999)["rho"] - 0.05) < 1e-12  # linear warm-up over 2,000 iterations
    assert abs(T.learning_rates(cfg, 2000)["rho"] - 0.1) < 1e-12
    assert abs(T.learning_rates(cfg, 4000)["tex_vd"] - T.learning_rates(cfg, 4000)["tex"]) < 1e-15
    assert T.learning_rates(cfg, 18_000)["sites"] == 0.0  # sites fixed for the last 2,000 iterations
    assert abs(T.learning_rates(cfg, 19_999)["tex"] - 5e-4) < 1e-6


def test_traffic_record_survives_comment_edits(tmp_path):
    """bench.py keys recorded DRAM traffic to the kernel sources' code: a
    comment edit keeps the record, a code edit drops it."""
    import shutil
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    src = os.path.join(bench.ROOT, "paper_2608_17682_gb300", "csrc")
    dst = tmp_path / "paper_2608_17682_gb300" / "csrc"
    shutil.copytree(src, dst)
    (tmp_path / "profiles").mkdir()
    old_root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        h = bench.kernel_source_hash()
        (tmp_path / "profiles" / "x.md").write_text(f"TRAFFIC k_walk<BWD,f16> prec3m 123 {h}\n")
        assert bench.recorded_traffic("k_walk<BWD,f16>", "prec3m") == 123
        assert bench.recorded_traffic("k_walk<BWD,f32>", "prec3m") is None
        f = dst / "vt_render.cu"
        f.write_text(f.read_text() + "\n// a comment\n/* another */\n")
        assert bench.kernel_source_hash() == h
        f.write_text(f.read_text() + "\nstatic int extra_symbol_for_test;\n")
        assert bench.kernel_source_hash() != h
        assert bench.recorded_traffic("k_walk<BWD,f16>", "prec3m") is None
    finally:
        bench.ROOT = old_root


def test_reference_arm_json_line():
    """bench.py --impl reference times the oracle on the host and prints one
    JSON line with the contract's keys (runs without a GPU)."""
    import json
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1",
                          "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["unit"] == "Mrays/s" and j["value"] > 0 and j["higher_is_better"]
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["value"] == j["value"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    assert j["steps"] == 1 and j["warmup"] == 1 and j["n_gpus"] == 1
    # the same metric and workload names as the CUDA arm's line
    sys.path.insert(0, root)
    import bench
    from paper_2608_17682_gb300 import workloads as W
    args = bench.parse(["--workload", "tiny"])
    wl = W.make_workload("tiny")
    assert j["metric"] == bench.metric_name(args)
    assert j["config"]["workload"] == bench.workload_name(args, wl, bench.rank_cameras(wl, 0))


def test_api_rejects_tensors_the_kernels_cannot_take():
    """Tensors reach the kernels as raw pointers, so api.py checks device,
    dtype, shape and contiguity first and raises before any library call."""
    import types
    import torch
    from paper_2608_17682_gb300 import api
    from paper_2608_17682_gb300 import workloads as W
    scene = types.SimpleNamespace(handle=0, n=5, R=4, has_tex_vd=False, device=torch.device("cpu"))
    P = api.make_params()
    cpu = torch.zeros(4, 3)
    for call in (lambda: api.render_fwd(scene, cpu, cpu, P),
                 lambda: api.render_bwd(scene, cpu, cpu, P, cpu, cpu),
                 lambda: api.trace_cells(scene, cpu, cpu, P),
                 lambda: api.l2_loss(cpu, cpu),
                 lambda: api.average_samples(cpu, 2),
                 lambda: api.average_samples_bwd(cpu, 2),
                 lambda: api.sigma_from_rho(torch.zeros(5)),
                 lambda: api.sigma_from_rho_bwd(torch.zeros(5), torch.zeros(5)),
                 lambda: api.generate_rays([W.look_at_camera(0, 2, 2, (0.0, -2.0, 0.0), (0.0, 0.0, 0.0))],
                                           out=(cpu, cpu, torch.zeros(4)))):
        with pytest.raises(ValueError):
            call()
    with pytest.raises(ValueError):  # not a multiple of the sample count
        api.average_samples(torch.zeros(10, 3), 4)
    # the checker itself: dtype, shape and contiguity come before the device
    with pytest.raises(ValueError, match="float32"):
        api._arr(torch.zeros(4, 3, dtype=torch.float64), "x", (4, 3))
    with pytest.raises(ValueError, match="shape"):
        api._arr(torch.zeros(4, 4), "x", (4, 3))
    with pytest.raises(ValueError, match="contiguous"):
        api._arr(torch.zeros(3, 4).t(), "x", (4, 3))
    with pytest.raises(ValueError, match="CUDA"):
        api._arr(torch.zeros(4, 3), "x", (4, 3))
    with pytest.raises(ValueError, match="required"):
        api._arr(None, "x", (4, 3))
    api._arr(None, "x", (4, 3), optional=True)


def test_oracle_and_cuda_path_share_no_code():
    """The oracle includes only the C standard library and imports only numpy
    and its own modules; the product package and the CUDA sources never name
    the oracle. Only the seeded input generators (workloads.py) serve both."""
    import glob
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    c_src = open(os.path.join(root, "oracle", "vt_oracle.c")).read()
    assert set(re.findall(r'#include\s*[<"]([^>"]+)[>"]', c_src)) <= {"math.h", "pthread.h", "stdint.h", "stdlib.h",
                                                                      "string.h"}
    for f in glob.glob(os.path.join(root, "oracle", "*.py")):
        mods = re.findall(r"^\s*(?:from|import)\s+([\w.]+)", open(f).read(), re.M)
        assert all(m.split(".")[0] in {"__future__", "ctypes", "os", "subprocess", "numpy", "math"} or m == "."
                   for m in mods), (f, mods)
    product = glob.glob(os.path.join(root, "paper_2608_17682_gb300", "*.py")) + \
        glob.glob(os.path.join(root, "paper_2608_17682_gb300", "csrc", "*")) + glob.glob(os.path.join(root, "include", "*"))
    for f in product:
        text = open(f, errors="replace").read()
        assert not re.search(r"^\s*(from|import)\s+oracle|vt_oracle|libvt_oracle|\bvto_", text, re.M), f


def test_density_and_texture_recipes():
    """The stated input recipe: uniform scenes with sigma = exp(N(0, 1.5^2)),
    surface scenes with exp(N(3,1)) on the 70% surface sites and exp(N(-2,1))
    elsewhere, textures U[0,1]."""
    from paper_2608_17682_gb300 import workloads as W
    sc = W.make_scene("uniform", 4000, 4, 11)
    ls = np.log(sc.sigma.astype(np.float64))
    assert abs(ls.mean()) < 0.1 and abs(ls.std() - 1.5) < 0.1
    assert np.all((sc.sites >= 0) & (sc.sites <= 1))
    assert sc.tex.min() >= 0 and sc.tex.max() <= 1 and abs(sc.tex.mean() - 0.5) < 0.01
    sc = W.make_scene("surface", 20000, 4, 12)
    ls = np.log(sc.sigma.astype(np.float64))
    # a two-component mixture: 0.7 N(3,1) + 0.3 N(-2,1)
    assert abs(ls.mean() - (0.7 * 3.0 + 0.3 * -2.0)) < 0.05
    from math import erf, sqrt
    above = 0.7 * 0.5 * (1 + erf(2.5 / sqrt(2))) + 0.3 * 0.5 * (1 - erf(2.5 / sqrt(2)))
    assert abs((ls > 0.5).mean() - above) < 0.01


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "vt.h"

int main(void) {
  vt_render_params p;
  memset(&p, 0xff, sizeof(p));
  vt_render_params_default(&p);
  vt_camera c;
  memset(&c, 0, sizeof(c));
  c.kind = VT_CAM_THIN_LENS;
  c.w = 12;
  c.h = 10;
  c.lens_samples = 4;
  vt_scene* s = (vt_scene*)0;
  /* host-side argument checks only: nothing here reaches a GPU */
  vt_status st = vt_render_fwd(s, 1, 0, 0, 0, &p, 0, 0, 0, 0, 0, 0);
  printf("%g %g %g %d %lld %s %s\n", p.t_near, p.t_far, p.T_eps, p.appearance, (long long)vt_camera_n_rays(&c),
         vt_status_str(VT_OK), vt_status_str(st));
  return 0;
}
"""


def test_plain_c_client_compiles_links_and_calls_the_abi(vt, tmp_path):
    """include/vt.h is plain C: a C11 program includes it, links libvt.so and
    calls the entry points that need no GPU."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(vt.LIB_PATH)
    cuda_lib = "/usr/local/cuda/lib64"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-l:libvt.so",
                           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}", f"-L{cuda_lib}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    t_near, t_far, T_eps, app, n_rays, ok, err = out.stdout.split()
    assert (float(t_near), float(t_far), float(T_eps), int(app)) == (0.0, 20.0, 1e-4, 0)
    assert int(n_rays) == 12 * 10 * 4
    assert ok == "VT_OK" and err == "VT_ERR_INVALID_ARG"  # a NULL scene is rejected on the host


def test_missing_library_fails_loudly():
    """Without libvt.so the package raises on import: there is no CPU
    fallback for the renderer."""
    env = dict(os.environ, VT_LIB_PATH=os.path.join(ROOT, "no-such-dir", "libvt.so"))
    out = subprocess.run([sys.executable, "-c", "from paper_2608_17682_gb300 import api"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode != 0 and "ImportError" in out.stderr and "no CPU fallback" in out.stderr
