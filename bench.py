"""Benchmark: Mrays/s of the differentiable Voronoi ray-traversal renderer.

One step = one pass of the whole hot path over one batch of views: ray
generation -> start-cell search -> forward walk/composite -> L2 loss ->
backward re-traversal with gradient atomics (sites, sigma, texels).

Default workload "prec3m": 3,000,000 surface-concentrated sites with 8x8
octahedral textures, four 1280x832 pinhole cameras (4,259,840 rays), textures
stored in FP16 (the headline) and also timed in FP32 and BF16. Inputs are
synthetic and seeded (the paper's Mip-NeRF 360 scenes are not available).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch under torch.distributed.run; each rank renders its own
views of the same scene (weak scaling, no collective in the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_17682_gb300 import workloads as W  # noqa: E402

METRIC = "Mrays/s fwd+bwd (FP16 textures)"
HBM_FALLBACK_GBS = 6800.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="prec3m", choices=list(W.WORKLOADS))
    ap.add_argument("--sites", type=int, default=0, help="override the site count (smaller runs)")
    ap.add_argument("--tex", default="f16", choices=["f16", "f32", "bf16"])
    ap.add_argument("--no-extra", action="store_true", help="skip the FP32/BF16 comparison timings")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--appearance", type=int, default=0, choices=[0, 1],
                    help="1: time the paper's two-texture appearance model as the main step")
    ap.add_argument("--skip-sweep", action="store_true",
                    help="forward-only timing and image change for cell-skip thresholds 0 ... 1e-2")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the forward pass with the inference-stack toggles (Morton order, 4x8 tiles, "
                         "cell skip 1e-3), cumulatively as in the paper's Sec. 6.3 ablation")
    return ap.parse_args(argv)


def metric_name(args):
    """The metric of the line: Mrays/s fwd+bwd, named for the texture storage
    type and the appearance model timed."""
    m = METRIC if args.tex == "f16" else METRIC.replace("FP16", args.tex.upper())
    return m + (", paper appearance model" if args.appearance else "")


def workload_name(args, wl, cams):
    """The workload one rank renders, by size (the `config.workload` key)."""
    c0 = cams[0]
    n_rays = sum(c.n_rays for c in cams)
    return (f"{args.workload}: {wl.scene.n} sites, {wl.scene.R}x{wl.scene.R} {args.tex} textures"
            f"{' (two maps, sigmoid)' if args.appearance else ''}, "
            f"{len(cams)} x {c0.w}x{c0.h} cameras, {n_rays} rays/GPU")


def appearance_maps(wl):
    """Logit maps (T_vi, T_vd) of the paper's appearance model for the
    workload, seed 5000+k."""
    rng_app = np.random.default_rng(5000 + wl.seed)
    tvd = rng_app.normal(0.0, 0.5, size=wl.scene.tex.shape).astype(np.float32)
    tvi = rng_app.normal(0.0, 1.5, size=wl.scene.tex.shape).astype(np.float32)
    return tvi, tvd


def oracle_setup(args, wl):
    """The oracle's copy of the timed scene and its render parameters."""
    import oracle as O

    if args.appearance:
        tvi, tvd = appearance_maps(wl)
        sc = wl.scene
        return (O.OracleScene(sc.sites, sc.sigma, tvi, sc.offsets, sc.indices, tex_vd=tvd),
                O.make_params(**wl.params, appearance=1))
    return O.OracleScene.from_workload_scene(wl.scene), O.make_params(**wl.params)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_cameras(wl, rank):
    """Weak scaling: rank r renders the workload's views rotated by r*7.5 deg."""
    if rank == 0:
        return wl.cameras
    cams = []
    for c in wl.cameras:
        eye = np.asarray(c.eye)
        a = math.radians(7.5 * rank)
        R = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
        e2 = R @ eye
        f2 = R @ np.asarray(c.fwd)
        cams.append(W.Camera(**{**c.__dict__, "eye": tuple(e2), "fwd": tuple(f2)}))
    return cams


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def _code_only(text):
    """Source text without comments and blank space, so that a comment edit
    does not count as a kernel change."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash():
    """Hash of the code (comments and spacing ignored) of the translation
    unit that holds the walk kernels and the gradient permute, and of its
    internal header: the sources the recorded ncu figures depend on."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2608_17682_gb300", "csrc")
    for f in ("vt_internal.cuh", "vt_render.cu"):
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            h.update(f.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summaries under profiles/
    (lines "TRAFFIC <kernel> <workload> <bytes> <source hash>"), if they were
    taken on the current kernel sources (else None)."""
    d = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(d))
    except OSError:
        return None
    h = kernel_source_hash()
    for n in names:
        if not n.endswith(".md"):
            continue
        with open(os.path.join(d, n)) as f:
            for line in f:
                w = line.split()
                if len(w) == 5 and w[0] == "TRAFFIC" and w[1] == kernel and w[2] == workload and w[4] == h:
                    return int(w[3])
    return None


def recorded_issue(kernel):
    """Issue-slot activity (fraction of cycles a warp instruction issued) of
    the kernel from the committed ncu summaries (lines "ISSUE <kernel>
    <workload> <fraction> <source hash>", taken on a smaller workload than the
    benchmark's because the metric needs several ncu passes), on the current
    sources only: {"value", "workload"} or None."""
    d = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(d))
    except OSError:
        return None
    h = kernel_source_hash()
    for n in names:
        if not n.endswith(".md"):
            continue
        with open(os.path.join(d, n)) as f:
            for line in f:
                w = line.split()
                if len(w) == 5 and w[0] == "ISSUE" and w[1] == kernel and w[4] == h:
                    return {"value": float(w[3]), "workload": w[2]}
    return None


def l2_bandwidth(torch, dev, stream):
    """L2 read bandwidth: vt_stream_read over buffers that fit in the 129 MB
    L2, repeated in one kernel, CUDA events; the best over the sizes. Also the
    same probe over a 4 GB buffer (HBM read bandwidth) for context."""
    from paper_2608_17682_gb300 import _vt

    sink = torch.zeros(1, device=dev)
    out = {}
    best = 0.0
    for mb in (24, 48, 96):
        buf = torch.ones(mb * (1 << 20) // 4, device=dev)
        reps = max(4, int(64e9 // buf.numel() // 4 // 4))  # about 16 GB read per timing
        _vt.vt_stream_read(buf.data_ptr(), buf.numel() * 4, 2, sink.data_ptr(), stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _vt.vt_stream_read(buf.data_ptr(), buf.numel() * 4, reps, sink.data_ptr(), stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        gbs = buf.numel() * 4 * reps / (a.elapsed_time(b) * 1e-3) / 1e9
        out[f"{mb}MB"] = round(gbs, 1)
        best = max(best, gbs)
        del buf
    big = torch.ones((4 << 30) // 4, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    _vt.vt_stream_read(big.data_ptr(), big.numel() * 4, 3, sink.data_ptr(), stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    hbm = big.numel() * 4 * 3 / (a.elapsed_time(b) * 1e-3) / 1e9
    del big
    return {"l2_read_gbs": round(best, 1), "by_buffer": out, "hbm_read_gbs_4GB": round(hbm, 1)}


# ---------------------------------------------------------------- our arm

def run_ours(args, ws, rank, local):
    import torch

    from paper_2608_17682_gb300 import _vt, api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    wl = W.make_workload(args.workload, n_sites=args.sites or None)
    cams = rank_cameras(wl, rank)
    n_img = len(cams)
    c0 = cams[0]
    spp = c0.spp
    n_rays = sum(c.n_rays for c in cams)
    uniform = all(c.w == c0.w and c.h == c0.h and c.n_rays == c0.n_rays for c in cams)
    if uniform:
        layout = dict(img_w=c0.w * spp, img_h=c0.h, n_images=n_img)
    else:  # one launch over images of different sizes (lens samples widen a row)
        layout = dict(image_sizes=[(c.w * c.spp, c.h) for c in cams])
    params = api.make_params(**wl.params, **layout, appearance=args.appearance)
    Y = torch.as_tensor(W.target_image(n_rays, wl.seed), device=dev)

    # the paper's appearance model (Sec. 5.1-5.2): two maps of logits, sigmoid
    tvi, tvd = appearance_maps(wl)

    def make_scene(t, appearance, **kw):
        if appearance:
            return api.Scene(wl.scene.sites, wl.scene.sigma, tvi, wl.scene.offsets, wl.scene.indices, tex_dtype=t,
                             device=dev, tex_vd=tvd, **kw)
        return api.Scene.from_workload(wl.scene, tex_dtype=t, device=dev, **kw)

    scenes = {}
    dtypes = [args.tex] + ([] if args.no_extra else [t for t in ("f32", "bf16", "f16") if t != args.tex])
    for t in dtypes:
        scenes[t] = make_scene(t, args.appearance)
    stream = torch.cuda.current_stream()
    o = torch.empty(n_rays, 3, device=dev)
    d = torch.empty(n_rays, 3, device=dev)
    tm = torch.empty(n_rays, device=dev)
    rgb = torch.empty(n_rays, 3, device=dev)
    T = torch.empty(n_rays, device=dev)
    steps = torch.empty(n_rays, dtype=torch.int32, device=dev)
    res = torch.empty(n_rays, 3, device=dev)  # float-float residual of the colour, for the backward
    N, R = wl.scene.n, wl.scene.R
    gs = torch.empty(N, 3, device=dev)
    gsig = torch.empty(N, device=dev)
    gt = torch.empty(N, R, R, 3, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)  # 256 MB > 129 MB L2

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def walk_events(pair):
        """Make the library record `pair` around its next walk kernel."""
        params.walk_events[0] = pair[0].cuda_event if pair else None
        params.walk_events[1] = pair[1].cuda_event if pair else None

    def step(scene, marks=None, fwd_only=False, scene_order=False):
        # marks: 4 events around the fwd / bwd calls, then 4 the library
        # records around the forward and backward walk kernels themselves
        api.generate_rays(cams, out=(o, d, tm))
        if marks:
            marks[0].record(stream)
            walk_events(marks[4:6])
        api.render_fwd(scene, o, d, params, time=tm, out=(rgb, T, steps), residual=None if fwd_only else res)
        walk_events(None)
        if marks:
            marks[1].record(stream)
        if fwd_only:
            return
        loss, grad = api.l2_loss(rgb, Y)
        if marks:
            marks[2].record(stream)
            walk_events(marks[6:8])
        if scene_order:  # gradients left in the scene's cell order (no permute)
            api.render_bwd_scene_order(scene, o, d, params, rgb, grad, time=tm, residual=res)
        else:
            api.render_bwd(scene, o, d, params, rgb, grad, time=tm, out=(gs, gsig, gt), residual=res)
        walk_events(None)
        if marks:
            marks[3].record(stream)
        return loss

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(scene, K, fwd_only=False, walks=None, scene_order=False):
        """K steps, L2 flushed between steps (outside the timed events). If
        `walks` is a dict it receives the mean forward / backward walk-kernel
        times (events recorded by the library around the kernel launches)."""
        for _ in range(args.warmup):
            step(scene, fwd_only=fwd_only, scene_order=scene_order)
        barrier()
        st, en, marks = [], [], []
        for _ in range(K):
            flush.zero_()
            a, b = ev(), ev()
            m = [ev() for _ in range(8)]
            for e in m[4:]:
                e.record(stream)  # creates the event handle the library records into
            a.record(stream)
            step(scene, m, fwd_only=fwd_only, scene_order=scene_order)
            b.record(stream)
            st.append(a)
            en.append(b)
            marks.append(m)
        barrier()
        per_step = [x.elapsed_time(y) for x, y in zip(st, en)]
        total = sum(per_step)
        fwd = sum(m[0].elapsed_time(m[1]) for m in marks) / K
        bwd = 0.0 if fwd_only else sum(m[2].elapsed_time(m[3]) for m in marks) / K
        if walks is not None:
            walks["fwd"] = sum(m[4].elapsed_time(m[5]) for m in marks) / K
            walks["bwd"] = 0.0 if fwd_only else sum(m[6].elapsed_time(m[7]) for m in marks) / K
            walks["step_median"] = statistics.median(per_step)
        return total / K, fwd, bwd

    main = scenes[args.tex]
    clocks = ClockSampler(local)
    clocks.start()
    walks = {}
    launches0 = _vt.vt_kernel_launches()
    ms_step, ms_fwd, ms_bwd = timed(main, args.steps, walks=walks)
    # the library's own kernel launches per step, counted by the library
    # (warm-up and timed steps are identical)
    launches_per_step = (_vt.vt_kernel_launches() - launches0) / (args.warmup + args.steps)
    clk = clocks.stop()
    grads_main = [x.clone() for x in (gs, gsig, gt)] if not args.no_extra else None
    # the max over ranks
    if ws > 1:
        t = torch.tensor([ms_step], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = t.item()
    err, fp64 = main.get_error()
    if err:
        raise RuntimeError(f"kernel error {err}")
    sum_steps = int(steps.long().sum().item())
    total_rays = n_rays * ws
    value = total_rays / (ms_step * 1e-3) / 1e6

    # forward-only and other texture precisions (context keys)
    extra = {}
    ms_f, fwd_only_fwd, _ = timed(main, max(3, args.steps // 2), fwd_only=True)
    extra["fwd_only_mrays_s"] = round(n_rays / (ms_f * 1e-3) / 1e6 * ws, 2)
    # the same step with the gradients left in the scene's cell order
    # (vt_render_bwd_scene_order: no permute to user order)
    w_so = {}
    m_s, m_f, m_b = timed(main, max(3, args.steps // 2), walks=w_so, scene_order=True)
    extra["scene_order_grads"] = {"fwd_bwd_mrays_s": round(n_rays / (m_s * 1e-3) / 1e6 * ws, 2),
                                  "ms_bwd": round(m_b, 3), "ms_bwd_walk_kernel": round(w_so["bwd"], 4),
                                  "ms_bwd_outside_walk": round(m_b - w_so["bwd"], 4)}
    grads_by_dtype = {args.tex: grads_main}
    for t in dtypes[1:]:
        w_t = {}
        m_s, m_f, m_b = timed(scenes[t], max(3, args.steps // 2), walks=w_t)
        extra[t] = {"fwd_bwd_mrays_s": round(n_rays / (m_s * 1e-3) / 1e6 * ws, 2), "ms_fwd": round(m_f, 3),
                    "ms_bwd": round(m_b, 3), "ms_walk_kernel": {"fwd": round(w_t["fwd"], 4),
                                                                "bwd": round(w_t["bwd"], 4)}}
        grads_by_dtype[t] = [x.clone() for x in (gs, gsig, gt)]
    # FP16 against FP32 textures, interleaved: three rounds of both, so that
    # the comparison carries its run-to-run spread
    if "f32" in scenes and args.tex != "f32":
        rounds = {args.tex: [], "f32": []}
        for _ in range(3):
            for t in (args.tex, "f32"):
                rounds[t].append(n_rays / (timed(scenes[t], max(3, args.steps // 2))[0] * 1e-3) / 1e6 * ws)
        extra["tex_vs_f32_interleaved"] = {
            t: {"median_mrays_s": round(statistics.median(v), 2), "min": round(min(v), 2), "max": round(max(v), 2)}
            for t, v in rounds.items()}
        extra["tex_vs_f32_interleaved"]["median_ratio"] = round(
            statistics.median(rounds[args.tex]) / statistics.median(rounds["f32"]), 4)
    # gradients of the same L2 step with each texture storage against the FP32 kernel's
    if "f32" in grads_by_dtype and grads_by_dtype["f32"] is not None:
        ref = grads_by_dtype["f32"]
        for t, gg in grads_by_dtype.items():
            if t == "f32" or gg is None:
                continue
            extra.setdefault(t, {})["grad_vs_f32_kernel"] = {
                name: round(((a.double() - b.double()).norm() / b.double().norm()).item(), 6)
                for name, a, b in zip(("sites", "sigma", "tex"), gg, ref)}
    del grads_by_dtype, grads_main

    # region 3 of the timing protocol: the torch.autograd.Function path
    # (VTRender.apply, an L2 loss in torch ops, loss.backward())
    if not args.appearance:
        sites_t = torch.tensor(wl.scene.sites, device=dev, requires_grad=True)
        sigma_t = torch.tensor(wl.scene.sigma, device=dev, requires_grad=True)
        tex_t = torch.tensor(wl.scene.tex, device=dev, requires_grad=True)

        def autograd_step():
            for p_ in (sites_t, sigma_t, tex_t):
                p_.grad = None
            api.generate_rays(cams, out=(o, d, tm))
            img = api.render(sites_t, sigma_t, tex_t, o, d, main, params)
            loss_ = ((img - Y) ** 2).mean()
            loss_.backward()

        for _ in range(args.warmup):
            autograd_step()
        barrier()
        reps, tot = max(3, args.steps // 2), 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            autograd_step()
            b.record(stream)
            barrier()
            tot += a.elapsed_time(b)
        extra["autograd_region"] = {"fwd_bwd_mrays_s": round(n_rays / (tot / reps * 1e-3) / 1e6 * ws, 2),
                                    "ms_per_step": round(tot / reps, 3),
                                    "what": "VTRender.apply + torch L2 loss + loss.backward(), ray generation "
                                            "included, L2 flushed between steps"}
        del sites_t, sigma_t, tex_t
    if not args.no_extra:
        # the other appearance model as a comparison line
        other = 1 - args.appearance
        sc_app = make_scene(args.tex, other)
        params_main = params
        params = api.make_params(**wl.params, **layout, appearance=other)
        m_s, m_f, m_b = timed(sc_app, max(3, args.steps // 2))
        extra[f"appearance{other}"] = {"fwd_bwd_mrays_s": round(n_rays / (m_s * 1e-3) / 1e6 * ws, 2),
                                       "ms_fwd": round(m_f, 3), "ms_bwd": round(m_b, 3), "tex": args.tex}
        params = params_main
        sc_app.close()
        # inference with FP16 neighbour offsets (Sec. 5.6): forward only
        sc_h = make_scene(args.tex, args.appearance, half_offsets=True)
        api.generate_rays(cams, out=(o, d, tm))
        api.render_fwd(main, o, d, params, time=tm, out=(rgb, T, steps))
        ref_img = rgb.clone()
        ms_h, _, _ = timed(sc_h, max(3, args.steps // 2), fwd_only=True)
        mse = ((rgb.double() - ref_img.double()) ** 2).mean().item()
        extra["half_offsets_fwd"] = {"fwd_only_mrays_s": round(n_rays / (ms_h * 1e-3) / 1e6 * ws, 2),
                                     "psnr_vs_fp32_offsets_db": None if mse == 0 else round(-10 * math.log10(mse), 2),
                                     "max_abs_diff": round((rgb - ref_img).abs().max().item(), 6)}
        sc_h.close()
        del ref_img
        # training step with the distortion loss (Eq. 2) fused into both passes
        dist = torch.empty(n_rays, 3, device=dev)
        gdist = torch.full((n_rays,), 1e-2 / n_rays, device=dev)

        def step_dist():
            api.generate_rays(cams, out=(o, d, tm))
            api.render_fwd(main, o, d, params, time=tm, out=(rgb, T, steps), residual=res, dist=dist)
            loss, grad = api.l2_loss(rgb, Y)
            api.render_bwd(main, o, d, params, rgb, grad, time=tm, out=(gs, gsig, gt), residual=res, dist=dist,
                           grad_dist=gdist)

        for _ in range(args.warmup):
            step_dist()
        barrier()
        reps, tot = max(3, args.steps // 2), 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            step_dist()
            b.record(stream)
            barrier()
            tot += a.elapsed_time(b)
        extra["distortion_loss"] = {"fwd_bwd_mrays_s": round(n_rays / (tot / reps * 1e-3) / 1e6 * ws, 2),
                                    "mean_L_dist": round(dist[:, 0].double().mean().item(), 6)}
        del dist, gdist
        # one optimisation iteration of the training loop (Eq. 5 with the paper's
        # appearance model, distortion loss, regularisers, Adam; no Delaunay refresh)
        from paper_2608_17682_gb300 import train as TRN

        rng = np.random.default_rng(6000 + wl.seed)
        cfg = TRN.TrainConfig(iters=1000, rays_per_iter=1 << 20, refresh_every=0)
        tr = TRN.Trainer(wl.scene.sites, np.log(np.maximum(wl.scene.sigma, 1e-6)),
                         rng.normal(0.0, 1.0, size=wl.scene.tex.shape).astype(np.float32),
                         np.zeros(wl.scene.tex.shape, np.float32), cams, Y, dict(wl.params), cfg, device=dev,
                         offsets=wl.scene.offsets, indices=wl.scene.indices)
        for _ in range(args.warmup):
            tr.step()
        barrier()
        reps = max(3, args.steps // 2)
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            tr.step()
        b.record(stream)
        barrier()
        ms_it = a.elapsed_time(b) / reps
        st_, _ = tr.scene.get_error()
        extra["train_iteration"] = {"rays_per_iter": tr.B, "ms_per_iter": round(ms_it, 3),
                                    "mrays_s": round(tr.B / (ms_it * 1e-3) / 1e6, 2), "kernel_status": st_,
                                    "note": "sigma=exp(rho), sampling, fwd+bwd (appearance 1, distortion), "
                                            "Smooth-L1, gradients left in scene order and consumed by fused Adam "
                                            "steps (regularisers and Eq. 4 inside); L2 not flushed"}
        tr.scene.close()
        del tr

    if args.ablation:
        # cumulative: user order + row-major 1-D rays -> + Morton -> + 4x8 tiles -> + skip 1e-3
        base_scene = make_scene(args.tex, args.appearance, keep_order=True)
        p_1d = api.make_params(**wl.params, appearance=args.appearance)
        p_skip = api.make_params(**{**wl.params, "skip_weight": 1e-3}, **layout, appearance=args.appearance)
        rows = []
        for name, sc_, pp in (("base", base_scene, p_1d), ("+morton", main, p_1d), ("+tiles", main, params),
                              ("+skip1e-3", main, p_skip)):
            for _ in range(args.warmup):
                api.generate_rays(cams, out=(o, d, tm))
                api.render_fwd(sc_, o, d, pp, time=tm, out=(rgb, T, steps))
            barrier()
            tot = 0.0
            for _ in range(max(3, args.steps // 2)):
                flush.zero_()
                a, b = ev(), ev()
                a.record(stream)
                api.render_fwd(sc_, o, d, pp, time=tm, out=(rgb, T, steps))
                b.record(stream)
                barrier()
                tot += a.elapsed_time(b)
            ms = tot / max(3, args.steps // 2)
            rows.append({"config": name, "ms_fwd": round(ms, 3), "mrays_s": round(n_rays / (ms * 1e-3) / 1e6, 1),
                         "fps": round(n_img / (ms * 1e-3), 1)})
        extra["ablation_fwd"] = rows
        del base_scene

    if args.skip_sweep:
        # inference speed / quality trade-off of the low-contribution cell skip
        # (Sec. 5.6): PSNR of each image against the unskipped render
        rows = []
        exact = None
        for thr in (0.0, 1e-5, 1e-4, 3e-4, 1e-3, 3e-3, 1e-2):
            pp = api.make_params(**{**wl.params, "skip_weight": thr}, **layout, appearance=args.appearance)
            for _ in range(args.warmup):
                api.generate_rays(cams, out=(o, d, tm))
                api.render_fwd(main, o, d, pp, time=tm, out=(rgb, T, steps))
            barrier()
            tot = 0.0
            reps = max(3, args.steps // 2)
            for _ in range(reps):
                flush.zero_()
                a, b = ev(), ev()
                a.record(stream)
                api.render_fwd(main, o, d, pp, time=tm, out=(rgb, T, steps))
                b.record(stream)
                barrier()
                tot += a.elapsed_time(b)
            ms = tot / reps
            img = rgb.double()
            if exact is None:
                exact = img.clone()
            mse = ((img - exact) ** 2).mean().item()
            psnr = None if mse == 0 else round(10 * math.log10(1.0 / mse), 2)
            rows.append({"threshold": thr, "ms_fwd": round(ms, 3), "fps": round(n_img / (ms * 1e-3), 1),
                         "mrays_s": round(n_rays / (ms * 1e-3) / 1e6, 1), "psnr_vs_unskipped_db": psnr,
                         "max_abs_diff": round((img - exact).abs().max().item(), 6)})
        extra["skip_sweep_fwd"] = rows
        del exact

    # the same step captured once in a CUDA graph and replayed: one host
    # launch per step instead of the library's nine kernel launches and
    # memsets (the scratch was allocated by the earlier, uncaptured calls)
    try:
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(2):
                step(main)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph):
            step(main)
        for _ in range(args.warmup):
            graph.replay()
        barrier()
        reps, tot = max(3, args.steps), 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            graph.replay()
            b.record(stream)
            barrier()
            tot += a.elapsed_time(b)
        extra["cuda_graph_step"] = {"fwd_bwd_mrays_s": round(n_rays / (tot / reps * 1e-3) / 1e6 * ws, 2),
                                    "ms_per_step": round(tot / reps, 4)}
        del graph
    except RuntimeError as e:  # report, do not fail the benchmark line
        extra["cuda_graph_step"] = {"error": str(e).splitlines()[0][:200]}

    # end to end through the public API with host buffers: every step copies
    # its target image from pinned host memory to the device and reads the
    # rendered image and the loss back, inside the timed region. The copies
    # run on a second stream: the image read-back overlaps the step's
    # backward and the next step's target upload overlaps this step, so the
    # copy engines work beside the kernels (the first upload and the last
    # read-back are inside the timed events too).
    Yh = torch.as_tensor(W.target_image(n_rays, wl.seed)).pin_memory()
    rgb_h = torch.empty(n_rays, 3).pin_memory()
    loss_h = torch.empty(1).pin_memory()
    Yd = [torch.empty_like(Y) for _ in range(2)]
    copy = torch.cuda.Stream()
    y_ready = [torch.cuda.Event() for _ in range(2)]
    fwd_done, d2h_done = torch.cuda.Event(), torch.cuda.Event()

    def e2e_run(n_steps):
        copy.wait_stream(stream)
        with torch.cuda.stream(copy):
            Yd[0].copy_(Yh, non_blocking=True)
            y_ready[0].record(copy)
        for k in range(n_steps):
            if k > 0:
                stream.wait_event(d2h_done)  # the previous image is on the host before rgb is rewritten
            api.generate_rays(cams, out=(o, d, tm))
            api.render_fwd(main, o, d, params, time=tm, out=(rgb, T, steps), residual=res)
            fwd_done.record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(fwd_done)
                rgb_h.copy_(rgb, non_blocking=True)
                d2h_done.record(copy)
                if k + 1 < n_steps:
                    Yd[(k + 1) % 2].copy_(Yh, non_blocking=True)
                    y_ready[(k + 1) % 2].record(copy)
            stream.wait_event(y_ready[k % 2])
            loss, grad = api.l2_loss(rgb, Yd[k % 2])
            loss_h.copy_(loss, non_blocking=True)
            api.render_bwd(main, o, d, params, rgb, grad, time=tm, out=(gs, gsig, gt), residual=res)
        stream.wait_event(d2h_done)

    e2e_run(args.warmup)
    barrier()
    a, b = ev(), ev()
    a.record(stream)
    e2e_run(args.steps)
    b.record(stream)
    barrier()
    ms_e2e = a.elapsed_time(b) / args.steps
    e2e = {"value": round(total_rays / (ms_e2e * 1e-3) / 1e6, 3), "unit": "Mrays/s",
           "h2d_bytes_per_step": int(Yh.numel() * 4), "d2h_bytes_per_step": int(rgb_h.numel() * 4 + 4),
           "copies": "on a second stream, overlapped with the kernels"}

    # roofline of the dominant kernel: algorithmic (demand) bytes per visited
    # cell, the byte model of the scope table: cell record, neighbour records,
    # texels; the backward adds the gradient operands sent to the L2 atomics
    # (sigma 4 B, both sites of the crossed face 24 B, 4 texels x 3 channels
    # 48 B per map)
    peaks, peak_kind = measured_peaks()
    E = main.n_edges
    tb = 8 if args.tex in ("f16", "bf16") else 16
    n_maps = 2 if args.appearance else 1  # texture maps read per coloured cell
    b_fwd_step = 32 + 16 * E / N + 4 * n_maps * tb
    b_bwd_step = b_fwd_step + 4 + 24 + 48 * n_maps
    io_fwd, io_bwd = 24 + 20, 24 + 24
    dom = "bwd" if walks["bwd"] >= walks["fwd"] else "fwd"
    ms_dom = walks[dom]  # the walk kernel alone (library-recorded events)
    alg = sum_steps * (b_bwd_step if dom == "bwd" else b_fwd_step) + n_rays * (io_bwd if dom == "bwd" else io_fwd)
    achieved = alg / (ms_dom * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    l2 = l2_bandwidth(torch, dev, stream)
    # the walk instantiation: mode, texel storage, appearance model
    kname = f"k_walk<{dom.upper()},{args.tex}" + (",appearance1>" if args.appearance else ">")
    traffic = recorded_traffic(kname, args.workload)
    issue = recorded_issue(kname)
    # achieved = demand bytes / event-timed kernel; frac against the measured
    # HBM copy peak; the same demand against the L2 read bandwidth measured
    # here; DRAM bytes (ncu) / kernel time against the HBM peak. The kernel is
    # bound by instruction issue (ncu), not by either bandwidth.
    roof = {"bound": "issue", "kernel": kname, "achieved": round(achieved, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
            "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": int(alg),
            "bytes_per_step": {"fwd": round(b_fwd_step, 1), "bwd": round(b_bwd_step, 1)},
            "ms_per_launch": round(ms_dom, 4),
            "l2_read_gbs": l2["l2_read_gbs"], "demand_vs_l2_frac": round(achieved / l2["l2_read_gbs"], 4),
            "dram_gbs": None if traffic is None else round(traffic / (ms_dom * 1e-3) / 1e9, 1),
            "dram_frac": None if traffic is None else round(traffic / (ms_dom * 1e-3) / 1e9 / hbm_peak, 4),
            "issue_active_ncu": issue, "probe": l2}

    line = {
        "metric": metric_name(args),
        "value": round(value * 1.0, 3), "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "ms_per_step_median": round(walks["step_median"], 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args, wl, cams),
                   "global_batch": total_rays, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed between timed steps (256 MB write outside the timed events)",
                   "scene_bytes": int(N * 32 + E * 16 + N * R * R * tb)},
        "ms_fwd": round(ms_fwd, 4), "ms_bwd": round(ms_bwd, 4),
        "ms_walk_kernel": {"fwd": round(walks["fwd"], 4), "bwd": round(walks["bwd"], 4)},
        "fps_fwd_bwd": round(n_img / (ms_step * 1e-3), 2),
        "mean_cells_per_ray": round(sum_steps / n_rays, 3), "fp64_rechecks_per_step": fp64 / max(1, args.steps + args.warmup),
        "clocks": clk, "e2e": e2e, "gpu_launches": int(round(launches_per_step * args.steps)),
        "gpu_launches_per_step": launches_per_step, "roofline": roof, **extra,
    }
    if rank == 0 and ws == 1 and not args.no_cpu:
        # the oracle leg: the oracle timed on the host cores, and the timed
        # kernels' error against it on a strided sample of the same rays
        line["cpu_baseline"], line["accuracy"] = cpu_baseline(args, wl, cams, args.cpu_seconds, scenes, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- oracle arm

def oracle_sample_rays(cams, n):
    """A fixed strided sample of n rays of the views, generated by the oracle."""
    import oracle as O

    per = [c.n_rays for c in cams]
    total = sum(per)
    stride = max(1, total // n)
    pick = np.arange(0, total, stride)[:n]
    os_, ds = [], []
    base = 0
    for c, m in zip(cams, per):
        sel = pick[(pick >= base) & (pick < base + m)] - base
        if len(sel):
            o, d, _ = O.raygen(c)
            os_.append(o[sel].astype(np.float32))
            ds.append(d[sel].astype(np.float32))
        base += m
    return np.concatenate(os_), np.concatenate(ds)


def oracle_step(osc, o, d, Y, params):
    import oracle as O

    rgb, T, steps, flags = O.render(osc, o, d, params=params)
    g = 2 * (rgb - Y) / (3 * len(o))
    O.render_bwd(osc, o, d, g, params=params)


def cpu_baseline(args, wl, cams, seconds, scenes=None, dev=None):
    """The oracle leg of the benchmark: the FP64 oracle timed on a bounded
    strided sample of the workload's rays on all host cores; with `scenes`,
    also the accuracy of the timed kernels against the oracle
    (accuracy_vs_oracle). Returns (cpu_baseline, accuracy or None)."""
    base = _cpu_timing(args, wl, cams, seconds)
    acc = accuracy_vs_oracle(args, wl, cams, scenes, dev) if scenes else None
    return base, acc


def _cpu_timing(args, wl, cams, seconds):
    osc, params = oracle_setup(args, wl)
    n = 64
    while True:
        o, d = oracle_sample_rays(cams, n)
        Y = W.target_image(len(o), wl.seed)
        t = time.time()
        oracle_step(osc, o, d, Y, params)
        dt = time.time() - t
        if dt * 4 > seconds or n >= 1 << 20:
            break
        n *= 4
    rate = len(o) / dt / 1e6
    return {"value": round(rate, 6), "unit": "Mrays/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(o)} rays strided over the views, fwd (threaded) + bwd (threaded walk, serial "
                      f"accumulation), FP64, {dt:.1f} s"}


def accuracy_vs_oracle(args, wl, cams, scenes, dev, n=4096):
    """Error of the timed kernels against the FP64 oracle (the oracle leg of
    the benchmark, outside every timed region), per texture storage type, on
    a fixed strided sample of the benchmark's rays (generated by the oracle's
    ray generation, FP32, rendered by both sides in one 1-D launch):
      image RMSE / max abs vs the oracle on the FP32 textures (total error)
      and on the dequantised textures (kernel error), over the rays outside
      the degenerate band; band-flagged rays and how many of them follow
      another cell sequence; gradient error of a backward in which only the
      sample's unflagged rays carry dL/dC (seeded normal), worst entry of
      |g - g_ref| / max(|g_ref|, 1e-3 max|g_ref|) against the oracle on the
      stored (dequantised) textures."""
    import torch

    import oracle as O
    from paper_2608_17682_gb300 import api

    o, d = oracle_sample_rays(cams, n)
    osc32, op = oracle_setup(args, wl)
    orgb32, oT, osteps, flags = O.render(osc32, o, d, params=op)
    ok = (flags & O.BAND_FLAGS) == 0
    oc, _, on, _ = O.trace(osc32, o, d, max_cells=1024, params=op)
    g = (np.random.default_rng(17).normal(size=(len(o), 3)) * ok[:, None]).astype(np.float32)
    to = torch.as_tensor(o, device=dev)
    td = torch.as_tensor(d, device=dev)
    tg = torch.as_tensor(g, device=dev)
    P1 = api.make_params(**wl.params, appearance=args.appearance)
    out = {"sample": f"{len(o)} rays strided over the views (oracle ray generation), 1-D launch",
           "rays_outside_band": int(ok.sum()), "band_flagged": int((~ok).sum())}
    first = next(iter(scenes.values()))
    cells, _, n_cells = api.trace_cells(first, to, td, P1, max_cells=1024)
    same = (n_cells.cpu().numpy() == on) & np.all(cells.cpu().numpy() == oc, axis=1)
    out["band_seq_mismatch"] = int((~ok & ~same).sum())
    out["unflagged_seq_mismatch"] = int((ok & ~same).sum())

    def img_err(a, b):
        e = np.abs(a[ok].astype(np.float64) - b[ok])
        return {"rmse": float(f"{math.sqrt(np.mean(e ** 2)):.3g}"), "max_abs": float(f"{e.max():.3g}")}

    def grad_err(a, b):
        a = a.cpu().numpy().astype(np.float64)
        floor = 1e-3 * np.abs(b).max()
        return float(f"{(np.abs(a - b) / np.maximum(np.abs(b), floor)).max():.3g}") if floor > 0 else 0.0

    qt = {"f16": torch.float16, "bf16": torch.bfloat16}
    for t, scene in scenes.items():
        res = torch.empty(len(o), 3, device=dev)
        rgb, _, steps = api.render_fwd(scene, to, td, P1, residual=res)
        if t == "f32":
            osq, orgb_q = osc32, orgb32
        else:
            q = lambda x: torch.as_tensor(x).to(qt[t]).float().numpy()  # noqa: E731
            sc = wl.scene
            if args.appearance:
                tvi, tvd = appearance_maps(wl)
                osq = O.OracleScene(sc.sites, sc.sigma, q(tvi), sc.offsets, sc.indices, tex_vd=q(tvd))
            else:
                osq = O.OracleScene(sc.sites, sc.sigma, q(sc.tex), sc.offsets, sc.indices)
            orgb_q = O.render(osq, o, d, params=op)[0]
        rgb_h = rgb.cpu().numpy()
        entry = {"image_vs_oracle_fp32_tex": img_err(rgb_h, orgb32),
                 "image_vs_oracle_stored_tex": img_err(rgb_h, orgb_q),
                 "steps_equal_outside_band": bool(np.array_equal(steps.cpu().numpy()[ok], osteps[ok]))}
        gvd = torch.empty(wl.scene.n, wl.scene.R, wl.scene.R, 3, device=dev) if args.appearance else None
        gs_, gsig_, gt_ = api.render_bwd(scene, to, td, P1, rgb, tg, residual=res, tex_vd_out=gvd)
        ref = O.render_bwd(osq, o, d, g.astype(np.float64), params=op)
        entry["grad_rel_err_vs_oracle"] = {"sites": grad_err(gs_, ref[0]), "sigma": grad_err(gsig_, ref[1]),
                                           "tex": grad_err(gt_, ref[2])}
        if args.appearance:
            entry["grad_rel_err_vs_oracle"]["tex_vd"] = grad_err(gvd, ref[3])
        out[t] = entry
        del ref, osq, gs_, gsig_, gt_, gvd
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = W.make_workload(args.workload, n_sites=args.sites or None)
    osc, params = oracle_setup(args, wl)
    n = 256
    o, d = oracle_sample_rays(wl.cameras, n)
    Y = W.target_image(len(o), wl.seed)
    for _ in range(args.warmup):
        oracle_step(osc, o, d, Y, params)
    t = time.time()
    for _ in range(args.steps):
        oracle_step(osc, o, d, Y, params)
    dt = (time.time() - t) / args.steps
    v = len(o) / dt / 1e6
    line = {"impl": "reference", "metric": metric_name(args), "value": round(v, 6), "unit": "Mrays/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, wl, rank_cameras(wl, 0)),
                       "sample": f"the oracle times a {len(o)}-ray strided sample of these rays per step"},
            "cpu_baseline": {"value": round(v, 6), "unit": "Mrays/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{len(o)} rays strided over the views per step"},
            "e2e": {"value": round(v, 6), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
