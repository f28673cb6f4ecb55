"""Multi-process (world size 2, gloo on CPU) checks of the N>1 host logic.

* Rays shard across ranks with no exchange in the forward pass; the one
  exchange a data-parallel trainer needs is an all-reduce (sum) of the scene
  gradients. With the FP64 oracle as each rank's renderer, the all-reduced
  shard gradients equal the gradient of all rays.
* bench.py gives each rank its own views (weak scaling) and reports the
  maximum step time over ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_2608_17682_gb300 import workloads as W
        import bench

        wl = W.make_workload("tiny")
        o, d = W.workload_rays(wl)
        g = np.random.default_rng(4).normal(size=(len(o), 3))
        sc = O.OracleScene.from_workload_scene(wl.scene)
        p = O.make_params(**wl.params)
        mine = slice(rank, None, world)  # interleaved ray shards
        gs, gsig, gt = O.render_bwd(sc, o[mine], d[mine], g[mine], params=p)
        flat = torch.from_numpy(np.concatenate([gs.ravel(), gsig, gt.ravel()]))
        dist.all_reduce(flat, op=dist.ReduceOp.SUM)
        # per-rank views and the max-over-ranks step time of the benchmark
        cams = bench.rank_cameras(wl, rank)
        eye = torch.tensor(cams[0].eye, dtype=torch.float64)
        eyes = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(eyes, eye)
        t = torch.tensor([10.0 + rank])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            full = O.render_bwd(sc, o, d, g, params=p)
            ref = np.concatenate([full[0].ravel(), full[1], full[2].ravel()])
            out.put(("grad", float(np.abs(flat.numpy() - ref).max()), float(np.abs(ref).max())))
            out.put(("eyes", [e.tolist() for e in eyes]))
            out.put(("tmax", float(t.item())))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_and_gradient_allreduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(3):
        item = q.get(timeout=300)
        res[item[0]] = item[1:]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    err, scale = res["grad"]
    assert err <= 1e-12 * max(1.0, scale)
    e0, e1 = res["eyes"][0]
    assert not np.allclose(e0, e1)  # each rank renders its own views
    assert abs(np.linalg.norm(e0) - np.linalg.norm(e1)) < 1e-9  # same orbit radius
    assert res["tmax"][0] == 11.0
