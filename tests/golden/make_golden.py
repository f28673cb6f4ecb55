"""Writes the stored expected values under tests/golden/ from the FP64 oracle
only (no CUDA code is imported): 36 rays of the 2,000-site tiny scene, their
colours, transmittance, visited-cell counts, cell sequences and exit
parameters, plus the per-ray distortion loss (Eq. 2).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2608_17682_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny_rays.json")


def golden_rays():
    """The fixture's rays: a 6 x 6 grid of pixels (rows and columns 21, 25,
    ..., 41) around the centre of the tiny workload's 64x64 view, where the
    rays cross the unit cube."""
    wl = W.make_workload("tiny")
    o, d = W.workload_rays(wl)
    px = np.arange(21, 42, 4)
    sel = (px[:, None] * 64 + px[None, :]).ravel()
    return wl, o[sel], d[sel], sel


def compute():
    wl, o, d, sel = golden_rays()
    osc = O.OracleScene.from_workload_scene(wl.scene)
    p = O.make_params(**wl.params)
    rgb, T, steps, flags = O.render(osc, o, d, params=p, n_threads=1)
    cells, t_out, n_cells, _ = O.trace(osc, o, d, max_cells=64, params=p, n_threads=1)
    L = O.distortion(osc, o, d, params=p, n_threads=1)
    rays = []
    for r in range(len(o)):
        n = int(n_cells[r])
        rays.append({"index": int(sel[r]), "rgb": [float(x) for x in rgb[r]], "T": float(T[r]), "steps": int(steps[r]),
                     "flags": int(flags[r]), "cells": [int(c) for c in cells[r, :n]],
                     "t_exit": [float(t) if np.isfinite(t) else None for t in t_out[r, :n]], "L_dist": float(L[r])})
    return {"source": "FP64 oracle (oracle/vt_oracle.c) on the seeded tiny workload "
                      "(2,000 sites U[0,1]^3, 4x4 textures, one 64x64 pinhole camera, unit-cube clip); "
                      "written by tests/golden/make_golden.py",
            "workload": "tiny", "rays": rays}


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, separators=(",", ":"))
    print("wrote", OUT)
