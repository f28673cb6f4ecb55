"""Plain float64 numpy definitions of the training-step helpers (Eq. 5 and the
appendix's optimiser settings), for the parity tests of vt_train.cu.

TEST INFRASTRUCTURE ONLY (imported by tests/); the product never imports it.
"""
from __future__ import annotations

import numpy as np

from . import uniform


def smooth_l1(rgb, y, beta):
    """L_rgb of Eq. 5 as the mean Smooth-L1 over all channels: 0.5 r^2 / beta
    for |r| < beta, else |r| - beta / 2; returns (loss, dL/drgb)."""
    r = np.asarray(rgb, np.float64) - np.asarray(y, np.float64)
    a = np.abs(r)
    small = a < beta
    loss = np.where(small, 0.5 * r * r / beta, a - 0.5 * beta)
    grad = np.where(small, r / beta, np.sign(r))
    return loss.mean(), grad / r.size


def texture_regularizers(tex, tex_vd, lam_vd, lam_mean):
    """lam_vd L_vd + lam_mean L_mean of Eq. 5 on [N, R, R, 3] maps:
    L_vd = 1/(N R^2) sum_i |T_i^vd|^2,
    L_mean = 1/(N R^2) sum_{i,u} |T_{i,u} - mean_v T_{i,v}|^2.
    Returns (loss, dL/dtex, dL/dtex_vd)."""
    t = np.asarray(tex, np.float64)
    v = np.asarray(tex_vd, np.float64)
    n, R = t.shape[0], t.shape[1]
    scale = 1.0 / (n * R * R)
    mean = t.reshape(n, R * R, 3).mean(axis=1)
    dev = t - mean[:, None, None, :]
    loss = lam_vd * scale * np.sum(v * v) + lam_mean * scale * np.sum(dev * dev)
    # d/dT_w sum_u |T_u - m|^2 = 2 (T_w - m) - (2 / R^2) sum_u (T_u - m) = 2 (T_w - m)
    return loss, 2.0 * lam_mean * scale * dev, 2.0 * lam_vd * scale * v


def adam(p, g, m, v, lr, b1, b2, eps, step):
    """One Adam step (Kingma & Ba 2015) with bias correction; returns (p, m, v)."""
    p, g, m, v = (np.asarray(x, np.float64) for x in (p, g, m, v))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def stratified_indices(n_pool, n, seed):
    """Index k drawn uniformly in its stratum [k n_pool/n, (k+1) n_pool/n),
    jitter = SplitMix64 counter hash of (seed, k)."""
    stride = n_pool / n
    out = np.empty(n, np.int64)
    for k in range(n):
        i = int((k + uniform(seed, k)) * stride)
        out[k] = min(i, int((k + 1) * stride) - 1, n_pool - 1)
    return out
