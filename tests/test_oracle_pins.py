"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, not against the oracle's own formulas.

Every function of oracle/vt_oracle.c is checked here by an independent route:
inverse maps, exactly reproduced linear functions, a brute-force walk built
only from nearest-site queries and bisection, closed forms, published test
vectors and finite differences.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle as O
from paper_2608_17682_gb300 import workloads as W

RNG = np.random.default_rng(12345)


def _fd_ok(fd, an, floor):
    """Central difference `fd` against the analytic derivative `an` at 1e-4
    relative (floor `floor`). All three must be finite: an infinite analytic
    value or floor would otherwise pass its own relative bound."""
    return (math.isfinite(fd) and math.isfinite(an) and math.isfinite(floor)
            and abs(fd - an) <= 1e-4 * max(abs(an), floor))


# ---------------------------------------------------------------- octahedral map (Sec. 5.1)

def _oct_inverse(u, v):
    """Inverse of the octahedral unfold, written from the geometry: the
    diamond |u|+|v|<=1 is the upper half of the octahedron, the corners fold
    back onto the lower half."""
    z = 1.0 - abs(u) - abs(v)
    if z >= 0:
        x, y = u, v
    else:
        x = (1.0 - abs(v)) * (1.0 if u >= 0 else -1.0)
        y = (1.0 - abs(u)) * (1.0 if v >= 0 else -1.0)
    q = np.array([x, y, z])
    return q / np.linalg.norm(q)


def test_oct_special_directions():
    assert np.allclose(O.octahedral([0, 0, 1]), [0, 0])
    assert np.allclose(O.octahedral([1, 0, 0]), [1, 0])
    assert np.allclose(O.octahedral([0, 1, 0]), [0, 1])
    assert np.allclose(O.octahedral([-1, 0, 0]), [-1, 0])
    assert np.allclose(O.octahedral([0, -1, 0]), [0, -1])
    # the south pole goes to a corner; with sign(0)=+1 it is (1,1)
    assert np.allclose(O.octahedral([0, 0, -1]), [1, 1])
    # scale invariance
    assert np.allclose(O.octahedral([2, -3, 0.5]), O.octahedral([0.2, -0.3, 0.05]))


def test_oct_continuous_across_equator():
    for d in ([1, 0, 0], [0.3, -0.7, 0], [-0.2, 0.5, 0]):
        d = np.array(d, float)
        up = O.octahedral(d + [0, 0, 1e-9])
        dn = O.octahedral(d - [0, 0, 1e-9])
        assert np.allclose(up, dn, atol=1e-8)


def test_oct_hemispheres_and_inverse():
    for _ in range(2000):
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        u, v = O.octahedral(d)
        assert abs(u) <= 1 + 1e-15 and abs(v) <= 1 + 1e-15
        assert (abs(u) + abs(v) <= 1 + 1e-12) == (d[2] >= 0) or abs(d[2]) < 1e-12
        assert np.allclose(_oct_inverse(u, v), d, atol=1e-12)
    for _ in range(500):
        u, v = RNG.uniform(-1, 1, size=2)
        assert np.allclose(O.octahedral(_oct_inverse(u, v)), [u, v], atol=1e-12)


# ---------------------------------------------------------------- bilinear fetch

@pytest.mark.parametrize("R", [2, 4, 8])
def test_bilinear_reproduces_linear_function(R):
    # texture t(x,y) = a + b*x + c*y over texel centres; bilinear interpolation
    # is exact for it inside [0,R-1]^2 (clamped outside).
    a, b, c = 0.3, 0.11, -0.07
    for _ in range(300):
        u, v = RNG.uniform(-1, 1, size=2)
        idx, w = O.bilinear_taps(R, u, v)
        assert abs(w.sum() - 1) < 1e-14 and np.all(w >= -1e-15)
        val = sum(w[k] * (a + b * (idx[k] % R) + c * (idx[k] // R)) for k in range(4))
        x = min(max((u + 1) / 2 * R - 0.5, 0), R - 1)
        y = min(max((v + 1) / 2 * R - 0.5, 0), R - 1)
        assert abs(val - (a + b * x + c * y)) < 1e-12


def test_bilinear_texel_centres_and_clamp():
    R = 4
    for ty in range(R):
        for tx in range(R):
            u = (tx + 0.5) / R * 2 - 1
            v = (ty + 0.5) / R * 2 - 1
            idx, w = O.bilinear_taps(R, u, v)
            got = {int(i): float(x) for i, x in zip(idx, w) if x > 1e-12}
            assert got == pytest.approx({ty * R + tx: 1.0})
    idx, w = O.bilinear_taps(R, -1.0, -1.0)  # corner clamps to texel (0,0)
    assert {int(i) for i, x in zip(idx, w) if x > 0} == {0}
    idx, w = O.bilinear_taps(R, 1.0, 1.0)
    assert {int(i) for i, x in zip(idx, w) if x > 0} == {R * R - 1}


# ---------------------------------------------------------------- nearest site

def test_nearest_matches_kdtree():
    s = RNG.uniform(0, 1, size=(500, 3))
    tree = cKDTree(s)
    for q in RNG.uniform(-0.2, 1.2, size=(200, 3)):
        assert O.nearest(s, q) == tree.query(q)[1]


def test_nearest_ties_go_to_the_lower_id():
    """Start-cell reading: a point equidistant from two sites (exactly, in
    binary) belongs to the site with the lower index."""
    s = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [1.0, 5.0, 0.0]])
    q = [1.0, 0.3, -0.2]
    assert O.nearest(s, q) == 0
    assert O.nearest(s[[1, 0, 2]], q) == 0


def test_exact_exit_ties_keep_the_earlier_csr_entry():
    """Exit reading: when two bisector planes give the same crossing t (the
    ray leaves through a Voronoi edge), the neighbour listed first in the
    cell's adjacency row is taken."""
    s = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    tex = np.full((3, 2, 2, 3), 0.5)
    o = np.array([0.25, 0.25, 0.0])
    d = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    for row0 in ([1, 2], [2, 1]):
        idx = np.array(row0 + [0, 2, 0, 1], np.int32)
        sc = O.OracleScene(s, [1.0, 1.0, 1.0], tex, [0, 2, 4, 6], idx)
        cells, t_out, n, _ = O.trace(sc, o[None], d[None], max_cells=4, t_far=3.0, T_eps=0.0)
        assert cells[0, 0] == 0 and cells[0, 1] == row0[0], (row0, cells[0])
        assert abs(t_out[0, 0] - 0.75 * math.sqrt(2.0)) < 1e-15


# ---------------------------------------------------------------- walk + compositing

@pytest.fixture(scope="module")
def tiny():
    wl = W.make_workload("tiny")
    return wl, O.OracleScene.from_workload_scene(wl.scene)


def _brute_walk(sites, sigma, colour, o, d, t0, t1, h=2e-5):
    """Independent walk: sample the nearest site along the ray and bisect each
    change of nearest site to 1e-13. Returns cells and boundaries."""
    tree = cKDTree(sites)
    ts = np.arange(t0, t1, h)
    ts = np.append(ts, t1)
    nn = tree.query(o[None] + ts[:, None] * d[None])[1]
    cells, bounds = [nn[0]], [t0]
    for k in np.nonzero(nn[1:] != nn[:-1])[0]:
        lo, hi = ts[k], ts[k + 1]
        a = nn[k]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if tree.query(o + mid * d)[1] == a:
                lo = mid
            else:
                hi = mid
        bounds.append(0.5 * (lo + hi))
        cells.append(nn[k + 1])
    bounds.append(t1)
    return np.array(cells), np.array(bounds)


def _slab(o, d, lo, hi, t_near, t_far):
    a, b = t_near, t_far
    for k in range(3):
        ta, tb = (lo[k] - o[k]) / d[k], (hi[k] - o[k]) / d[k]
        a, b = max(a, min(ta, tb)), min(b, max(ta, tb))
    return a, b


def test_walk_matches_nearest_site_bisection(tiny):
    wl, sc = tiny
    o, d = W.workload_rays(wl)
    sel = np.arange(0, len(o), 13)
    p = O.make_params(**{**wl.params, 'T_eps': 0.0})  # no early termination here
    checked = 0
    for r in sel:
        oo, dd = o[r].astype(np.float64), d[r].astype(np.float64)
        t0, t1 = _slab(oo, dd, np.zeros(3), np.ones(3), 0.0, 1e3)
        if t1 <= t0:
            continue
        seg = O.segments(sc, oo, dd, params=p)
        comp = seg["composited"] == 1
        cells, bounds = _brute_walk(sc.sites, sc.sigma, None, oo, dd, t0, t1)
        if min(np.min(np.diff(bounds)), np.min(seg["delta"][comp])) < 1e-4:
            continue  # a sliver the sampling grid cannot resolve
        assert np.array_equal(seg["cell"][comp], cells)
        assert np.allclose(seg["a"][comp], bounds[:-1], atol=1e-10)
        assert np.allclose(seg["b"][comp], bounds[1:], atol=1e-10)
        checked += 1
    assert checked > 40


def test_segment_invariants(tiny):
    wl, sc = tiny
    o, d = W.workload_rays(wl)
    p = O.make_params(**wl.params)
    n_term = 0
    for r in range(0, len(o), 11):
        oo, dd = o[r].astype(np.float64), d[r].astype(np.float64)
        t0, t1 = _slab(oo, dd, np.zeros(3), np.ones(3), 0.0, 1e3)
        seg = O.segments(sc, oo, dd, params=p)
        if t1 <= t0:
            assert len(seg["cell"]) == 0
            continue
        comp = seg["composited"] == 1
        a, b, delta = seg["a"][comp], seg["b"][comp], seg["delta"][comp]
        assert np.all(delta > 0)
        assert np.allclose(a[1:], b[:-1], rtol=0, atol=1e-12)  # contiguous
        T = seg["T_before"][comp]
        assert np.all(np.diff(T) <= 0)  # monotone transmittance
        tau = np.cumsum(sc.sigma[seg["cell"][comp]] * delta)
        assert np.allclose(T[1:], np.exp(-tau[:-1]), rtol=1e-12)
        T_final = T[-1] * (1 - seg["alpha"][comp][-1])
        if T_final >= 1e-4:  # walked to t_far': lengths sum to the clipped extent
            assert abs(delta.sum() - (t1 - t0)) <= 1e-12 * max(1.0, t1)
        else:
            n_term += 1
            assert abs(b[-1] - a[0] - delta.sum()) < 1e-12
            assert T[-1] >= 1e-4  # stopped right after the crossing cell
    assert n_term > 0


def test_midpoints_lie_in_their_cells(tiny):
    wl, sc = tiny
    tree = cKDTree(sc.sites)
    o, d = W.workload_rays(wl)
    p = O.make_params(**wl.params)
    n = 0
    for r in range(0, len(o), 5):
        seg = O.segments(sc, o[r], d[r], params=p)
        for c, a, b, k in zip(seg["cell"], seg["a"], seg["b"], seg["composited"]):
            if not k:
                continue
            x = o[r].astype(np.float64) + 0.5 * (a + b) * d[r].astype(np.float64)
            assert tree.query(x)[1] == c
            n += 1
    assert n > 1000


def _one_site_scene(s, sigma, colour, R=4):
    tex = np.broadcast_to(np.asarray(colour, float), (1, R, R, 3)).copy()
    return O.OracleScene(np.array([s], float), [sigma], tex, [0, 0], np.zeros(0, np.int32))


def test_closed_form_single_cell():
    # one site, no neighbours: the cell is all of space. Constant colour c.
    c = np.array([0.2, 0.5, 0.9])
    bg = np.array([1.0, 0.8, 0.6])
    sc = _one_site_scene([0.1, 0.2, 0.3], 1.7, c)
    for _ in range(20):
        o = RNG.uniform(-2, 2, size=3)
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        t_near, t_far = 0.2, RNG.uniform(0.5, 3)
        rgb, T, steps, fl = O.render(sc, o[None], d[None], t_near=t_near, t_far=t_far, bg=bg, T_eps=0.0)
        L = t_far - t_near
        assert np.allclose(rgb[0], (1 - np.exp(-1.7 * L)) * c + np.exp(-1.7 * L) * bg, atol=1e-14)
        assert abs(T[0] - np.exp(-1.7 * L)) < 1e-14 and steps[0] == 1


def test_closed_form_two_cells():
    # two sites: crossing at the bisector, t* = ((s2-s1).((s1+s2)/2 - o)) / ((s2-s1).d)
    s1, s2 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.2, -0.1])
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    tex = np.stack([np.broadcast_to(c1, (4, 4, 3)), np.broadcast_to(c2, (4, 4, 3))])
    sc = O.OracleScene(np.stack([s1, s2]), [0.9, 2.5], tex, [0, 1, 2], np.array([1, 0], np.int32))
    o = np.array([-1.0, 0.05, 0.02])
    d = np.array([1.0, 0.1, 0.0])
    d /= np.linalg.norm(d)
    tstar = np.dot(s2 - s1, 0.5 * (s1 + s2) - o) / np.dot(s2 - s1, d)
    # crossing point is equidistant from both sites
    x = o + tstar * d
    assert abs(np.linalg.norm(x - s1) - np.linalg.norm(x - s2)) < 1e-12
    t_far = 4.0
    rgb, T, steps, _ = O.render(sc, o[None], d[None], t_far=t_far, T_eps=0.0, bg=(0, 0, 0))
    a1 = 1 - np.exp(-0.9 * tstar)
    a2 = 1 - np.exp(-2.5 * (t_far - tstar))
    assert np.allclose(rgb[0], a1 * c1 + (1 - a1) * a2 * c2, atol=1e-14)
    assert steps[0] == 2


def test_skip_rule_two_cells_closed_form_and_adjoint():
    """Cell skipping (Sec. 5.6, read as: a cell whose weight w = T alpha is
    below the threshold adds no colour but still attenuates T). Two cells, the
    first too thin to pass the threshold: closed forms for C, for dC/dsigma of
    both cells and for the texel gradients, and the threshold-free limit."""
    s1, s2 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.2, -0.1])
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    bg = np.array([0.3, 0.6, 0.9])
    tex = np.stack([np.broadcast_to(c1, (4, 4, 3)), np.broadcast_to(c2, (4, 4, 3))])
    sig1, sig2 = 0.02, 2.5
    sc = O.OracleScene(np.stack([s1, s2]), [sig1, sig2], tex, [0, 1, 2], np.array([1, 0], np.int32))
    o = np.array([-1.0, 0.05, 0.02])
    d = np.array([1.0, 0.1, 0.0])
    d /= np.linalg.norm(d)
    t_far = 4.0
    tstar = np.dot(s2 - s1, 0.5 * (s1 + s2) - o) / np.dot(s2 - s1, d)
    d1, d2 = tstar, t_far - tstar
    e1, e2 = np.exp(-sig1 * d1), np.exp(-sig2 * d2)
    w1, w2 = 1 - e1, e1 * (1 - e2)
    T = e1 * e2
    skip = 0.1
    assert w1 < skip < w2
    kw = dict(t_far=t_far, T_eps=0.0, bg=tuple(bg))
    rgb, Tout, steps, flags = O.render(sc, o[None], d[None], skip_weight=skip, **kw)
    assert flags[0] == 0 and steps[0] == 2
    assert np.allclose(rgb[0], w2 * c2 + T * bg, atol=1e-14)
    assert abs(Tout[0] - T) < 1e-15
    g = np.array([0.7, -1.3, 0.4])
    gs, gsig, gt = O.render_bwd(sc, o[None], d[None], g[None], skip_weight=skip, **kw)
    # sigma_1 only attenuates what lies behind it; sigma_2 trades background for c2
    assert abs(gsig[0] - g @ (-d1 * (w2 * c2 + T * bg))) < 1e-13
    assert abs(gsig[1] - g @ (e1 * d2 * e2 * (c2 - bg))) < 1e-13
    assert np.all(gt[0] == 0.0)
    assert np.allclose(gt[1].reshape(-1, 3).sum(0), w2 * g, atol=1e-14)
    # a threshold below every weight changes nothing
    ref = O.render(sc, o[None], d[None], skip_weight=0.0, **kw)
    low = O.render(sc, o[None], d[None], skip_weight=0.5 * w1, **kw)
    assert np.array_equal(ref[0], low[0]) and np.array_equal(ref[1], low[1])
    assert np.allclose(ref[0][0], w1 * c1 + w2 * c2 + T * bg, atol=1e-14)
    # the adjoint agrees with central differences away from the threshold
    h = 1e-6
    for i, sg in enumerate((sig1, sig2)):
        sp, sm = [sig1, sig2], [sig1, sig2]
        sp[i], sm[i] = sg + h, sg - h
        fp = O.render(O.OracleScene(np.stack([s1, s2]), sp, tex, [0, 1, 2], np.array([1, 0], np.int32)),
                      o[None], d[None], skip_weight=skip, **kw)[0][0]
        fm = O.render(O.OracleScene(np.stack([s1, s2]), sm, tex, [0, 1, 2], np.array([1, 0], np.int32)),
                      o[None], d[None], skip_weight=skip, **kw)[0][0]
        assert abs(g @ (fp - fm) / (2 * h) - gsig[i]) < 1e-8
    # a weight within 1e-4 relative of the threshold is flagged as ambiguous
    _, _, _, fl = O.render(sc, o[None], d[None], skip_weight=w1 * (1 + 5e-5), **kw)
    assert fl[0] != 0
    # the test is on the weight T alpha, not on alpha: behind a dense first
    # cell the second has alpha above the threshold but weight below it
    sig1, sig2 = 2.0, 0.8
    sc = O.OracleScene(np.stack([s1, s2]), [sig1, sig2], tex, [0, 1, 2], np.array([1, 0], np.int32))
    e1, e2 = np.exp(-sig1 * d1), np.exp(-sig2 * d2)
    w1, a2, w2 = 1 - e1, 1 - e2, e1 * (1 - e2)
    skip = 0.2
    assert w2 < skip < a2 and w1 > skip
    rgb, Tout, _, flags = O.render(sc, o[None], d[None], skip_weight=skip, **kw)
    assert flags[0] == 0
    assert np.allclose(rgb[0], w1 * c1 + e1 * e2 * bg, atol=1e-14)


def test_two_cell_site_gradients_both_ways():
    """dL/ds of both sites through the plane crossing, against central
    differences of the forward pass, for a ray from cell 0 into cell 1 and
    for one from cell 1 into cell 0 (with different colours and densities)."""
    s = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, -0.1]])
    tex = np.stack([np.broadcast_to([1.0, 0.2, 0.1], (4, 4, 3)), np.broadcast_to([0.1, 0.3, 1.0], (4, 4, 3))])
    sig = [0.9, 2.5]
    adj = ([0, 1, 2], np.array([1, 0], np.int32))
    g = np.array([0.7, -1.3, 0.4])
    kw = dict(t_far=4.0, T_eps=0.0, bg=(0.2, 0.4, 0.6))
    for o, d in ((np.array([-1.0, 0.05, 0.02]), np.array([1.0, 0.1, 0.0])),
                 (np.array([2.0, 0.3, 0.1]), np.array([-1.0, -0.05, 0.03]))):
        d = d / np.linalg.norm(d)
        gs, _, _ = O.render_bwd(O.OracleScene(s, sig, tex, *adj), o[None], d[None], g[None], **kw)
        assert np.abs(gs).max() > 1e-3  # a non-trivial gradient to check
        h = 1e-6
        for i in range(2):
            for k in range(3):
                sp, sm = s.copy(), s.copy()
                sp[i, k] += h
                sm[i, k] -= h
                fp = O.render(O.OracleScene(sp, sig, tex, *adj), o[None], d[None], **kw)[0][0]
                fm = O.render(O.OracleScene(sm, sig, tex, *adj), o[None], d[None], **kw)[0][0]
                fd = g @ (fp - fm) / (2 * h)
                assert _fd_ok(fd, gs[i, k], 1e-3 * np.abs(gs).max()), (o, i, k, fd, gs[i, k])


def test_texel_gradients_reach_the_first_texel():
    """One cell, a ray whose bilinear taps sit in the octahedral corner
    (-1,-1): all of w g lands on texel (0,0) of cell 0. With the paper's
    model, a view direction -d in that corner sends w g c (1 - c) to texel
    (0,0) of the view-dependent map."""
    R, sig, L = 4, 1.3, 0.8
    w = 1 - math.exp(-sig * L)
    g = np.array([0.7, -0.4, 0.2])
    c = np.array([0.3, 0.6, 0.9])
    tex = np.broadcast_to(c, (1, R, R, 3)).copy()
    d = np.array([-0.01, -0.01, -1.0])
    d /= np.linalg.norm(d)
    kw = dict(t_far=L, T_eps=0.0, bg=(0.0, 0.0, 0.0))
    sc = O.OracleScene(np.zeros((1, 3)), [sig], tex, [0, 0], np.zeros(0, np.int32))
    _, gsig, gt = O.render_bwd(sc, np.zeros((1, 3)), d[None], g[None], **kw)
    expect = np.zeros((1, R, R, 3))
    expect[0, 0, 0] = w * g
    assert np.allclose(gt, expect, rtol=0, atol=1e-15)
    assert abs(gsig[0] - (g @ c) * L * math.exp(-sig * L)) < 1e-14
    tvd = np.broadcast_to([0.1, -0.2, 0.3], (1, R, R, 3)).copy()
    sc = O.OracleScene(np.zeros((1, 3)), [sig], tex, [0, 0], np.zeros(0, np.int32), tex_vd=tvd)
    _, _, _, gvd = O.render_bwd(sc, np.zeros((1, 3)), -d[None], g[None], appearance=1, **kw)
    cc = 1 / (1 + np.exp(-(c + tvd[0, 0, 0])))
    expect = np.zeros((1, R, R, 3))
    expect[0, 0, 0] = w * g * cc * (1 - cc)
    assert np.allclose(gvd, expect, rtol=0, atol=1e-15)


def test_constant_texture_any_direction():
    c = np.array([0.25, 0.5, 0.75])
    sc = _one_site_scene([0, 0, 0], 3.0, c, R=8)
    for _ in range(50):
        d = RNG.normal(size=3)
        rgb, T, _, _ = O.render(sc, np.zeros((1, 3)), d[None] / np.linalg.norm(d), t_far=1.0, T_eps=0.0,
                                bg=(0, 0, 0))
        assert np.allclose(rgb[0], (1 - np.exp(-3.0)) * c, atol=1e-14)


def test_colour_is_bilinear_fetch_at_ray_direction():
    R = 8
    tex = RNG.uniform(0, 1, size=(1, R, R, 3))
    sc = O.OracleScene(np.zeros((1, 3)), [50.0], tex, [0, 0], np.zeros(0, np.int32))
    for _ in range(50):
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        rgb, _, _, _ = O.render(sc, np.zeros((1, 3)), d[None], t_far=1.0, T_eps=0.0, bg=(0, 0, 0))
        # direct bilinear interpolation, written independently of the tap routine
        u, v = _oct_from_geometry(d)
        x = min(max((u + 1) / 2 * R - 0.5, 0), R - 1)
        y = min(max((v + 1) / 2 * R - 0.5, 0), R - 1)
        x0, y0 = min(int(x), R - 2), min(int(y), R - 2)
        fx, fy = x - x0, y - y0
        t = tex[0]
        c = ((1 - fy) * ((1 - fx) * t[y0, x0] + fx * t[y0, x0 + 1]) + fy * ((1 - fx) * t[y0 + 1, x0] + fx * t[y0 + 1, x0 + 1]))
        assert np.allclose(rgb[0], (1 - np.exp(-50.0)) * c, atol=1e-12)


def _oct_from_geometry(d):
    # point where the ray from the origin meets the octahedron |x|+|y|+|z|=1,
    # then the fold (u,v) used by the paper's map
    q = d / np.abs(d).sum()
    if q[2] >= 0:
        return q[0], q[1]
    return ((1 - abs(q[1])) * (1 if q[0] >= 0 else -1), (1 - abs(q[0])) * (1 if q[1] >= 0 else -1))


def test_riemann_integral_matches(tiny):
    """Volume rendering integral by fine Riemann sums over nearest-site
    lookups (no adjacency, no planes) agrees with the walk's composite."""
    wl, sc = tiny
    tree = cKDTree(sc.sites)
    o, d = W.workload_rays(wl)
    # per-cell constant colour so that colour depends on the cell only
    cols = RNG.uniform(0, 1, size=(sc.n, 3))
    tex = np.broadcast_to(cols[:, None, None, :], (sc.n, 4, 4, 3)).copy()
    sc2 = O.OracleScene(sc.sites, sc.sigma, tex, sc.off, sc.idx)
    bg = np.array([1.0, 1.0, 1.0])
    done = 0
    for r in range(3, len(o), 97):
        oo, dd = o[r].astype(np.float64), d[r].astype(np.float64)
        t0, t1 = _slab(oo, dd, np.zeros(3), np.ones(3), 0.0, 1e3)
        if t1 <= t0:
            continue
        rgb, T, _, _ = O.render(sc2, oo[None], dd[None], **{**wl.params, 'T_eps': 0.0})
        h = (t1 - t0) / 200000
        tm = t0 + (np.arange(200000) + 0.5) * h
        cell = tree.query(oo[None] + tm[:, None] * dd[None])[1]
        sg = sc.sigma[cell]
        tau = np.concatenate([[0.0], np.cumsum(sg * h)])
        Tm = np.exp(-tau[:-1])
        # exact integral of sigma*T over each sub-interval with constant sigma
        contrib = Tm * (1 - np.exp(-sg * h))
        C = (contrib[:, None] * cols[cell]).sum(0) + np.exp(-tau[-1]) * bg
        assert np.allclose(rgb[0], C, atol=2e-3), (r, rgb[0], C)
        done += 1
    assert done >= 8


def test_early_termination_bound(tiny):
    wl, sc = tiny
    o, d = W.workload_rays(wl)
    full, Tf, kf, _ = O.render(sc, o, d, **{**wl.params, 'T_eps': 0.0})
    term, Tt, kt, _ = O.render(sc, o, d, **{**wl.params, 'T_eps': 1e-4})
    assert np.all(kt <= kf)
    # stopping once T<1e-4 changes the colour by at most T (colours and bg in [0,1])
    assert np.max(np.abs(full - term)) <= 1e-4 + 1e-12
    assert np.all(Tt[kt < kf] < 1e-4)


def test_band_flags_edge_ray():
    # three sites in the plane z=0; a ray along the line where all three
    # bisectors meet crosses a Voronoi edge -> flagged near-edge
    s = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, 0.8, 0.0], [0.5, 0.3, 1.0], [0.5, 0.3, -1.0]])
    from scipy.spatial import Delaunay
    ip, ind = Delaunay(s).vertex_neighbor_vertices
    tex = np.full((5, 2, 2, 3), 0.5)
    sc = O.OracleScene(s, [1.0] * 5, tex, ip, ind)
    # circumcentre of the first three sites in z=0
    A = np.array([[2 * (s[1] - s[0])[:2]], [2 * (s[2] - s[0])[:2]]]).reshape(2, 2)
    bvec = np.array([s[1, :2] @ s[1, :2] - s[0, :2] @ s[0, :2], s[2, :2] @ s[2, :2] - s[0, :2] @ s[0, :2]])
    cc = np.linalg.solve(A, bvec)
    o = np.array([cc[0] - 0.3, cc[1], 0.1])
    d = np.array([1.0, 0.0, 0.0])
    _, _, _, fl = O.render(sc, o[None], d[None], t_far=5.0, T_eps=0.0)
    assert fl[0] & O.F_NEAR_EDGE
    o2 = o.copy()
    o2[1] = cc[1] + 0.25  # away from the edge
    _, _, _, fl2 = O.render(sc, o2[None], d[None], t_far=5.0, T_eps=0.0)
    assert fl2[0] & O.F_NEAR_EDGE == 0
    # the same configuration turned, moved and relabelled: the flags depend
    # neither on the axes nor on the site ids
    Q, _ = np.linalg.qr(np.random.default_rng(21).normal(size=(3, 3)))
    shift = np.array([0.3, -0.7, 1.1])
    sq = (s @ Q.T + shift)[[4, 2, 3, 0, 1]]
    ipq, indq = Delaunay(sq).vertex_neighbor_vertices
    scq = O.OracleScene(sq, [1.0] * 5, tex, ipq, indq)
    _, _, _, fq = O.render(scq, (Q @ o + shift)[None], (Q @ d)[None], t_far=5.0, T_eps=0.0)
    _, _, _, fq2 = O.render(scq, (Q @ o2 + shift)[None], (Q @ d)[None], t_far=5.0, T_eps=0.0)
    assert fq[0] & O.F_NEAR_EDGE and fq2[0] & O.F_NEAR_EDGE == 0


def test_band_flag_for_a_crossing_next_to_the_clip_ends():
    """A plane crossing within band_eps of t_near or t_far is flagged; one 5e-6
    away is not (two sites in general position, crossing at t*)."""
    s = np.array([[0.1, 0.2, 0.3], [0.9, 0.5, -0.2]])
    tex = np.full((2, 2, 2, 3), 0.5)
    sc = O.OracleScene(s, [1.0, 1.0], tex, [0, 1, 2], np.array([1, 0], np.int32))
    o = np.array([-0.4, 0.1, 0.5])
    n = s[1] - s[0]
    # a unit direction, and a long one (|d| = 3) nearly along n, for which a
    # t-gap of 0.5e-6 puts the ray end 1.5e-6 from the plane: the band is
    # measured in t
    unit = np.array([0.9, 0.3, -0.2]) / np.linalg.norm([0.9, 0.3, -0.2])
    along = n / np.linalg.norm(n) + [0.0, 0.05, 0.02]
    for d in (unit, 3.0 * along / np.linalg.norm(along)):
        tstar = n @ (0.5 * (s[0] + s[1]) - o) / (n @ d)
        assert O.nearest(s, o) == 0 and tstar > 0.1
        for gap, flagged in ((0.5e-6, True), (5e-6, False)):
            for kw in (dict(t_far=tstar + gap), dict(t_far=tstar - gap), dict(t_near=tstar - gap, t_far=5.0),
                       dict(t_near=tstar + gap, t_far=5.0)):
                _, _, _, fl = O.render(sc, o[None], d[None], T_eps=0.0, **kw)
                assert bool(fl[0] & O.F_NEAR_CLIP) == flagged, (gap, kw)


def test_band_flag_for_an_origin_next_to_a_face():
    """An origin within band_eps (1e-6) of a bisector plane of its cell is
    flagged; one 5e-6 away is not. Two sites in general position."""
    s = np.array([[0.1, 0.2, 0.3], [0.9, 0.5, -0.2]])
    tex = np.full((2, 2, 2, 3), 0.5)
    sc = O.OracleScene(s, [1.0, 1.0], tex, [0, 1, 2], np.array([1, 0], np.int32))
    n = (s[1] - s[0]) / np.linalg.norm(s[1] - s[0])
    tang = np.cross(n, [0.3, -0.4, 0.8])
    foot = 0.5 * (s[0] + s[1]) + 0.2 * tang / np.linalg.norm(tang)
    d = np.array([[0.2, 0.9, 0.3]])
    for side in (-1.0, 1.0):  # origins in the cell of site 0, then of site 1
        for dist, flagged in ((0.5e-6, True), (5e-6, False)):
            _, _, _, fl = O.render(sc, (foot + side * dist * n)[None], d, t_far=1.0, T_eps=0.0)
            assert bool(fl[0] & O.F_NEAR_ORIGIN) == flagged, (side, dist)


def test_band_flag_for_an_ambiguous_termination():
    """Early termination (Sec. 3.2) stops after the cell that brings T below
    T_eps. Where T after a cell lies within 1e-4 relative of T_eps, FP32 and
    FP64 may stop at different cells, so the ray is flagged F_T_AMBIG; 5e-3
    away it is not. Two cells with closed-form transmittances: T = 1 before
    the first cell, e1 = exp(-sigma_1 t*) after it and e1 e2 after the second.
    The flag must read T after compositing a cell: a T_eps next to the final
    e1 e2 (which no T before a cell equals) is flagged, one next to the initial
    T = 1 is not."""
    s1, s2 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.2, -0.1])
    tex = np.full((2, 4, 4, 3), 0.5)
    sig1, sig2 = 0.9, 2.5
    sc = O.OracleScene(np.stack([s1, s2]), [sig1, sig2], tex, [0, 1, 2], np.array([1, 0], np.int32))
    o = np.array([-1.0, 0.05, 0.02])
    d = np.array([1.0, 0.1, 0.0])
    d /= np.linalg.norm(d)
    t_far = 4.0
    tstar = np.dot(s2 - s1, 0.5 * (s1 + s2) - o) / np.dot(s2 - s1, d)
    e1 = math.exp(-sig1 * tstar)
    e12 = e1 * math.exp(-sig2 * (t_far - tstar))
    assert 1e-5 < e12 < 0.5 * e1 < 0.5

    def run(T_eps):
        _, T, k, fl = O.render(sc, o[None], d[None], t_far=t_far, T_eps=T_eps, bg=(1, 1, 1))
        return T[0], int(k[0]), int(fl[0])

    # next to the T after the first cell: flagged on both sides, and the stop
    # follows T < T_eps after compositing (one cell above, two below)
    for rel, steps in ((5e-5, 1), (-5e-5, 2)):
        T, k, fl = run(e1 * (1 + rel))
        assert fl & O.F_T_AMBIG and k == steps, (rel, fl, k)
    # 5e-3 away: not flagged, same stopping rule
    for rel, steps in ((5e-3, 1), (-5e-3, 2)):
        T, k, fl = run(e1 * (1 + rel))
        assert fl == 0 and k == steps, (rel, fl, k)
        assert abs(T - (e1 if steps == 1 else e12)) < 1e-15
    # next to the final T (after the second cell): flagged; 5e-3 away: not
    assert run(e12 * (1 + 5e-5))[2] & O.F_T_AMBIG
    assert run(e12 * (1 - 5e-5))[2] & O.F_T_AMBIG
    assert run(e12 * (1 + 5e-3))[2] == 0
    # next to the T before the first cell (1), which is never a T after a
    # cell here: not flagged
    T, k, fl = run(1.0 - 5e-5)
    assert fl == 0 and k == 1


def test_max_steps_flag(tiny):
    wl, sc = tiny
    o, d = W.workload_rays(wl)
    _, _, k, fl = O.render(sc, o, d, **wl.params, max_steps=3)
    assert np.all(k <= 3)
    assert np.any(fl & O.F_MAX_STEPS)


# ---------------------------------------------------------------- gradients

def _small_scene(n=300, seed=7, R=4):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0, 1, size=(n, 3))
    sig = np.exp(rng.normal(0.5, 1.0, size=n))
    tex = rng.uniform(0, 1, size=(n, R, R, 3))
    from scipy.spatial import Delaunay
    ip, ind = Delaunay(s).vertex_neighbor_vertices
    return s, sig, tex, ip.astype(np.int64), ind.astype(np.int32)


def _small_rays(n_side=10, seed=3):
    c = np.array([0.5, 0.5, 0.5])
    eye = W.orbit_eye(c, 2.0, 40.0, 25.0)
    o, d = W.frustum_rays(eye, c, n_side, n_side, np.random.default_rng(seed), fov_y=math.radians(30))
    return o.astype(np.float64), d.astype(np.float64)


def _loss(sc, o, d, Y, p):
    rgb, _, _, _ = O.render(sc, o, d, params=p, n_threads=1)
    return 0.5 * np.sum((rgb - Y) ** 2), rgb


def test_eq3_eq4_identities():
    # one cell, C = alpha c + (1-alpha) bg. dL/dalpha = g.(c - bg).
    c = np.array([0.2, 0.6, 0.3])
    bg = np.array([1.0, 1.0, 1.0])
    sigma, L = 2.3, 0.7
    sc = _one_site_scene([0, 0, 0], sigma, c)
    g = np.array([0.3, -0.5, 0.8])
    gs, gsig, gt = O.render_bwd(sc, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), g[None], t_far=L, T_eps=0.0,
                                bg=bg)
    alpha = 1 - math.exp(-sigma * L)
    dL_dalpha = g @ (c - bg)
    assert abs(gsig[0] - dL_dalpha * L * (1 - alpha)) < 1e-14  # Eq. 3
    assert abs(gsig[0] * sigma - dL_dalpha * (1 - alpha) * math.log(1 / (1 - alpha))) < 1e-13  # Eq. 4
    assert np.allclose(gt.sum(axis=(1, 2))[0], g * alpha)  # dL/dc = g * T alpha


@pytest.fixture(scope="module")
def fd_setup():
    s, sig, tex, ip, ind = _small_scene()
    o, d = _small_rays()
    Y = np.random.default_rng(9).uniform(0, 1, size=(len(o), 3))
    p = O.make_params(t_far=1e3, use_clip_box=True, T_eps=1e-4)
    sc = O.OracleScene(s, sig, tex, ip, ind)
    _, rgb = _loss(sc, o, d, Y, p)
    gs, gsig, gt = O.render_bwd(sc, o, d, rgb - Y, params=p)
    return s, sig, tex, ip, ind, o, d, Y, p, gs, gsig, gt


def test_fd_sigma_and_texels(fd_setup):
    s, sig, tex, ip, ind, o, d, Y, p, gs, gsig, gt = fd_setup
    rng = np.random.default_rng(1)
    cand = np.nonzero(np.abs(gsig) > 1e-6)[0]
    assert len(cand) > 20
    for i in rng.choice(cand, size=20, replace=False):
        h = 1e-6 * max(1.0, sig[i])
        vals = []
        for sgn in (1, -1):
            sg = sig.copy()
            sg[i] += sgn * h
            vals.append(_loss(O.OracleScene(s, sg, tex, ip, ind), o, d, Y, p)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gsig[i]) <= 1e-6 * max(1.0, abs(gsig[i])), (i, fd, gsig[i])
    cand = np.argwhere(np.abs(gt) > 1e-6)
    for q in cand[rng.choice(len(cand), size=20, replace=False)]:
        q = tuple(q)
        vals = []
        for sgn in (1, -1):
            tx = tex.copy()
            tx[q] += sgn * 1e-3
            vals.append(_loss(O.OracleScene(s, sig, tx, ip, ind), o, d, Y, p)[0])
        fd = (vals[0] - vals[1]) / 2e-3
        assert abs(fd - gt[q]) <= 1e-9 * max(1.0, abs(gt[q])) + 1e-12


def test_fd_site_positions(fd_setup):
    s, sig, tex, ip, ind, o, d, Y, p, gs, gsig, gt = fd_setup
    sc = O.OracleScene(s, sig, tex, ip, ind)
    base_cells = O.trace(sc, o, d, params=p, n_threads=1)[0]
    rng = np.random.default_rng(2)
    cand = np.argwhere(np.abs(gs) > 1e-5)
    checked = 0
    for q in cand[rng.permutation(len(cand))]:
        i, c = int(q[0]), int(q[1])
        h = 1e-7
        vals = []
        same = True
        for sgn in (1, -1):
            ss = s.copy()
            ss[i, c] += sgn * h
            scp = O.OracleScene(ss, sig, tex, ip, ind)
            if not np.array_equal(O.trace(scp, o, d, params=p, n_threads=1)[0], base_cells):
                same = False
                break
            vals.append(_loss(scp, o, d, Y, p)[0])
        if not same:
            continue  # perturbation changes a cell sequence: no derivative there
        fd = (vals[0] - vals[1]) / (2 * h)
        assert _fd_ok(fd, gs[i, c], 1e-3 * np.abs(gs).max()), (i, c, fd, gs[i, c])
        checked += 1
        if checked >= 25:
            break
    assert checked >= 25


# ---------------------------------------------------------------- ray generation

def test_splitmix64_published_values():
    # first two outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014;
    # reference implementation by Vigna): state advances by the golden gamma.
    assert O.mix64(0) == 0xE220A8397B1DCDAF
    assert O.mix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    u = [O.uniform(7, c) for c in range(4000)]
    assert min(u) >= 0 and max(u) < 1 and abs(np.mean(u) - 0.5) < 0.02
    assert all(x * 16777216 == int(x * 16777216) for x in u[:50])  # 24-bit values


def test_concentric_map():
    for (a, b), ex in [((1, 0), (1, 0)), ((0, 1), (0, 1)), ((-1, 0), (-1, 0)), ((0, -1), (0, -1)), ((0, 0), (0, 0))]:
        assert np.allclose(O.concentric(a, b), ex, atol=1e-15)
    for a, b in RNG.uniform(-1, 1, size=(300, 2)):
        r = np.linalg.norm(O.concentric(a, b))
        assert abs(r - max(abs(a), abs(b))) < 1e-14  # squares map to circles
    # equal-area: uniform square samples -> uniform disk (mean r^2 = 1/2) ...
    pts = np.array([O.concentric(a, b) for a, b in RNG.uniform(-1, 1, size=(20000, 2))])
    assert abs(np.mean(np.sum(pts ** 2, 1)) - 0.5) < 0.01
    # ... with a uniform angle: each eighth of the disk gets an eighth of the samples
    sector = np.floor((np.arctan2(pts[:, 1], pts[:, 0]) + np.pi) / (np.pi / 4)).astype(int) % 8
    assert np.all(np.abs(np.bincount(sector, minlength=8) / len(pts) - 0.125) < 0.012)
    # continuous across the square's diagonals, where the two wedges meet
    for sa, sb in [(1, 1), (1, -1), (-1, 1), (-1, -1)]:
        for r in (0.3, 1.0):
            p = np.array(O.concentric(sa * r, sb * r * (1 - 1e-9)))
            q = np.array(O.concentric(sa * r * (1 - 1e-9), sb * r))
            assert np.allclose(p, q, atol=1e-8)


def test_pinhole_rays():
    cam = W.look_at_camera(0, 64, 48, (3.0, 1.0, 0.5), (0.0, 0.0, 0.0), fov_y=math.radians(50))
    o, d, t = O.raygen(cam)
    f = -np.array(cam.eye) / np.linalg.norm(cam.eye)
    assert np.allclose(np.linalg.norm(d, axis=1), 1) and np.allclose(o, cam.eye) and np.all(t == 0)
    img = d.reshape(48, 64, 3)
    # left/right and top/bottom pixel pairs are symmetric about the axis
    assert np.allclose(img[:, ::-1] @ f, img @ f) and np.allclose(img[::-1] @ f, img @ f)
    # vertical angle between the top and bottom pixel centres of the middle columns
    top = 0.5 * (img[0, 31] + img[0, 32])
    bot = 0.5 * (img[47, 31] + img[47, 32])
    ang = math.acos(np.dot(top, bot) / np.linalg.norm(top) / np.linalg.norm(bot))
    assert abs(ang - 2 * math.atan((1 - 1 / 48) * math.tan(math.radians(25)))) < 1e-3
    # image "up" is world +z-ish: top rows look higher than bottom rows
    assert img[0, 32, 2] > img[47, 32, 2]


def test_pinhole_basis_with_a_tilted_up_vector():
    """Camera frame f = fwd/|fwd|, right = f x up (normalised), up' = right x f,
    for an up vector off every axis: the centre pixel looks along f, the
    centre row stays in the (f, right) plane and the centre column in the
    (f, up') plane, right/top edges lean towards +right/+up', and the
    horizontal field of view follows from the vertical one and the aspect."""
    w, h, fov = 31, 21, math.radians(50)
    cam = W.look_at_camera(0, w, h, (2.0, -1.5, 0.7), (0.1, 0.2, -0.3), up=(0.3, 0.2, 1.0), fov_y=fov)
    _, d, _ = O.raygen(cam)
    img = d.reshape(h, w, 3)
    f = np.asarray(cam.fwd) / np.linalg.norm(cam.fwd)
    right = np.cross(f, cam.up)
    right /= np.linalg.norm(right)
    upc = np.cross(right, f)
    assert np.allclose(img[h // 2, w // 2], f, atol=1e-15)
    assert np.abs(img[h // 2] @ upc).max() < 1e-15 and np.abs(img[:, w // 2] @ right).max() < 1e-15
    assert img[h // 2, -1] @ right > 0 and img[0, w // 2] @ upc > 0
    ang = math.acos(np.clip(img[h // 2, 0] @ img[h // 2, -1], -1, 1))
    assert abs(ang - 2 * math.atan((1 - 1 / w) * math.tan(fov / 2) * w / h)) < 1e-12


def test_fisheye_equidistant():
    cam = W.look_at_camera(1, 40, 30, (0.0, -2.0, 0.0), (0.0, 0.0, 0.0), fisheye_fov=math.pi)
    o, d, _ = O.raygen(cam)
    f = np.array([0.0, 1.0, 0.0])
    img = d.reshape(30, 40, 3)
    for y in range(30):
        for x in range(40):
            rpx = math.hypot(x + 0.5 - 20, 15 - (y + 0.5))
            theta = math.acos(np.clip(img[y, x] @ f, -1, 1))
            assert abs(theta - rpx / (20 / (math.pi / 2))) < 1e-12
    # azimuth: a ray bends towards its pixel's offset from the image centre,
    # measured in the camera's right / up axes (right = f x up, up' = right x f)
    up = np.asarray(cam.up, float)
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    upc = np.cross(right, f)
    for y in range(30):
        for x in range(40):
            px, py = x + 0.5 - 20, 15 - (y + 0.5)
            az = math.atan2(img[y, x] @ upc, img[y, x] @ right)
            diff = (az - math.atan2(py, px) + math.pi) % (2 * math.pi) - math.pi
            assert abs(diff) < 1e-9, (x, y)


def test_rolling_shutter():
    v = (0.05, 0.0, 0.0)
    cam = W.look_at_camera(2, 16, 8, (0.0, -2.0, 0.0), (0.0, 0.0, 0.0), rs_velocity=v)
    o, d, t = O.raygen(cam)
    pin = O.raygen(W.look_at_camera(0, 16, 8, (0.0, -2.0, 0.0), (0.0, 0.0, 0.0)))
    assert np.allclose(d, pin[1])
    rows = np.repeat(np.arange(8), 16)
    assert np.allclose(t, rows / 8)
    assert np.allclose(o, np.array([0.0, -2.0, 0.0]) + (rows / 8)[:, None] * np.array(v))


def test_thin_lens_focus():
    cam = W.look_at_camera(3, 12, 10, (0.0, -3.0, 0.0), (0.0, 0.0, 0.0), lens_radius=0.05, focus_dist=2.0,
                           lens_samples=4, seed=11)
    o, d, t = O.raygen(cam)
    assert o.shape == (480, 3)
    eye = np.array(cam.eye)
    f = np.array([0.0, 1.0, 0.0])
    # origins lie on the lens disk (plane through the eye, normal f)
    assert np.allclose((o - eye) @ f, 0, atol=1e-15)
    assert np.all(np.linalg.norm(o - eye, axis=1) <= 0.05 + 1e-15)
    # all samples of one pixel meet on the plane of focus at a common point
    tt = (2.0 - (o - eye) @ f) / (d @ f)
    P = (o + tt[:, None] * d).reshape(120, 4, 3)
    assert np.allclose(P, P[:, :1], atol=1e-12)
    # ...which is where the pinhole ray of that pixel meets the plane
    pin_o, pin_d, _ = O.raygen(W.look_at_camera(0, 12, 10, (0.0, -3.0, 0.0), (0.0, 0.0, 0.0)))
    Pp = pin_o + (2.0 / (pin_d @ f))[:, None] * pin_d
    assert np.allclose(P[:, 0], Pp, atol=1e-12)
    # stratified 2x2: sample s = sy*2+sx lands in lens quadrant (sign x, sign y)
    r = np.array([1.0, 0.0, 0.0])
    u = np.cross(r, f)
    lx = ((o - eye) @ r).reshape(120, 4)
    ly = ((o - eye) @ u).reshape(120, 4)
    for s_ in range(4):
        sx, sy = s_ % 2, s_ // 2
        assert np.all(np.sign(lx[:, s_]) == (1 if sx else -1))
        assert np.all(np.sign(ly[:, s_]) == (1 if sy else -1))


def test_motion_blur_times_and_origins():
    """Camera motion blur (Sec. 6.5): S time samples per pixel over the
    exposure [0, 1), one per stratum, with the camera centre moved linearly
    (eye + t * velocity) and the pinhole direction of that pixel."""
    v = np.array([0.04, -0.01, 0.02])
    S = 5
    cam = W.look_at_camera(4, 14, 9, (0.0, -3.0, 0.0), (0.0, 0.0, 0.0), rs_velocity=tuple(v), lens_samples=S,
                           seed=77)
    assert cam.n_rays == 14 * 9 * S
    o, d, t = O.raygen(cam)
    assert o.shape == (14 * 9 * S, 3)
    _, pin_d, _ = O.raygen(W.look_at_camera(0, 14, 9, (0.0, -3.0, 0.0), (0.0, 0.0, 0.0)))
    assert np.allclose(d, np.repeat(pin_d, S, axis=0), atol=1e-15)
    tt = t.reshape(-1, S)
    strata = np.arange(S)[None, :]
    assert np.all(tt >= strata / S) and np.all(tt < (strata + 1) / S)  # one sample per stratum
    assert np.allclose(o, np.array(cam.eye) + t[:, None] * v, atol=1e-15)
    # jitter: the SplitMix64 counter hash of (seed, pixel * S + s), even counters
    pix = np.repeat(np.arange(14 * 9), S)
    s_ = np.tile(np.arange(S), 14 * 9)
    j = np.array([O.uniform(77, int((p_ * S + k) << 1)) for p_, k in zip(pix, s_)])
    assert np.allclose(t, (s_ + j) / S, atol=1e-15)
    # the offsets within the strata are uniform: mean 1/2, variance 1/12
    u = tt * S - strata
    assert abs(u.mean() - 0.5) < 0.05 and abs(u.var() - 1 / 12) < 0.02
    # a resting camera reproduces the pinhole image sample by sample
    still = O.raygen(W.look_at_camera(4, 14, 9, (0.0, -3.0, 0.0), (0.0, 0.0, 0.0), lens_samples=S, seed=77))
    assert np.allclose(still[0], np.array(cam.eye)) and np.allclose(still[1], d)


def test_motion_blur_render_is_time_average(tiny):
    """The per-pixel mean of the motion-blur samples estimates the time
    average of pinhole renders along the camera path: with many samples it
    agrees with a fine Riemann sum over shifted pinhole cameras."""
    wl, osc = tiny
    p = O.make_params(**wl.params)
    eye = np.array(W.orbit_eye(np.zeros(3), 2.2, 30.0, 15.0))
    v = np.array([0.0, 0.0, 0.3])
    S = 64
    cam = W.look_at_camera(4, 6, 5, tuple(eye), (0.0, 0.0, 0.0), rs_velocity=tuple(v), lens_samples=S, seed=5)
    o, d, _ = O.raygen(cam)
    rgb, _, _, _ = O.render(osc, o, d, params=p)
    blur = rgb.reshape(30, S, 3).mean(1)
    M = 256
    acc = np.zeros((30, 3))
    for k in range(M):
        e = eye + (k + 0.5) / M * v
        po, pd, _ = O.raygen(W.look_at_camera(0, 6, 5, tuple(e), tuple(e - eye), fov_y=cam.fov_y))
        acc += O.render(osc, po, pd, params=p)[0]
    acc /= M
    # stratified estimate of a piecewise-smooth integrand: error well below 1e-2
    assert np.abs(blur - acc).max() < 3e-2 and np.abs(blur - acc).mean() < 5e-3


# ---------------------------------------------------------------- the 1,000-site crop (surface distribution)

def crop_setup():
    sc = W.surface_crop()
    lo, hi = sc.sites.min(0).astype(np.float64), sc.sites.max(0).astype(np.float64)
    c = 0.5 * (lo + hi)
    eye = c + np.array([0.45, -0.35, 0.25])
    o, d = W.frustum_rays(eye, c, 32, 32, np.random.default_rng(5), fov_y=math.radians(50))
    Y = np.random.default_rng(6).uniform(0, 1, size=(len(o), 3))
    params = dict(t_far=1e3, use_clip_box=True, clip_lo=tuple(lo), clip_hi=tuple(hi), T_eps=1e-4)
    return sc, o.astype(np.float64), d.astype(np.float64), Y, params


def fd_crop(sc, o, d, Y, params, n_each=20, seed=3):
    """Central finite differences of L = 0.5 sum (C - Y)^2 with the FP64
    oracle for sampled sigma, texel and site parameters (site parameters
    whose +-h perturbation changes any cell sequence are skipped).
    Returns list of (kind, index, fd, analytic)."""
    p = O.make_params(**params)
    osc = O.OracleScene.from_workload_scene(sc)
    s64, sig64, tex64 = osc.sites, osc.sigma, osc.tex
    rgb = O.render(osc, o, d, params=p, n_threads=1)[0]
    gs, gsig, gt = O.render_bwd(osc, o, d, rgb - Y, params=p)
    base_cells = O.trace(osc, o, d, params=p, n_threads=1)[0]
    rng = np.random.default_rng(seed)
    out = []

    def L(sites=s64, sigma=sig64, tex=tex64):
        sc2 = O.OracleScene(sites, sigma, tex, sc.offsets, sc.indices)
        return 0.5 * np.sum((O.render(sc2, o, d, params=p, n_threads=1)[0] - Y) ** 2), sc2

    for i in rng.choice(np.nonzero(np.abs(gsig) > 1e-9)[0], size=n_each, replace=False):
        h = 1e-6 * max(1.0, sig64[i])
        v = []
        for sgn in (1, -1):
            sg = sig64.copy()
            sg[i] += sgn * h
            v.append(L(sigma=sg)[0])
        out.append(("sigma", (int(i),), (v[0] - v[1]) / (2 * h), gsig[i]))
    cand = np.argwhere(np.abs(gt) > 1e-9)
    for q in cand[rng.choice(len(cand), size=n_each, replace=False)]:
        v = []
        for sgn in (1, -1):
            tx = tex64.copy()
            tx[tuple(q)] += sgn * 1e-3
            v.append(L(tex=tx)[0])
        out.append(("tex", tuple(int(x) for x in q), (v[0] - v[1]) / 2e-3, gt[tuple(q)]))
    cand = np.argwhere(np.abs(gs) > 1e-7)
    n = 0
    for q in cand[rng.permutation(len(cand))]:
        v = []
        for sgn in (1, -1):
            ss = s64.copy()
            ss[q[0], q[1]] += sgn * 1e-7
            val, sc2 = L(sites=ss)
            if not np.array_equal(O.trace(sc2, o, d, params=p, n_threads=1)[0], base_cells):
                v = None
                break
            v.append(val)
        if v is None:
            continue
        out.append(("sites", (int(q[0]), int(q[1])), (v[0] - v[1]) / 2e-7, gs[tuple(q)]))
        n += 1
        if n >= n_each:
            break
    return out, (gs, gsig, gt)


def test_fd_on_surface_crop():
    sc, o, d, Y, params = crop_setup()
    res, (gs, gsig, gt) = fd_crop(sc, o, d, Y, params)
    floors = {"sigma": 1e-3 * np.abs(gsig).max(), "tex": 1e-3 * np.abs(gt).max(), "sites": 1e-3 * np.abs(gs).max()}
    kinds = [r[0] for r in res]
    assert kinds.count("sites") >= 15 and kinds.count("sigma") == 20 and kinds.count("tex") == 20
    for kind, idx, fd, an in res:
        assert _fd_ok(fd, an, floors[kind]), (kind, idx, fd, an)


# ---------------------------------------------------------------- appearance model of Sec. 5.1-5.2

def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def test_paper_appearance_closed_form_single_cell():
    a = np.array([0.3, -1.2, 2.0])
    b = np.array([-0.5, 0.4, 0.1])
    tex = np.broadcast_to(a, (1, 4, 4, 3)).copy()
    tvd = np.broadcast_to(b, (1, 4, 4, 3)).copy()
    sc = O.OracleScene([[0.1, 0.2, 0.3]], [1.3], tex, [0, 0], np.zeros(0, np.int32), tex_vd=tvd)
    bg = np.array([1.0, 0.9, 0.8])
    for _ in range(10):
        o = RNG.uniform(-1, 1, size=3)
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        rgb, T, _, _ = O.render(sc, o[None], d[None], t_far=2.0, T_eps=0.0, bg=bg, appearance=1)
        L = 2.0
        assert np.allclose(rgb[0], (1 - np.exp(-1.3 * L)) * _sigmoid(a + b) + np.exp(-1.3 * L) * bg, atol=1e-14)


def test_paper_appearance_surface_directions():
    """Two cells: the origin cell is coloured at its exit point, the next cell at
    its entry point -- the same bisector crossing x*. Textures linear in texel
    coordinates make the colour a closed form of oct((x* - s)/|x* - s|)."""
    R = 8
    s1, s2 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.3, -0.2])
    A = [np.array([0.1, -0.2, 0.3]), np.array([-0.4, 0.2, 0.0])]
    Bx = [np.array([0.05, -0.1, 0.2]), np.array([0.3, 0.05, -0.07])]
    By = [np.array([-0.2, 0.15, 0.02]), np.array([0.01, -0.3, 0.11])]
    ys, xs = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    tex = np.stack([A[k] + Bx[k] * xs[..., None] + By[k] * ys[..., None] for k in range(2)])
    tvd = np.zeros_like(tex)
    sc = O.OracleScene(np.stack([s1, s2]), [0.7, 3.0], tex, [0, 1, 2], np.array([1, 0], np.int32), tex_vd=tvd)
    o = np.array([-0.6, 0.05, 0.02])
    d = np.array([1.0, 0.12, -0.05])
    d /= np.linalg.norm(d)
    tstar = np.dot(s2 - s1, 0.5 * (s1 + s2) - o) / np.dot(s2 - s1, d)
    x = o + tstar * d
    cols = []
    for k, s in enumerate((s1, s2)):
        u, v = _oct_from_geometry((x - s) / np.linalg.norm(x - s))
        xt = min(max((u + 1) / 2 * R - 0.5, 0), R - 1)
        yt = min(max((v + 1) / 2 * R - 0.5, 0), R - 1)
        cols.append(_sigmoid(A[k] + Bx[k] * xt + By[k] * yt))
    t_far = 3.0
    rgb, _, _, _ = O.render(sc, o[None], d[None], t_far=t_far, T_eps=0.0, bg=(0, 0, 0), appearance=1)
    a1 = 1 - np.exp(-0.7 * tstar)
    a2 = 1 - np.exp(-3.0 * (t_far - tstar))
    assert np.allclose(rgb[0], a1 * cols[0] + (1 - a1) * a2 * cols[1], atol=1e-13)


def test_fd_paper_appearance_on_surface_crop():
    sc, o, d, Y, params = crop_setup()
    rng = np.random.default_rng(21)
    tex_vi = rng.normal(0.0, 1.5, size=sc.tex.shape)
    tex_vd = rng.normal(0.0, 0.5, size=sc.tex.shape)
    params = dict(params, appearance=1)
    p = O.make_params(**params)
    osc = O.OracleScene(sc.sites, sc.sigma, tex_vi, sc.offsets, sc.indices, tex_vd=tex_vd)
    s64, sig64 = osc.sites, osc.sigma
    rgb = O.render(osc, o, d, params=p, n_threads=1)[0]
    gs, gsig, gt, gtv = O.render_bwd(osc, o, d, rgb - Y, params=p)
    base_cells = O.trace(osc, o, d, params=p, n_threads=1)[0]

    def L(sites=s64, sigma=sig64, tvi=tex_vi, tvd=tex_vd):
        sc2 = O.OracleScene(sites, sigma, tvi, sc.offsets, sc.indices, tex_vd=tvd)
        return 0.5 * np.sum((O.render(sc2, o, d, params=p, n_threads=1)[0] - Y) ** 2), sc2

    def check(fd, an, scale):
        assert _fd_ok(fd, an, 1e-3 * scale), (fd, an)

    for arr, g, name in ((tex_vi, gt, "vi"), (tex_vd, gtv, "vd")):
        cand = np.argwhere(np.abs(g) > 1e-9)
        for q in cand[rng.choice(len(cand), size=10, replace=False)]:
            v = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2[tuple(q)] += sgn * 1e-5
                v.append(L(**({"tvi": a2} if name == "vi" else {"tvd": a2}))[0])
            check((v[0] - v[1]) / 2e-5, g[tuple(q)], np.abs(g).max())
    for i in rng.choice(np.nonzero(np.abs(gsig) > 1e-9)[0], size=10, replace=False):
        h = 1e-6 * max(1.0, sig64[i])
        v = []
        for sgn in (1, -1):
            sg = sig64.copy()
            sg[i] += sgn * h
            v.append(L(sigma=sg)[0])
        check((v[0] - v[1]) / (2 * h), gsig[i], np.abs(gsig).max())
    cand = np.argwhere(np.abs(gs) > 1e-7)
    n = 0
    for q in cand[rng.permutation(len(cand))]:
        v = []
        for sgn in (1, -1):
            ss = s64.copy()
            ss[q[0], q[1]] += sgn * 1e-7
            val, sc2 = L(sites=ss)
            if not np.array_equal(O.trace(sc2, o, d, params=p, n_threads=1)[0], base_cells):
                v = None
                break
            v.append(val)
        if v is None:
            continue
        check((v[0] - v[1]) / 2e-7, gs[tuple(q)], np.abs(gs).max())
        n += 1
        if n >= 20:
            break
    assert n >= 15


def test_fd_paper_appearance_rays_starting_inside():
    """Origins inside the crop: the cell holding the origin is composited and
    coloured at its exit point, so its site and exit crossing get gradients."""
    sc, o_out, d_out, Y, params = crop_setup()
    rng = np.random.default_rng(22)
    lo, hi = np.array(params["clip_lo"]), np.array(params["clip_hi"])
    c = 0.5 * (lo + hi)
    n = 400
    o = c + rng.uniform(-0.05, 0.05, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = rng.uniform(0, 1, size=(n, 3))
    tex_vi = rng.normal(0.0, 1.5, size=sc.tex.shape)
    tex_vd = rng.normal(0.0, 0.5, size=sc.tex.shape)
    p = O.make_params(**dict(params, appearance=1))
    osc = O.OracleScene(sc.sites, sc.sigma, tex_vi, sc.offsets, sc.indices, tex_vd=tex_vd)
    rgb = O.render(osc, o, d, params=p, n_threads=1)[0]
    gs = O.render_bwd(osc, o, d, rgb - Y, params=p)[0]
    base_cells = O.trace(osc, o, d, params=p, n_threads=1)[0]
    first = set(base_cells[:, 0].tolist())  # origin cells
    checked = 0
    for i in rng.permutation(sorted(first)):
        for k in range(3):
            if abs(gs[i, k]) < 1e-7:
                continue
            v = []
            for sgn in (1, -1):
                ss = osc.sites.copy()
                ss[i, k] += sgn * 1e-7
                sc2 = O.OracleScene(ss, osc.sigma, tex_vi, sc.offsets, sc.indices, tex_vd=tex_vd)
                if not np.array_equal(O.trace(sc2, o, d, params=p, n_threads=1)[0], base_cells):
                    v = None
                    break
                v.append(0.5 * np.sum((O.render(sc2, o, d, params=p, n_threads=1)[0] - Y) ** 2))
            if v is None:
                continue
            fd = (v[0] - v[1]) / 2e-7
            assert _fd_ok(fd, gs[i, k], 1e-3 * np.abs(gs).max()), (i, k, fd, gs[i, k])
            checked += 1
        if checked >= 12:
            break
    assert checked >= 8


# ---------------------------------------------------------------- distortion loss (Eq. 2) and sigma = exp(rho)

def _s(t):
    return 1.0 - 1.0 / (1.0 + t)


def test_distortion_single_cell_closed_form():
    # one cell over [t_near, t_far]: only the self term, w^2 (s(b) - s(a)) / 3
    sc = _one_site_scene([0.1, 0.2, 0.3], 1.3, [0.5, 0.5, 0.5])
    for _ in range(10):
        o = RNG.uniform(-2, 2, size=3)
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        a, b = 0.2, RNG.uniform(0.5, 3)
        L = O.distortion(sc, o[None], d[None], t_near=a, t_far=b, T_eps=0.0)
        w = 1 - math.exp(-1.3 * (b - a))
        assert abs(L[0] - w * w * (_s(b) - _s(a)) / 3) < 1e-15


def test_distortion_two_cells_closed_form():
    s1, s2 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.2, -0.1])
    tex = np.full((2, 4, 4, 3), 0.5)
    sc = O.OracleScene(np.stack([s1, s2]), [0.9, 2.5], tex, [0, 1, 2], np.array([1, 0], np.int32))
    o = np.array([-1.0, 0.05, 0.02])
    d = np.array([1.0, 0.1, 0.0])
    d /= np.linalg.norm(d)
    tstar = np.dot(s2 - s1, 0.5 * (s1 + s2) - o) / np.dot(s2 - s1, d)
    L = O.distortion(sc, o[None], d[None], t_far=4.0, T_eps=0.0)[0]
    w1 = 1 - math.exp(-0.9 * tstar)
    w2 = (1 - w1) * (1 - math.exp(-2.5 * (4.0 - tstar)))
    m1, m2 = 0.5 * (_s(0) + _s(tstar)), 0.5 * (_s(tstar) + _s(4.0))
    # ordered pairs (1,2) and (2,1), then the two self terms
    ex = 2 * w1 * w2 * (m2 - m1) + (w1 ** 2 * (_s(tstar) - _s(0)) + w2 ** 2 * (_s(4.0) - _s(tstar))) / 3
    assert abs(L - ex) < 1e-15


def test_distortion_is_double_integral_of_weight_histogram(tiny):
    """Mip-NeRF 360: the loss equals the double integral of |u - v| against
    the step-function weight density (w_k spread uniformly over
    [s(a_k), s(b_k)]). Midpoint quadrature with m points per interval has
    relative error 1/m^2 on the self terms."""
    wl, osc = tiny
    p = O.make_params(**wl.params)
    o, d = W.workload_rays(wl)
    rng = np.random.default_rng(8)
    L = O.distortion(osc, o, d, params=p)
    checked = 0
    m = 400
    for r in rng.permutation(len(o)):
        sg = O.segments(osc, o[r], d[r], params=p)
        sel = sg["composited"] == 1
        if sel.sum() < 3:
            continue
        a, b = sg["a"][sel], sg["b"][sel]
        w = sg["T_before"][sel] * sg["alpha"][sel]
        lo, hi = _s(a), _s(b)
        x = (np.arange(m) + 0.5) / m
        u = (lo[:, None] + x[None, :] * (hi - lo)[:, None]).ravel()
        wu = np.repeat(w / m, m)
        I = 0.0
        for c in range(0, len(u), 2000):
            I += np.sum(wu[c:c + 2000, None] * wu[None, :] * np.abs(u[c:c + 2000, None] - u[None, :]))
        assert abs(I - L[r]) <= 2e-5 * L[r] + 1e-15, (r, I, L[r])
        checked += 1
        if checked >= 8:
            break
    assert checked == 8


def _crop_dist_fd(params, n_each=15, seed=4):
    """Central differences of sum_r gd_r L_dist(r) on the 1,000-site crop
    against the oracle's adjoint (grad_rgb = 0)."""
    sc, o, d, _, _ = crop_setup()
    p = O.make_params(**params)
    osc = O.OracleScene.from_workload_scene(sc)
    gd = np.random.default_rng(11).uniform(0.5, 1.5, size=len(o))
    gs, gsig, gt = O.render_bwd(osc, o, d, np.zeros((len(o), 3)), params=p, grad_dist=gd)
    assert np.all(gt == 0)
    s64, sig64 = osc.sites, osc.sigma
    base_cells = O.trace(osc, o, d, params=p, n_threads=1)[0]

    def F(sites=s64, sigma=sig64):
        sc2 = O.OracleScene(sites, sigma, osc.tex, sc.offsets, sc.indices)
        return float(gd @ O.distortion(sc2, o, d, params=p, n_threads=1)), sc2

    rng = np.random.default_rng(seed)
    out = []
    for i in rng.choice(np.nonzero(np.abs(gsig) > 1e-9)[0], size=n_each, replace=False):
        h = 1e-6 * max(1.0, sig64[i])
        v = []
        for sgn in (1, -1):
            sg = sig64.copy()
            sg[i] += sgn * h
            v.append(F(sigma=sg)[0])
        out.append(("sigma", (v[0] - v[1]) / (2 * h), gsig[i], np.abs(gsig).max()))
    cand = np.argwhere(np.abs(gs) > 1e-9)
    n_sites = 0
    for q in cand[rng.permutation(len(cand))]:
        i, c = int(q[0]), int(q[1])
        h = 1e-7
        v = []
        for sgn in (1, -1):
            ss = s64.copy()
            ss[i, c] += sgn * h
            val, sc2 = F(sites=ss)
            if not np.array_equal(O.trace(sc2, o, d, params=p, n_threads=1)[0], base_cells):
                break
            v.append(val)
        if len(v) < 2:
            continue
        out.append(("sites", (v[0] - v[1]) / (2 * h), gs[i, c], np.abs(gs).max()))
        n_sites += 1
        if n_sites >= n_each:
            break
    return out


def test_fd_distortion_on_surface_crop():
    sc, o, d, Y, params = crop_setup()
    res = _crop_dist_fd(params)
    assert sum(r[0] == "sites" for r in res) >= 10
    for kind, fd, an, mx in res:
        assert _fd_ok(fd, an, 1e-3 * mx), (kind, fd, an)


def test_distortion_gradient_adds_to_colour_gradient(tiny):
    # the adjoint is linear in (dL/dC, dL/dL_dist)
    wl, osc = tiny
    p = O.make_params(**wl.params)
    o, d = W.workload_rays(wl)
    o, d = o[:600], d[:600]
    rng = np.random.default_rng(3)
    g = rng.normal(size=(len(o), 3))
    gd = rng.uniform(0, 1, size=len(o))
    a = O.render_bwd(osc, o, d, g, params=p)
    b = O.render_bwd(osc, o, d, np.zeros_like(g), params=p, grad_dist=gd)
    c = O.render_bwd(osc, o, d, g, params=p, grad_dist=gd)
    for x, y, z in zip(a, b, c):
        assert np.allclose(x + y, z, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(z).max()))


def test_exp_density_gradient_is_size_invariant():
    """Eq. 4: with sigma = exp(rho), dL/drho = dL/dalpha (1 - alpha) ln(1/(1 - alpha)):
    two single-cell rays of equal opacity but segment lengths 0.1 and 2.0
    give the same dL/drho; dL/dsigma differs by the length ratio (Eq. 3)."""
    c, bg = np.array([0.9, 0.1, 0.4]), np.array([0.0, 0.0, 0.0])
    g = np.array([0.5, -0.2, 0.3])
    alpha = 0.6
    out = []
    for L in (0.1, 2.0):
        rho = math.log(-math.log(1 - alpha) / L)
        sigma = O.density_from_log([rho])
        sc = _one_site_scene([0, 0, 0], sigma[0], c)
        _, gsig, _ = O.render_bwd(sc, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), g[None], t_far=L, T_eps=0.0, bg=bg)
        grho = O.density_log_bwd(sigma, gsig)[0]
        out.append((gsig[0], grho))
        assert abs(grho - (g @ (c - bg)) * (1 - alpha) * math.log(1 / (1 - alpha))) < 1e-14
    assert abs(out[0][1] - out[1][1]) < 1e-14
    assert abs(out[0][0] / out[1][0] - 0.1 / 2.0) < 1e-12


# ---------------------------------------------------------------- training-step helpers (Eq. 5, appendix)

def test_smooth_l1_matches_library():
    import torch
    from oracle import training as TR
    rng = np.random.default_rng(31)
    a, b = rng.uniform(0, 1, size=(500, 3)), rng.uniform(0, 1, size=(500, 3))
    for beta in (1e-2, 0.1, 1.0):
        L, g = TR.smooth_l1(a, b, beta)
        ta = torch.tensor(a, requires_grad=True)
        tl = torch.nn.functional.smooth_l1_loss(ta, torch.tensor(b), beta=beta)
        tl.backward()
        assert abs(L - tl.item()) < 1e-15 and np.allclose(g, ta.grad.numpy(), atol=1e-18, rtol=1e-12)


def test_adam_matches_library():
    import torch
    from oracle import training as TR
    rng = np.random.default_rng(32)
    p0 = rng.normal(size=40)
    gs = [rng.normal(size=40) for _ in range(4)]
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(40), np.zeros(40)
    for k, g in enumerate(gs, 1):
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = TR.adam(p, g, m, v, 3e-2, 0.9, 0.999, 1e-8, k)
    assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-14)


def test_texture_regularizers_closed_forms_and_fd():
    from oracle import training as TR
    rng = np.random.default_rng(33)
    n, R = 5, 4
    # constant texture per cell: no deviation from the mean
    const = np.repeat(np.repeat(rng.normal(size=(n, 1, 1, 3)), R, 1), R, 2)
    L, gt, gv = TR.texture_regularizers(const, np.zeros_like(const), 1.0, 1.0)
    assert L < 1e-28 and np.abs(gt).max() < 1e-15 and not gv.any()  # zero up to the rounding of the mean
    # view-dependent map of constant c: L_vd = 3 c^2 (per texel, averaged over cells and texels)
    L, _, _ = TR.texture_regularizers(const, np.full_like(const, 0.3), 1.0, 0.0)
    assert abs(L - 3 * 0.09) < 1e-15
    # one texel raised by h in one channel of one cell: L_mean = h^2 (1 - 1/R^2) / (N R^2)
    t = np.zeros((n, R, R, 3))
    t[2, 1, 3, 0] = 0.7
    L, _, _ = TR.texture_regularizers(t, np.zeros_like(t), 0.0, 1.0)
    assert abs(L - 0.49 * (1 - 1 / R ** 2) / (n * R * R)) < 1e-15
    # gradients by central differences
    t = rng.normal(size=(n, R, R, 3))
    v = rng.normal(size=(n, R, R, 3))
    L, gt, gv = TR.texture_regularizers(t, v, 0.3, 0.7)
    for _ in range(12):
        q = tuple(rng.integers(0, s) for s in t.shape)
        for arr, g in ((t, gt), (v, gv)):
            h = 1e-6
            arr[q] += h
            lp = TR.texture_regularizers(t, v, 0.3, 0.7)[0]
            arr[q] -= 2 * h
            lm = TR.texture_regularizers(t, v, 0.3, 0.7)[0]
            arr[q] += h
            assert abs((lp - lm) / (2 * h) - g[q]) < 1e-9


def test_stratified_ray_sampling():
    from oracle import training as TR
    idx = TR.stratified_indices(10_000, 777, seed=5)
    stride = 10_000 / 777
    k = np.arange(777)
    assert np.all(idx >= np.floor(k * stride)) and np.all(idx < np.ceil((k + 1) * stride))
    assert np.all(np.diff(idx) > 0)
    # position inside the stratum is uniform: mean ~ 1/2, variance ~ 1/12
    pos = (idx + 0.5) / stride - k
    assert abs(np.mean(pos) - 0.5) < 0.05
    assert abs(np.var(pos) - 1.0 / 12.0) < 0.02


# ---------------------------------------------------------------- stored expected values

def test_oracle_matches_stored_golden_values():
    """tests/golden/oracle_tiny_rays.json was written by make_golden.py from
    the oracle; any change of the oracle's results on these rays shows here."""
    import json
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_golden
    stored = json.load(open(make_golden.OUT))
    now = make_golden.compute()
    assert len(stored["rays"]) == len(now["rays"]) == 36
    for a, b in zip(stored["rays"], now["rays"]):
        assert a["cells"] == b["cells"] and a["steps"] == b["steps"] and a["flags"] == b["flags"]
        assert np.allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-13) and abs(a["T"] - b["T"]) <= 1e-13
        assert abs(a["L_dist"] - b["L_dist"]) <= 1e-13
        ta = np.array([np.inf if t is None else t for t in a["t_exit"]])
        tb = np.array([np.inf if t is None else t for t in b["t_exit"]])
        assert np.array_equal(np.isinf(ta), np.isinf(tb)) and np.allclose(ta[np.isfinite(ta)], tb[np.isfinite(tb)],
                                                                             rtol=1e-13, atol=0)


def test_joint_translation_of_both_sites_moves_the_crossing():
    """Plane-crossing derivatives: moving both sites of the crossed face by the
    same e moves the crossing like moving the ray origin by -e (only the
    relative geometry matters), so the sum of the two site gradients equals the
    finite difference of that joint translation (two-cell scene, one ray)."""
    s1, s2 = np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.2, -0.1])
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    tex = np.stack([np.broadcast_to(c1, (4, 4, 3)), np.broadcast_to(c2, (4, 4, 3))])
    o = np.array([-1.0, 0.05, 0.02])
    d = np.array([1.0, 0.1, 0.0])
    d /= np.linalg.norm(d)
    g = np.array([0.7, -0.3, 0.5])
    p = O.make_params(t_far=4.0, T_eps=0.0, bg=(0.2, 0.2, 0.2))

    def loss(a, b):
        sc = O.OracleScene(np.stack([a, b]), [0.9, 2.5], tex, [0, 1, 2], np.array([1, 0], np.int32))
        return float(g @ O.render(sc, o[None], d[None], params=p)[0][0]), sc

    _, sc = loss(s1, s2)
    gs, _, _ = O.render_bwd(sc, o[None], d[None], g[None], params=p)
    n = s2 - s1
    for e in np.eye(3):
        h = 1e-6
        fd = (loss(s1 + h * e, s2 + h * e)[0] - loss(s1 - h * e, s2 - h * e)[0]) / (2 * h)
        assert abs(fd - (gs[0] + gs[1]) @ e) < 1e-7
    # and the sum is parallel to n: a joint move within the face plane does not move the crossing
    tot = gs[0] + gs[1]
    assert np.linalg.norm(np.cross(tot, n)) <= 1e-12 * max(1.0, np.linalg.norm(tot))


def test_fd_distortion_rays_starting_inside_with_termination():
    """Distortion loss for origins inside the crop (first interval starts at
    t_near = 0, not at a crossing) and with early termination at T < 1e-2:
    FD of sum gd L_dist for densities and sites against the adjoint."""
    sc, _, _, _, params = crop_setup()
    rng = np.random.default_rng(31)
    lo, hi = np.array(params["clip_lo"]), np.array(params["clip_hi"])
    c = 0.5 * (lo + hi)
    n = 300
    o = c + rng.uniform(-0.05, 0.05, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = O.make_params(**dict(params, T_eps=1e-2))
    osc = O.OracleScene.from_workload_scene(sc)
    _, T, _, flags = O.render(osc, o, d, params=p, n_threads=1)
    keep = (flags & O.BAND_FLAGS) == 0  # rays near a degenerate configuration are left out
    o, d, T = o[keep], d[keep], T[keep]
    n = len(o)
    assert (T < 1e-2).sum() > 20  # some rays terminate early
    gd = rng.uniform(0.5, 1.5, size=n)
    gs, gsig, _ = O.render_bwd(osc, o, d, np.zeros((n, 3)), params=p, grad_dist=gd)
    base_cells = O.trace(osc, o, d, params=p, n_threads=1)[0]

    def F(sites=osc.sites, sigma=osc.sigma):
        sc2 = O.OracleScene(sites, sigma, osc.tex, sc.offsets, sc.indices)
        return float(gd @ O.distortion(sc2, o, d, params=p, n_threads=1)), sc2

    for i in rng.choice(np.nonzero(np.abs(gsig) > 1e-9)[0], size=12, replace=False):
        h = 1e-6 * max(1.0, osc.sigma[i])
        v = []
        for sgn in (1, -1):
            sg = osc.sigma.copy()
            sg[i] += sgn * h
            v.append(F(sigma=sg)[0])
        fd = (v[0] - v[1]) / (2 * h)
        assert _fd_ok(fd, gsig[i], 1e-3 * np.abs(gsig).max()), (i, fd, gsig[i])
    checked = 0
    for q in np.argwhere(np.abs(gs) > 1e-9)[rng.permutation(int((np.abs(gs) > 1e-9).sum()))]:
        i, k = int(q[0]), int(q[1])
        v = []
        for sgn in (1, -1):
            ss = osc.sites.copy()
            ss[i, k] += sgn * 1e-7
            val, sc2 = F(sites=ss)
            if not np.array_equal(O.trace(sc2, o, d, params=p, n_threads=1)[0], base_cells):
                break
            v.append(val)
        if len(v) < 2:
            continue
        fd = (v[0] - v[1]) / 2e-7
        assert _fd_ok(fd, gs[i, k], 1e-3 * np.abs(gs).max()), (i, k, fd, gs[i, k])
        checked += 1
        if checked >= 12:
            break
    assert checked >= 10
