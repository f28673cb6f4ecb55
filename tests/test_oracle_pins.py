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
        assert abs(fd - gs[i, c]) <= 1e-4 * max(abs(gs[i, c]), 1e-3 * np.abs(gs).max()), (i, c, fd, gs[i, c])
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
    # equal-area: uniform square samples -> uniform disk (mean r^2 = 1/2)
    pts = np.array([O.concentric(a, b) for a, b in RNG.uniform(-1, 1, size=(20000, 2))])
    assert abs(np.mean(np.sum(pts ** 2, 1)) - 0.5) < 0.01


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
        assert abs(fd - an) <= 1e-4 * max(abs(an), floors[kind]), (kind, idx, fd, an)
