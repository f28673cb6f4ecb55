"""The oracle pins catch plausible mistakes.

Each mutant below is a copy of oracle/vt_oracle.c with one mistake of the kind
a careful reader could still make (a dropped term, a wrong sign, a transposed
index, an off-by-one, a wrong constant), compiled into a temporary library.
tests/test_oracle_pins.py then runs against that library (VT_ORACLE_LIB) and
must fail. An unmutated copy built the same way must pass, so a broken harness
cannot pass for a caught mutant. The oracle source itself is never modified.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vt_oracle.c")

# (mistake, text in the oracle, text of the mutant)
MUTANTS = [
    # walk (Sec. 3.1)
    ("exit = farthest forward crossing", "if (t < best_t) {", "if (t > best_t || best_t == INFINITY) {"),
    ("bisector through s_j instead of the midpoint", "0.5 * (si[0] + sj[0]) - o[0]", "sj[0] - o[0]"),
    ("backward-facing planes kept", "if (!(den > 0.0)) continue;", "if (den == 0.0) continue;"),
    # compositing (Sec. 3.2)
    ("weight without transmittance", "w = T * alpha", "w = alpha"),
    ("alpha from sigma alone", "double e = exp(-sig * delta);", "double e = exp(-sig);"),
    ("background dropped", "for (int ch = 0; ch < 3; ++ch) C[ch] += T * p->bg[ch];", ""),
    ("termination ten times early", "if (T < p->T_eps) stop = 1;", "if (T < 10.0 * p->T_eps) stop = 1;"),
    # cell skipping (Sec. 5.6)
    ("skip test on alpha, not on the weight", "if (!(p->skip_weight > 0.0) || w >= p->skip_weight) {",
     "if (!(p->skip_weight > 0.0) || alpha >= p->skip_weight) {"),
    # octahedral map and bilinear fetch (Sec. 5.1)
    ("fold uses the wrong coordinate", "uv[0] = (1.0 - fabs(qy)) * sx;", "uv[0] = (1.0 - fabs(qx)) * sx;"),
    ("sign(0) = -1 in the fold", "double sx = (qx >= 0.0) ? 1.0 : -1.0;", "double sx = (qx > 0.0) ? 1.0 : -1.0;"),
    ("texel centres off by half a texel", "double x = (u + 1.0) * 0.5 * R - 0.5;", "double x = (u + 1.0) * 0.5 * R;"),
    ("texel index transposed", "idx[1] = y0 * R + x1;", "idx[1] = x1 * R + y0;"),
    ("bilinear weight axes swapped", "w[1] = fx * (1.0 - fy);", "w[1] = fy * (1.0 - fx);"),
    # paper appearance model (Sec. 5.1-5.2)
    ("view direction towards the scene", "double om[3] = {-d[0], -d[1], -d[2]};", "double om[3] = {d[0], d[1], d[2]};"),
    ("origin cell coloured at its entry", "if (k > 1) {\n            s.t_x = t_in;", "if (k > 0) {\n            s.t_x = t_in;"),
    # backward (Eq. 3 and the plane crossings)
    ("suffix without the background", "double S[3] = {T * p->bg[0], T * p->bg[1], T * p->bg[2]};",
     "double S[3] = {0.0, 0.0, 0.0};"),
    ("suffix without the weights", "for (int ch = 0; ch < 3; ++ch) S[ch] += s->w * s->c[ch];",
     "for (int ch = 0; ch < 3; ++ch) S[ch] += s->c[ch];"),
    ("T after the cell taken before it", "double Tn = s->T_before * (1.0 - s->alpha);", "double Tn = s->T_before;"),
    ("dL/dsigma without the segment length", "st |= emit(&cb, n3 + i, dtau[q] * s->delta);",
     "st |= emit(&cb, n3 + i, dtau[q]);"),
    ("far cell's density dropped at a crossing", "if (q + 1 < sb.n) dt_b -= sc->sigma[j] * dtau[q + 1];", ""),
    ("crossing derivative with the wrong sign", "st |= emit(&cb, 3 * i + c, dt_b * (xb[c] - si[c]) / nd);",
     "st |= emit(&cb, 3 * i + c, dt_b * (si[c] - xb[c]) / nd);"),
    ("sigmoid derivative dropped",
     "for (int ch = 0; ch < 3; ++ch) gz[ch] = g[ch] * s->w * s->c[ch] * (1.0 - s->c[ch]);",
     "for (int ch = 0; ch < 3; ++ch) gz[ch] = g[ch] * s->w * s->c[ch];"),
    ("surface-direction gradient sign flipped", "st |= emit(&cb, 3 * i + c3, -gx[c3]);",
     "st |= emit(&cb, 3 * i + c3, gx[c3]);"),
    ("entry-point term of the crossing dropped", "if (s->x_on == 0 && q > 0) xterm[q - 1] += gt;", ""),
    ("octahedral Jacobian sign", "dv = -sg[1] * sg[0] * dq0;", "dv = sg[1] * sg[0] * dq0;"),
    # distortion loss (Eq. 2)
    ("cross-interval term halved", "L += a->w * b->w * fabs(sk - sl);", "L += 0.5 * a->w * b->w * fabs(sk - sl);"),
    ("self term 1/2 instead of 1/3", "L += a->w * a->w * (s_of_t(a->b) - s_of_t(a->a)) / 3.0;",
     "L += a->w * a->w * (s_of_t(a->b) - s_of_t(a->a)) / 2.0;"),
    ("distance not normalised", "static double s_of_t(double t) { return 1.0 - 1.0 / (1.0 + t); }",
     "static double s_of_t(double t) { return t; }"),
    ("self-term derivative 1/3 instead of 2/3", "dw += 2.0 / 3.0 * a->w * dsk;", "dw += 1.0 / 3.0 * a->w * dsk;"),
    ("earlier weights' derivative with the wrong sign", "if (sb->s[j].composited) dtau[j] -= gd * dw * a->w;",
     "if (sb->s[j].composited) dtau[j] += gd * dw * a->w;"),
    # cameras (Sec. 6.5) and the counter-based generator
    ("rolling-shutter time of the next row", "tm = (double)y / (double)c->h;", "tm = (double)(y + 1) / (double)c->h;"),
    ("fisheye angle halved", "double th = rr / fpx;", "double th = 0.5 * rr / fpx;"),
    ("thin-lens rays not refocused", "for (int k = 0; k < 3; ++k) dd[k] = c->eye[k] + c->focus_dist * pd[k] - oo[k];",
     "for (int k = 0; k < 3; ++k) dd[k] = c->focus_dist * pd[k];"),
    ("concentric map angle doubled", "phi = (M_PI / 4.0) * (b / a);", "phi = (M_PI / 2.0) * (b / a);"),
    ("motion-blur times not divided into strata", "tm = (s + vto_uniform(c->seed, (pix * S + s) << 1)) / S;",
     "tm = vto_uniform(c->seed, (pix * S + s) << 1);"),
    ("SplitMix64 constant", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "z = (z ^ (z >> 27)) * 0x94D049BB133111EDull;"),
    ("pinhole pixel centres off by half a pixel", "double py = (1.0 - 2.0 * (y + 0.5) / c->h) * ty;",
     "double py = (1.0 - 2.0 * y / c->h) * ty;"),
    ("thin-lens disk tilted out of the lens plane", "oo[k] += c->lens_radius * (disk[0] * r[k] + disk[1] * u[k]);",
     "oo[k] += c->lens_radius * (disk[0] * r[k] + disk[1] * f[k]);"),
    ("motion-blur origin at the end of the exposure",
     "tm = (s + vto_uniform(c->seed, (pix * S + s) << 1)) / S;\n            for (int k = 0; k < 3; ++k) oo[k] += tm * c->rs_velocity[k];",
     "tm = (s + vto_uniform(c->seed, (pix * S + s) << 1)) / S;\n            for (int k = 0; k < 3; ++k) oo[k] += c->rs_velocity[k];"),
    # more of the walk, the clip and the start cell
    ("nearest site ignores y", "double dd = dx * dx + dy * dy + dz * dz;", "double dd = dx * dx + dz * dz;"),
    ("far clip ignored", "if (hi < b) b = hi;", ""),
    ("cells before t_near composited", "s.a = t_in > t0 ? t_in : t0;", "s.a = t_in;"),
    ("plane distance not normalised", "return fabs(dot3(n, xm)) / sqrt(dot3(n, n));", "return fabs(dot3(n, xm));"),
    # more of the paper appearance model
    ("sigmoid of -z", "for (int ch = 0; ch < 3; ++ch) c[ch] = 1.0 / (1.0 + exp(-z[ch]));",
     "for (int ch = 0; ch < 3; ++ch) c[ch] = 1.0 / (1.0 + exp(z[ch]));"),
    ("view-dependent map read from the other texture", "const double* tv = sc->tex_vd + cell * RR * 3;",
     "const double* tv = sc->tex + cell * RR * 3;"),
    ("view-dependent texel gradients at the wrong direction", "double om[3] = {-drr[0], -drr[1], -drr[2]}, uvv[2];",
     "double om[3] = {drr[0], drr[1], drr[2]}, uvv[2];"),
    ("texel-space scale of the u derivative", "double cx = (x >= 0.0 && x <= R - 1.0) ? 0.5 * R : 0.0;",
     "double cx = (x >= 0.0 && x <= R - 1.0) ? R : 0.0;"),
    ("exit-point term of the origin cell dropped", "if (s->x_on == 1) xterm[q] += gt;", ""),
    # more of the distortion adjoint
    ("interval-start derivative with the wrong sign", "double dLda = gd * sa * (0.5 * dsbar - dds)",
     "double dLda = gd * sa * (0.5 * dsbar + dds)"),
    ("interval-end derivative dropped", "if (a->b == a->t_out && a->t_out < t1) xterm[k] += dLdb;", ""),
    ("ordering sign of the midpoints flipped", "(sk > sl ? 1.0 : (sk < sl ? -1.0 : 0.0))",
     "(sk > sl ? -1.0 : (sk < sl ? 1.0 : 0.0))"),
    # readings of ties and camera conventions
    ("nearest-site ties to the higher id", "if (dd < bd) {\n      bd = dd;", "if (dd <= bd) {\n      bd = dd;"),
    ("exact exit ties to the later CSR entry", "if (t < best_t) {", "if (t <= best_t) {"),
    ("fisheye azimuth axes swapped", "double cp = rr > 0.0 ? px / rr : 1.0, sp = rr > 0.0 ? py / rr : 0.0;",
     "double cp = rr > 0.0 ? py / rr : 1.0, sp = rr > 0.0 ? px / rr : 0.0;"),
    ("camera basis mirrored", "cross3(f, c->up, r);", "cross3(c->up, f, r);"),
    ("camera basis: wrong sign in a cross product", "c[0] = a[1] * b[2] - a[2] * b[1];",
     "c[0] = a[1] * b[2] + a[2] * b[1];"),
    ("pinhole aspect ratio inverted", "tx = ty * (double)c->w / (double)c->h;",
     "tx = ty / (double)c->w / (double)c->h;"),
    ("pinhole image mirrored", "for (int k = 0; k < 3; ++k) pd[k] = f[k] + px * r[k] + py * u[k];",
     "for (int k = 0; k < 3; ++k) pd[k] = f[k] - px * r[k] + py * u[k];"),
    # routing of gradients and the band test
    ("no site gradient at crossings into cell 0", "if (j < 0 || !isfinite(tb)) continue;",
     "if (j <= 0 || !isfinite(tb)) continue;"),
    ("first texel's gradient routed to a density", "else if (i < n4)\n", "else if (i <= n4)\n"),
    ("first view-dependent texel's gradient routed to the other map", "else if (i < nt)\n", "else if (i <= nt)\n"),
    ("distortion weight derivative divides by the distance", "dw += 2.0 * b->w * fabs(sk - sl);",
     "dw += 2.0 * b->w / fabs(sk - sl);"),
    ("band test: wrong plane normal", "double n[3] = {sb[0] - sa[0], sb[1] - sa[1], sb[2] - sa[2]};",
     "double n[3] = {sb[0] - sa[0], sb[1] - sa[1], sb[2] + sa[2]};"),
    ("band test: wrong plane midpoint",
     "double m[3] = {0.5 * (sa[0] + sb[0]), 0.5 * (sa[1] + sb[1]), 0.5 * (sa[2] + sb[2])};",
     "double m[3] = {0.5 * (sa[0] + sb[0]), 0.25 * (sa[1] + sb[1]), 0.5 * (sa[2] + sb[2])};"),
    ("band test: origin checked against the wrong site",
     "if (plane_dist(sc->sites + 3 * cell, sc->sites + 3 * (int64_t)sc->idx[q], o) < p->band_eps)",
     "if (plane_dist(sc->sites - 3 * cell, sc->sites + 3 * (int64_t)sc->idx[q], o) < p->band_eps)"),
    ("band test: wrong segment end point", "double xe[3] = {o[0] + te * d[0], o[1] + te * d[1], o[2] + te * d[2]};",
     "double xe[3] = {o[0] + te * d[0], o[1] - te * d[1], o[2] + te * d[2]};"),
    ("band test: segment end checked against the wrong neighbour",
     "if (plane_dist(si, sc->sites + 3 * j, xe) < p->band_eps) {", "if (plane_dist(si, sc->sites - 3 * j, xe) < p->band_eps) {"),
    ("band test: crossing near t_far never seen",
     "(fabs(best_t - t1) < p->band_eps || fabs(best_t - t0) < p->band_eps)",
     "(fabs(best_t + t1) < p->band_eps || fabs(best_t - t0) < p->band_eps)"),
    ("band test: crossing near t_near never seen",
     "(fabs(best_t - t1) < p->band_eps || fabs(best_t - t0) < p->band_eps)",
     "(fabs(best_t - t1) < p->band_eps || fabs(best_t + t0) < p->band_eps)"),
    ("band test: origin checked against the wrong neighbour",
     "if (plane_dist(sc->sites + 3 * cell, sc->sites + 3 * (int64_t)sc->idx[q], o) < p->band_eps)",
     "if (plane_dist(sc->sites + 3 * cell, sc->sites - 3 * (int64_t)sc->idx[q], o) < p->band_eps)"),
    ("termination band widened to 1e-2", "if (fabs(T / p->T_eps - 1.0) < 1e-4) *flags |= VTO_F_T_AMBIG;",
     "if (fabs(T / p->T_eps - 1.0) < 1e-2) *flags |= VTO_F_T_AMBIG;"),
    ("termination band narrowed to 1e-6", "if (fabs(T / p->T_eps - 1.0) < 1e-4) *flags |= VTO_F_T_AMBIG;",
     "if (fabs(T / p->T_eps - 1.0) < 1e-6) *flags |= VTO_F_T_AMBIG;"),
    ("termination band read on T before the cell",
     "T = T * e;\n      if (fabs(T / p->T_eps - 1.0) < 1e-4) *flags |= VTO_F_T_AMBIG;",
     "if (fabs(T / p->T_eps - 1.0) < 1e-4) *flags |= VTO_F_T_AMBIG;\n      T = T * e;"),
    ("termination band never flagged", "if (fabs(T / p->T_eps - 1.0) < 1e-4) *flags |= VTO_F_T_AMBIG;", ""),
    ("rolling-shutter origin fixed at mid-frame",
     "tm = (double)y / (double)c->h;\n            for (int k = 0; k < 3; ++k) oo[k] += tm * c->rs_velocity[k];",
     "tm = (double)y / (double)c->h;\n            for (int k = 0; k < 3; ++k) oo[k] += 0.5 * c->rs_velocity[k];"),
]


def _build(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-D_GNU_SOURCE", "-fPIC", "-shared", c,
                           "-o", so, "-lm", "-lpthread"])
    return so


def _run_pins(lib_path):
    env = dict(os.environ, VT_ORACLE_LIB=lib_path, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    tail = (r.stdout.strip().splitlines() or [""])[-1]
    return r.returncode, tail


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    jobs = [("unmutated", src)]
    for k, (what, a, b) in enumerate(MUTANTS):
        assert src.count(a) == 1, f"mutant {k} ({what}): target text not found once in the oracle"
        jobs.append((what, src.replace(a, b)))
    libs = [_build(text, str(tmp_path), f"m{k}") for k, (_, text) in enumerate(jobs)]
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run_pins, libs))
    rc0, tail0 = results[0]
    assert rc0 == 0, f"the pins fail on an unmutated copy of the oracle: {tail0}"
    # exit code 1 = tests failed (a crash or an error in collection would not count)
    missed = [(what, rc, tail) for (what, _), (rc, tail) in zip(jobs[1:], results[1:]) if rc != 1]
    assert not missed, f"mistakes no pin caught: {missed}"


# The numpy training helpers (oracle/training.py), mutated the same way and
# checked in-process by the pins that cover them.
TRAINING_SRC = os.path.join(ROOT, "oracle", "training.py")
TRAINING_PINS = ["test_smooth_l1_matches_library", "test_adam_matches_library",
                 "test_texture_regularizers_closed_forms_and_fd", "test_stratified_ray_sampling"]
TRAINING_MUTANTS = [
    ("Smooth-L1 linear branch offset by beta", "loss = np.where(small, 0.5 * r * r / beta, a - 0.5 * beta)",
     "loss = np.where(small, 0.5 * r * r / beta, a - beta)"),
    ("Smooth-L1 quadratic-branch gradient not divided by beta", "grad = np.where(small, r / beta, np.sign(r))",
     "grad = np.where(small, r, np.sign(r))"),
    ("Smooth-L1 gradient averaged over rays, not channels", "return loss.mean(), grad / r.size",
     "return loss.mean(), grad / len(r)"),
    ("regulariser normalised by N R, not N R^2", "scale = 1.0 / (n * R * R)", "scale = 1.0 / (n * R)"),
    ("L_mean without the cell mean", "dev = t - mean[:, None, None, :]", "dev = t"),
    ("L_mean gradient without its factor 2", "2.0 * lam_mean * scale * dev", "lam_mean * scale * dev"),
    ("L_vd gradient with the other weight", "2.0 * lam_vd * scale * v", "2.0 * lam_mean * scale * v"),
    ("Adam second moment of g, not g^2", "v = b2 * v + (1 - b2) * g * g", "v = b2 * v + (1 - b2) * np.abs(g)"),
    ("Adam without bias correction of m", "mh = m / (1 - b1 ** step)", "mh = m"),
    ("Adam epsilon inside the root", "p - lr * mh / (np.sqrt(vh) + eps)", "p - lr * mh / np.sqrt(vh + eps)"),
    ("stratified samples not jittered", "i = int((k + uniform(seed, k)) * stride)", "i = int((k + 0.5) * stride)"),
]


def test_every_planted_training_mistake_fails_a_pin(monkeypatch):
    import importlib.util

    import oracle
    import test_oracle_pins as pins

    src = open(TRAINING_SRC).read()

    def load(text, name):
        spec = importlib.util.spec_from_loader(f"oracle.{name}", loader=None, origin=TRAINING_SRC)
        mod = importlib.util.module_from_spec(spec)
        mod.__package__ = "oracle"
        exec(compile(text, TRAINING_SRC, "exec"), mod.__dict__)
        return mod

    def failures(mod):
        monkeypatch.setattr(oracle, "training", mod, raising=False)
        monkeypatch.setitem(sys.modules, "oracle.training", mod)
        n = 0
        for name in TRAINING_PINS:
            try:
                getattr(pins, name)()
            except AssertionError:
                n += 1
        return n

    assert failures(load(src, "training_unmutated")) == 0
    missed = []
    for k, (what, a, b) in enumerate(TRAINING_MUTANTS):
        assert src.count(a) == 1, f"training mutant {k} ({what}): target text not found once"
        if failures(load(src.replace(a, b), f"training_m{k}")) == 0:
            missed.append(what)
    assert not missed, f"mistakes no pin caught: {missed}"
