/*
 * vt_oracle.c -- plain, slow, FP64 CPU reference ("oracle") for differentiable
 * volume rendering by ray traversal of a 3D Voronoi diagram.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library. The CUDA library never
 * links, calls or includes anything from here, and this file includes nothing
 * from the CUDA library: the two share no code, headers or constants.
 *
 * Everything is computed in double precision on double inputs (the Python
 * wrapper promotes the FP32 scene and rays exactly). The oracle follows the
 * plain definitions of the paper:
 *   - Voronoi cell V_i = points nearest site p_i (Sec. 3.1).
 *   - Start cell = nearest site of the ray origin, by brute force over all
 *     sites (Sec. 3.1: the walk starts from one nearest-site lookup); ties -> lowest id.
 *   - Exit from cell i = nearest forward crossing of the bisector planes with
 *     the Delaunay neighbours j (Sec. 3.1 and its walk figure):
 *       t_j = n.((s_i+s_j)/2 - o) / (n.d),  n = s_j - s_i, only n.d > 0.
 *   - Piecewise-constant volume rendering (Sec. 3.2):
 *       alpha_k = 1 - exp(-sigma_{i_k} delta_k), T_{k+1} = T_k (1 - alpha_k),
 *       C = sum_k T_k alpha_k c_k + T_final * bg,
 *     stopping after the cell at which T < T_eps (early termination, Sec. 3.2).
 *   - Colour = bilinear fetch of the cell's R x R octahedral texture at the
 *     ray direction (Sec. 5.1 octahedral map, evaluated at the ray direction);
 *     or, in appearance mode 1, the paper's model (Sec. 5.1-5.2):
 *       c = sigmoid(T_vi(oct((x - p_i)/|x - p_i|)) + T_vd(oct(omega))),
 *     x = the point where the ray enters the cell (for the cell holding the
 *     origin: where it leaves it, or the end of its segment if it never
 *     leaves), omega = -d/|d| (towards the ray origin).
 *   - Backward: analytic adjoint of the above from the stored segment list
 *     (density gradient consistent with Eq. 3; plane-crossing gradient by
 *     differentiating t_j with respect to both sites).
 *   - Distortion loss of Mip-NeRF 360 (Eq. 2) per ray, over the composited
 *     intervals [a_k, b_k] with weights w_k = T_k alpha_k and s(t) = 1 - 1/(1+t):
 *       L = sum_{k,l} w_k w_l |sbar_k - sbar_l| + 1/3 sum_k w_k^2 ds_k,
 *     written out as the double sum; its gradient from the same definition.
 *   - Ray generation for pinhole, equidistant fisheye, rolling-shutter,
 *     thin-lens and motion-blur cameras (Sec. 6.5 and the application appendix).
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   sign(0) = +1 in the lower-hemisphere unfold; texel coordinates clamp to
 *   the edge; exact t ties keep the lower CSR position; termination is tested
 *   after compositing the current cell; the background is added with the final
 *   transmittance; the skip test is strict (w < skip_weight skips); the
 *   distortion loss runs over the composited intervals of the walk (after early
 *   termination) with t the ray parameter; motion blur samples the exposure
 *   [0, 1) in S jittered strata with linear camera motion.
 *
 * Parity pins for every function live in tests/test_oracle_pins.py; the
 * skip_weight > 0 rule (Sec. 5.6: below the threshold a cell attenuates T but
 * adds no colour) is pinned by a two-cell closed form of colour and adjoint.
 * tests/test_oracle_mutations.py compiles copies of this file, each with one
 * plausible mistake planted, and checks that the pins fail on every copy.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define VTO_OK 0
#define VTO_ERR_ARG 1
#define VTO_ERR_MEM 3

/* per-ray flag bits (degenerate band, see vto_params.band_eps) */
#define VTO_F_NEAR_EDGE 1    /* exit point within band_eps of another plane   */
#define VTO_F_NEAR_ORIGIN 2  /* origin within band_eps of a plane of its cell */
#define VTO_F_NEAR_CLIP 4    /* a crossing within band_eps of t_near'/t_far'  */
#define VTO_F_T_AMBIG 8      /* |T/T_eps - 1| < 1e-4 at some composited step  */
#define VTO_F_SKIP_AMBIG 16  /* |w/skip - 1| < 1e-4 at some step (skip > 0)   */
#define VTO_F_MAX_STEPS 32   /* walk exceeded max_steps                       */
#define VTO_F_BAD_RAY 64     /* zero / non-finite direction                   */

typedef struct {
  double t_near, t_far;
  int32_t use_clip_box;
  double clip_lo[3], clip_hi[3];
  double T_eps;
  double skip_weight;
  double bg[3];
  int32_t max_steps;
  double band_eps;
  int32_t appearance; /* 0: one texture at the ray direction; 1: Sec. 5.1-5.2 model */
} vto_params;

typedef struct {
  int64_t n;
  const double* sites; /* [n,3]        */
  const double* sigma; /* [n]          */
  const double* tex;   /* [n,R,R,3]    */
  int32_t R;
  const int64_t* off; /* [n+1]        */
  const int32_t* idx; /* [E]          */
  const double* tex_vd; /* [n,R,R,3] view-dependent logits (appearance 1) */
} vto_scene;

/* ------------------------------------------------------------------ */
/* Octahedral map, Sec. 5.1: l1-normalise, upper hemisphere maps to the
 * central diamond, points with z < 0 fold out into the four corners.   */
int vto_oct(const double d[3], double uv[2]) {
  double l1 = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
  if (!(l1 > 0.0) || !isfinite(l1)) return VTO_ERR_ARG;
  double qx = d[0] / l1, qy = d[1] / l1;
  if (d[2] >= 0.0) {
    uv[0] = qx;
    uv[1] = qy;
  } else {
    double sx = (qx >= 0.0) ? 1.0 : -1.0; /* sign(0) = +1 (reading) */
    double sy = (qy >= 0.0) ? 1.0 : -1.0;
    uv[0] = (1.0 - fabs(qy)) * sx;
    uv[1] = (1.0 - fabs(qx)) * sy;
  }
  return VTO_OK;
}

/* Bilinear taps: (u,v) in [-1,1]^2 rescaled to texel space, texel centres at
 * integer coordinates, clamp to edge (reading). Texel index = y*R + x.      */
void vto_bilinear_taps(int32_t R, double u, double v, int64_t idx[4], double w[4]) {
  double x = (u + 1.0) * 0.5 * R - 0.5;
  double y = (v + 1.0) * 0.5 * R - 0.5;
  if (x < 0.0) x = 0.0;
  if (x > R - 1.0) x = R - 1.0;
  if (y < 0.0) y = 0.0;
  if (y > R - 1.0) y = R - 1.0;
  int64_t x0 = (int64_t)floor(x), y0 = (int64_t)floor(y);
  if (x0 > R - 1) x0 = R - 1;
  if (y0 > R - 1) y0 = R - 1;
  int64_t x1 = x0 + 1 < R ? x0 + 1 : R - 1;
  int64_t y1 = y0 + 1 < R ? y0 + 1 : R - 1;
  double fx = x - (double)x0, fy = y - (double)y0;
  idx[0] = y0 * R + x0;
  idx[1] = y0 * R + x1;
  idx[2] = y1 * R + x0;
  idx[3] = y1 * R + x1;
  w[0] = (1.0 - fx) * (1.0 - fy);
  w[1] = fx * (1.0 - fy);
  w[2] = (1.0 - fx) * fy;
  w[3] = fx * fy;
}

/* Cell colour at direction d: bilinear fetch of texture of `cell`. */
static void cell_colour(const vto_scene* sc, int64_t cell, const int64_t taps[4], const double tw[4],
                        double c[3]) {
  const double* t = sc->tex + cell * (int64_t)sc->R * sc->R * 3;
  c[0] = c[1] = c[2] = 0.0;
  for (int q = 0; q < 4; ++q)
    for (int ch = 0; ch < 3; ++ch) c[ch] += tw[q] * t[taps[q] * 3 + ch];
}

/* Appearance 1 (Sec. 5.1-5.2): logit z = T_vi(oct(dsurf)) + T_vd(oct(-d)),
 * c = sigmoid(z). */
static void cell_colour_paper(const vto_scene* sc, int64_t cell, const double dsurf[3], const double d[3],
                              double c[3]) {
  int64_t RR = (int64_t)sc->R * sc->R;
  double uv[2], w[4];
  int64_t tp[4];
  double z[3] = {0.0, 0.0, 0.0};
  vto_oct(dsurf, uv);
  vto_bilinear_taps(sc->R, uv[0], uv[1], tp, w);
  const double* t = sc->tex + cell * RR * 3;
  for (int q = 0; q < 4; ++q)
    for (int ch = 0; ch < 3; ++ch) z[ch] += w[q] * t[tp[q] * 3 + ch];
  double om[3] = {-d[0], -d[1], -d[2]};
  vto_oct(om, uv);
  vto_bilinear_taps(sc->R, uv[0], uv[1], tp, w);
  const double* tv = sc->tex_vd + cell * RR * 3;
  for (int q = 0; q < 4; ++q)
    for (int ch = 0; ch < 3; ++ch) z[ch] += w[q] * tv[tp[q] * 3 + ch];
  for (int ch = 0; ch < 3; ++ch) c[ch] = 1.0 / (1.0 + exp(-z[ch]));
}

/* Brute-force nearest site (Sec. 3.1 cell definition); ties -> lowest id. */
int64_t vto_nearest(int64_t n, const double* sites, const double q[3]) {
  int64_t best = -1;
  double bd = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double dx = q[0] - sites[3 * i], dy = q[1] - sites[3 * i + 1], dz = q[2] - sites[3 * i + 2];
    double dd = dx * dx + dy * dy + dz * dz;
    if (dd < bd) {
      bd = dd;
      best = i;
    }
  }
  return best;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* distance from x to the bisector plane of sites a, b */
static double plane_dist(const double* sa, const double* sb, const double x[3]) {
  double n[3] = {sb[0] - sa[0], sb[1] - sa[1], sb[2] - sa[2]};
  double m[3] = {0.5 * (sa[0] + sb[0]), 0.5 * (sa[1] + sb[1]), 0.5 * (sa[2] + sb[2])};
  double xm[3] = {x[0] - m[0], x[1] - m[1], x[2] - m[2]};
  return fabs(dot3(n, xm)) / sqrt(dot3(n, n));
}

/* One walked cell of a ray. */
typedef struct {
  int64_t cell;
  double t_in, t_out; /* walked parameter interval; t_out = +inf if unbounded */
  int64_t next;       /* exit neighbour, -1 if none                             */
  double a, b;        /* composited interval (clipped); composited iff b > a   */
  int32_t composited, coloured;
  double delta, alpha, T_before, w;
  double c[3];
  /* appearance 1: surface point x = o + t_x d, which crossing it lies on
   * (0: entry face, 1: exit face, -1: none), direction from the site */
  double t_x, dsurf[3], rlen;
  int32_t x_on;
} vto_seg;

typedef struct {
  vto_seg* s;
  int64_t n, cap;
} seg_buf;

static int seg_push(seg_buf* b, const vto_seg* s) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 64;
    vto_seg* ns = (vto_seg*)realloc(b->s, (size_t)nc * sizeof(vto_seg));
    if (!ns) return VTO_ERR_MEM;
    b->s = ns;
    b->cap = nc;
  }
  b->s[b->n++] = *s;
  return VTO_OK;
}

/* Clip [t_near, t_far] against the optional axis-aligned box (slab test). */
static void clip_extent(const vto_params* p, const double o[3], const double d[3], double* t0,
                        double* t1) {
  double a = p->t_near, b = p->t_far;
  if (p->use_clip_box) {
    for (int k = 0; k < 3; ++k) {
      if (d[k] != 0.0) {
        double ta = (p->clip_lo[k] - o[k]) / d[k], tb = (p->clip_hi[k] - o[k]) / d[k];
        double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
        if (lo > a) a = lo;
        if (hi < b) b = hi;
      } else if (o[k] < p->clip_lo[k] || o[k] > p->clip_hi[k]) {
        b = a; /* parallel to the slab and outside: miss */
      }
    }
  }
  *t0 = a;
  *t1 = b;
}

/* Walk and composite one ray. Fills the segment list, colour, transmittance,
 * visited-cell count and band flags. Returns VTO_OK or VTO_ERR_MEM.        */
static int walk_ray(const vto_scene* sc, const vto_params* p, const double o[3], const double d[3],
                    seg_buf* segs, double C[3], double* T_out, int32_t* steps, int32_t* flags,
                    int64_t* last_next, double* last_t_out) {
  segs->n = 0;
  *flags = 0;
  C[0] = C[1] = C[2] = 0.0;
  *T_out = 1.0;
  *steps = 0;
  *last_next = -1;
  *last_t_out = INFINITY;
  double dn = sqrt(dot3(d, d));
  if (!(dn > 0.0) || !isfinite(dn)) {
    *flags |= VTO_F_BAD_RAY;
    return VTO_OK;
  }
  double t0, t1;
  clip_extent(p, o, d, &t0, &t1);
  if (!(t1 > t0)) {
    for (int ch = 0; ch < 3; ++ch) C[ch] = p->bg[ch];
    return VTO_OK;
  }
  double uv[2];
  vto_oct(d, uv);
  int64_t taps[4];
  double tw[4];
  vto_bilinear_taps(sc->R, uv[0], uv[1], taps, tw);

  int64_t cell = vto_nearest(sc->n, sc->sites, o);
  /* origin within band of a plane of its cell */
  for (int64_t q = sc->off[cell]; q < sc->off[cell + 1]; ++q) {
    if (plane_dist(sc->sites + 3 * cell, sc->sites + 3 * (int64_t)sc->idx[q], o) < p->band_eps)
      *flags |= VTO_F_NEAR_ORIGIN;
  }
  double T = 1.0, t_in = 0.0;
  int32_t k = 0;
  for (;;) {
    if (k >= p->max_steps) {
      *flags |= VTO_F_MAX_STEPS;
      break;
    }
    ++k;
    const double* si = sc->sites + 3 * cell;
    double best_t = INFINITY;
    int64_t best_j = -1;
    for (int64_t q = sc->off[cell]; q < sc->off[cell + 1]; ++q) {
      int64_t j = sc->idx[q];
      const double* sj = sc->sites + 3 * j;
      double n[3] = {sj[0] - si[0], sj[1] - si[1], sj[2] - si[2]};
      double den = dot3(n, d);
      if (!(den > 0.0)) continue;
      double mo[3] = {0.5 * (si[0] + sj[0]) - o[0], 0.5 * (si[1] + sj[1]) - o[1],
                      0.5 * (si[2] + sj[2]) - o[2]};
      double t = dot3(n, mo) / den;
      if (t < best_t) { /* strict: exact ties keep the lower CSR position */
        best_t = t;
        best_j = j;
      }
    }
    vto_seg s;
    memset(&s, 0, sizeof(s));
    s.cell = cell;
    s.t_in = t_in;
    s.t_out = best_t;
    s.next = best_j;
    s.a = t_in > t0 ? t_in : t0;
    s.b = best_t < t1 ? best_t : t1;
    s.T_before = T;
    /* band: the point where this segment ends is close to another plane */
    {
      double te = best_t < t1 ? best_t : t1;
      if (isfinite(te)) {
        double xe[3] = {o[0] + te * d[0], o[1] + te * d[1], o[2] + te * d[2]};
        for (int64_t q = sc->off[cell]; q < sc->off[cell + 1]; ++q) {
          int64_t j = sc->idx[q];
          if (j == best_j && best_t < t1) continue;
          if (plane_dist(si, sc->sites + 3 * j, xe) < p->band_eps) {
            *flags |= (best_t < t1) ? VTO_F_NEAR_EDGE : VTO_F_NEAR_CLIP;
          }
        }
      }
      if (isfinite(best_t) && (fabs(best_t - t1) < p->band_eps || fabs(best_t - t0) < p->band_eps))
        *flags |= VTO_F_NEAR_CLIP;
    }
    int stop = 0;
    if (s.b > s.a) {
      double delta = s.b - s.a;
      double sig = sc->sigma[cell];
      double e = exp(-sig * delta);
      double alpha = 1.0 - e;
      double w = T * alpha;
      s.composited = 1;
      s.delta = delta;
      s.alpha = alpha;
      s.w = w;
      if (p->skip_weight > 0.0 && fabs(w / p->skip_weight - 1.0) < 1e-4) *flags |= VTO_F_SKIP_AMBIG;
      if (!(p->skip_weight > 0.0) || w >= p->skip_weight) {
        s.coloured = 1;
        if (p->appearance == 1) {
          /* surface point: entry face, else (origin cell) exit face, else segment end */
          if (k > 1) {
            s.t_x = t_in;
            s.x_on = 0;
          } else if (isfinite(best_t)) {
            s.t_x = best_t;
            s.x_on = 1;
          } else {
            s.t_x = t1;
            s.x_on = -1;
          }
          double v[3] = {o[0] + s.t_x * d[0] - si[0], o[1] + s.t_x * d[1] - si[1], o[2] + s.t_x * d[2] - si[2]};
          s.rlen = sqrt(dot3(v, v));
          for (int c3 = 0; c3 < 3; ++c3) s.dsurf[c3] = s.rlen > 0.0 ? v[c3] / s.rlen : d[c3] / dn;
          cell_colour_paper(sc, cell, s.dsurf, d, s.c);
        } else {
          cell_colour(sc, cell, taps, tw, s.c);
        }
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * s.c[ch];
      }
      T = T * e;
      if (fabs(T / p->T_eps - 1.0) < 1e-4) *flags |= VTO_F_T_AMBIG;
      if (T < p->T_eps) stop = 1;
    }
    if (seg_push(segs, &s) != VTO_OK) return VTO_ERR_MEM;
    *last_next = best_j;
    *last_t_out = best_t;
    if (stop || !(best_t < t1) || best_j < 0) break;
    cell = best_j;
    t_in = best_t;
  }
  for (int ch = 0; ch < 3; ++ch) C[ch] += T * p->bg[ch];
  *T_out = T;
  *steps = k;
  return VTO_OK;
}

/* ------------------------------------------------------------------ */
/* Forward render, threaded over rays.                                  */
typedef struct {
  const vto_scene* sc;
  const vto_params* p;
  const double *o, *d;
  double *rgb, *T;
  int32_t *steps, *flags;
  int64_t lo, hi;
  /* optional trace output: per ray up to max_cells cells */
  int32_t max_cells;
  int32_t* cells;
  double* t_out;
  int32_t* n_cells;
  int status;
} render_job;

static void* render_worker(void* arg) {
  render_job* J = (render_job*)arg;
  seg_buf b = {0, 0, 0};
  J->status = VTO_OK;
  for (int64_t r = J->lo; r < J->hi; ++r) {
    double C[3], T;
    int32_t k, fl;
    int64_t ln;
    double lt;
    if (walk_ray(J->sc, J->p, J->o + 3 * r, J->d + 3 * r, &b, C, &T, &k, &fl, &ln, &lt) != VTO_OK) {
      J->status = VTO_ERR_MEM;
      break;
    }
    if (J->rgb)
      for (int ch = 0; ch < 3; ++ch) J->rgb[3 * r + ch] = C[ch];
    if (J->T) J->T[r] = T;
    if (J->steps) J->steps[r] = k;
    if (J->flags) J->flags[r] = fl;
    if (J->cells) {
      int64_t m = b.n < J->max_cells ? b.n : J->max_cells;
      for (int64_t q = 0; q < m; ++q) {
        J->cells[r * J->max_cells + q] = (int32_t)b.s[q].cell;
        if (J->t_out) J->t_out[r * J->max_cells + q] = b.s[q].t_out;
      }
      J->n_cells[r] = (int32_t)b.n;
    }
  }
  free(b.s);
  return NULL;
}

static int run_threads(render_job* proto, int64_t n_rays, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_rays < n_threads) n_threads = n_rays > 0 ? (int)n_rays : 1;
  pthread_t th[256];
  render_job jobs[256];
  int64_t chunk = (n_rays + n_threads - 1) / n_threads;
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = *proto;
    jobs[t].lo = t * chunk;
    jobs[t].hi = (t + 1) * chunk < n_rays ? (t + 1) * chunk : n_rays;
    if (jobs[t].lo >= jobs[t].hi) continue;
    if (n_threads == 1) {
      render_worker(&jobs[t]);
      continue;
    }
    pthread_create(&th[t], NULL, render_worker, &jobs[t]);
    started |= 1;
  }
  int st = VTO_OK;
  for (int t = 0; t < n_threads; ++t) {
    if (jobs[t].lo >= jobs[t].hi) continue;
    if (n_threads > 1) pthread_join(th[t], NULL);
    if (jobs[t].status != VTO_OK) st = jobs[t].status;
  }
  (void)started;
  return st;
}

int vto_render(const vto_scene* sc, int64_t n_rays, const double* o, const double* d,
               const vto_params* p, double* rgb, double* T, int32_t* steps, int32_t* flags,
               int n_threads) {
  render_job J;
  memset(&J, 0, sizeof(J));
  J.sc = sc;
  J.p = p;
  J.o = o;
  J.d = d;
  J.rgb = rgb;
  J.T = T;
  J.steps = steps;
  J.flags = flags;
  return run_threads(&J, n_rays, n_threads);
}

/* Per-ray visited cells (walk order) and exit parameters, up to max_cells. */
int vto_trace(const vto_scene* sc, int64_t n_rays, const double* o, const double* d,
              const vto_params* p, int32_t max_cells, int32_t* cells, double* t_out,
              int32_t* n_cells, int32_t* flags, int n_threads) {
  render_job J;
  memset(&J, 0, sizeof(J));
  J.sc = sc;
  J.p = p;
  J.o = o;
  J.d = d;
  J.flags = flags;
  J.max_cells = max_cells;
  J.cells = cells;
  J.t_out = t_out;
  J.n_cells = n_cells;
  return run_threads(&J, n_rays, n_threads);
}

/* Full segment list of one ray (for pins): arrays of length cap. Returns the
 * number of walked cells, or -1 on error.                                   */
int64_t vto_segments(const vto_scene* sc, const double o[3], const double d[3], const vto_params* p,
                     int64_t cap, int64_t* cell, double* a, double* b, double* delta,
                     int32_t* composited, double* T_before, double* alpha) {
  seg_buf sb = {0, 0, 0};
  double C[3], T;
  int32_t k, fl;
  int64_t ln;
  double lt;
  if (walk_ray(sc, p, o, d, &sb, C, &T, &k, &fl, &ln, &lt) != VTO_OK) {
    free(sb.s);
    return -1;
  }
  int64_t m = sb.n < cap ? sb.n : cap;
  for (int64_t q = 0; q < m; ++q) {
    cell[q] = sb.s[q].cell;
    a[q] = sb.s[q].a;
    b[q] = sb.s[q].b;
    delta[q] = sb.s[q].delta;
    composited[q] = sb.s[q].composited;
    T_before[q] = sb.s[q].T_before;
    alpha[q] = sb.s[q].alpha;
  }
  int64_t n = sb.n;
  free(sb.s);
  return n;
}

/* Bilinear value and its derivatives with respect to (u, v) for one cell's
 * texture (zero derivative where the texel coordinate is clamped). */
static void bilinear_uv_grad(int32_t R, const double* t, double u, double v, double dzdu[3], double dzdv[3]) {
  double x = (u + 1.0) * 0.5 * R - 0.5, y = (v + 1.0) * 0.5 * R - 0.5;
  double cx = (x >= 0.0 && x <= R - 1.0) ? 0.5 * R : 0.0;
  double cy = (y >= 0.0 && y <= R - 1.0) ? 0.5 * R : 0.0;
  if (x < 0.0) x = 0.0;
  if (x > R - 1.0) x = R - 1.0;
  if (y < 0.0) y = 0.0;
  if (y > R - 1.0) y = R - 1.0;
  int64_t x0 = (int64_t)floor(x), y0 = (int64_t)floor(y);
  if (x0 > R - 1) x0 = R - 1;
  if (y0 > R - 1) y0 = R - 1;
  int64_t x1 = x0 + 1 < R ? x0 + 1 : R - 1, y1 = y0 + 1 < R ? y0 + 1 : R - 1;
  double fx = x - (double)x0, fy = y - (double)y0;
  for (int c = 0; c < 3; ++c) {
    double t00 = t[(y0 * R + x0) * 3 + c], t01 = t[(y0 * R + x1) * 3 + c];
    double t10 = t[(y1 * R + x0) * 3 + c], t11 = t[(y1 * R + x1) * 3 + c];
    dzdu[c] = cx * ((1.0 - fy) * (t01 - t00) + fy * (t11 - t10));
    dzdv[c] = cy * ((1.0 - fx) * (t10 - t00) + fx * (t11 - t01));
  }
}

/* g_d = (d(u,v)/dd)^T (gu, gv) for the octahedral map of direction d. */
static void oct_vjp(const double d[3], double gu, double gv, double gd[3]) {
  double l1 = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
  double q[3] = {d[0] / l1, d[1] / l1, d[2] / l1};
  double sg[3] = {d[0] >= 0.0 ? 1.0 : -1.0, d[1] >= 0.0 ? 1.0 : -1.0, d[2] >= 0.0 ? 1.0 : -1.0};
  for (int j = 0; j < 3; ++j) {
    double dq0 = ((j == 0) - q[0] * sg[j]) / l1, dq1 = ((j == 1) - q[1] * sg[j]) / l1;
    double du, dv;
    if (d[2] >= 0.0) {
      du = dq0;
      dv = dq1;
    } else {
      du = -sg[0] * sg[1] * dq1;
      dv = -sg[1] * sg[0] * dq0;
    }
    gd[j] = gu * du + gv * dv;
  }
}

/* ------------------------------------------------------------------ */
/* Distortion loss (Eq. 2) from the plain definition.                    */
static double s_of_t(double t) { return 1.0 - 1.0 / (1.0 + t); }

static double ray_distortion(const seg_buf* sb) {
  double L = 0.0;
  for (int64_t k = 0; k < sb->n; ++k) {
    const vto_seg* a = &sb->s[k];
    if (!a->composited) continue;
    double sk = 0.5 * (s_of_t(a->a) + s_of_t(a->b));
    for (int64_t l = 0; l < sb->n; ++l) {
      const vto_seg* b = &sb->s[l];
      if (!b->composited) continue;
      double sl = 0.5 * (s_of_t(b->a) + s_of_t(b->b));
      L += a->w * b->w * fabs(sk - sl);
    }
    L += a->w * a->w * (s_of_t(a->b) - s_of_t(a->a)) / 3.0;
  }
  return L;
}

/* Adds gd * dL_dist/dtau_k to dtau[] and the direct derivatives of L_dist
 * with respect to the interval ends to the crossing terms xterm[] (index q:
 * the crossing at the exit of walked cell q):
 *   dL/dw_k    = 2 sum_l w_l |sbar_k - sbar_l| + 2/3 w_k ds_k
 *   dL/dsbar_k = 2 w_k sum_l w_l sign(sbar_k - sbar_l)
 *   dL/dds_k   = w_k^2 / 3
 *   w_k = T_k alpha_k: dw_k/dtau_j = -w_k (j < k), T_{k+1} (j = k)
 *   sbar = (s(a)+s(b))/2, ds = s(b)-s(a), s'(t) = 1/(1+t)^2.
 * An interval end moves with a crossing only where it is one (b_k = exit
 * crossing below t_far', a_k = entry crossing above t_near').            */
static void ray_distortion_bwd(const seg_buf* sb, double gd, double t0, double t1, double* dtau, double* xterm) {
  for (int64_t k = 0; k < sb->n; ++k) {
    const vto_seg* a = &sb->s[k];
    if (!a->composited) continue;
    double sk = 0.5 * (s_of_t(a->a) + s_of_t(a->b));
    double dw = 0.0, dsbar = 0.0;
    for (int64_t l = 0; l < sb->n; ++l) {
      const vto_seg* b = &sb->s[l];
      if (!b->composited) continue;
      double sl = 0.5 * (s_of_t(b->a) + s_of_t(b->b));
      dw += 2.0 * b->w * fabs(sk - sl);
      if (l != k) dsbar += 2.0 * a->w * b->w * (sk > sl ? 1.0 : (sk < sl ? -1.0 : 0.0));
    }
    double dsk = s_of_t(a->b) - s_of_t(a->a);
    dw += 2.0 / 3.0 * a->w * dsk;
    double dds = a->w * a->w / 3.0;
    /* through the weights */
    dtau[k] += gd * dw * a->T_before * (1.0 - a->alpha);
    for (int64_t j = 0; j < k; ++j)
      if (sb->s[j].composited) dtau[j] -= gd * dw * a->w;
    /* through the interval ends */
    double sa = 1.0 / ((1.0 + a->a) * (1.0 + a->a)), sbb = 1.0 / ((1.0 + a->b) * (1.0 + a->b));
    double dLda = gd * sa * (0.5 * dsbar - dds), dLdb = gd * sbb * (0.5 * dsbar + dds);
    if (a->b == a->t_out && a->t_out < t1) xterm[k] += dLdb;
    if (k > 0 && a->a == a->t_in && a->t_in > t0) xterm[k - 1] += dLda;
  }
}

/* Gradient contributions are produced per thread as (flat index, value)
 * pairs -- flat index: [0,3N) sites, [3N,4N) sigma, then texels -- and added
 * into the outputs under a mutex. */
typedef struct {
  int64_t i;
  double v;
} contrib;

typedef struct {
  contrib* c;
  int64_t n, cap;
} contrib_buf;

typedef struct {
  const vto_scene* sc;
  const vto_params* p;
  const double *o, *d, *g;
  const double* gdist; /* dL/dL_dist per ray, or NULL */
  double *g_sites, *g_sigma, *g_tex, *g_tex_vd;
  int64_t lo, hi;
  pthread_mutex_t* mu;
  int status;
} bwd_job;

static int emit(contrib_buf* b, int64_t i, double v) {
  if (v == 0.0) return VTO_OK;
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 4096;
    contrib* nb = (contrib*)realloc(b->c, (size_t)nc * sizeof(contrib));
    if (!nb) return VTO_ERR_MEM;
    b->c = nb;
    b->cap = nc;
  }
  b->c[b->n].i = i;
  b->c[b->n].v = v;
  b->n++;
  return VTO_OK;
}

static void flush_contribs(bwd_job* J, contrib_buf* b) {
  int64_t n3 = 3 * J->sc->n, n4 = 4 * J->sc->n;
  int64_t nt = n4 + J->sc->n * (int64_t)J->sc->R * J->sc->R * 3;
  pthread_mutex_lock(J->mu);
  for (int64_t k = 0; k < b->n; ++k) {
    int64_t i = b->c[k].i;
    if (i < n3)
      J->g_sites[i] += b->c[k].v;
    else if (i < n4)
      J->g_sigma[i - n3] += b->c[k].v;
    else if (i < nt)
      J->g_tex[i - n4] += b->c[k].v;
    else if (J->g_tex_vd)
      J->g_tex_vd[i - nt] += b->c[k].v;
  }
  pthread_mutex_unlock(J->mu);
  b->n = 0;
}

static void* bwd_worker(void* arg) {
  bwd_job* J = (bwd_job*)arg;
  const vto_scene* sc = J->sc;
  const vto_params* p = J->p;
  seg_buf sb = {0, 0, 0};
  contrib_buf cb = {0, 0, 0};
  double* dtau = NULL;
  double* xterm = NULL;
  int64_t dcap = 0;
  const int64_t RR = (int64_t)sc->R * sc->R, n3 = 3 * sc->n, n4 = 4 * sc->n;
  J->status = VTO_OK;
  for (int64_t r = J->lo; r < J->hi && J->status == VTO_OK; ++r) {
    const double* orr = J->o + 3 * r;
    const double* drr = J->d + 3 * r;
    double C[3], T;
    int32_t k, fl;
    int64_t last_next;
    double last_t;
    if (walk_ray(sc, p, orr, drr, &sb, C, &T, &k, &fl, &last_next, &last_t) != VTO_OK) {
      J->status = VTO_ERR_MEM;
      break;
    }
    if (fl & VTO_F_BAD_RAY) continue;
    const double* g = J->g + 3 * r;
    double t0, t1;
    clip_extent(p, orr, drr, &t0, &t1);
    if (!(t1 > t0)) continue;
    if (sb.n > dcap) {
      dcap = sb.n * 2;
      double* nd = (double*)realloc(dtau, (size_t)dcap * sizeof(double));
      double* nx = (double*)realloc(xterm, (size_t)dcap * sizeof(double));
      if (nd) dtau = nd;
      if (nx) xterm = nx;
      if (!nd || !nx) {
        J->status = VTO_ERR_MEM;
        break;
      }
    }
    double uv[2];
    vto_oct(drr, uv);
    int64_t taps[4];
    double tw[4];
    vto_bilinear_taps(sc->R, uv[0], uv[1], taps, tw);
    /* suffix S_k computed back to front from T_final * bg */
    double S[3] = {T * p->bg[0], T * p->bg[1], T * p->bg[2]};
    for (int64_t q = sb.n - 1; q >= 0; --q) {
      vto_seg* s = &sb.s[q];
      dtau[q] = 0.0;
      if (!s->composited) continue;
      double Tn = s->T_before * (1.0 - s->alpha);
      double acc = 0.0;
      for (int ch = 0; ch < 3; ++ch) acc += g[ch] * (Tn * (s->coloured ? s->c[ch] : 0.0) - S[ch]);
      dtau[q] = acc;
      if (s->coloured)
        for (int ch = 0; ch < 3; ++ch) S[ch] += s->w * s->c[ch];
    }
    int st = VTO_OK;
    const int64_t ntex = n4 + sc->n * RR * 3;
    /* direct dL/dt terms of crossings: appearance 1 colour and the distortion loss */
    for (int64_t q = 0; q < sb.n; ++q) xterm[q] = 0.0;
    if (J->gdist && J->gdist[r] != 0.0) ray_distortion_bwd(&sb, J->gdist[r], t0, t1, dtau, xterm);
    for (int64_t q = 0; q < sb.n && st == VTO_OK; ++q) {
      vto_seg* s = &sb.s[q];
      int64_t i = s->cell;
      if (s->composited) {
        st |= emit(&cb, n3 + i, dtau[q] * s->delta);
        if (s->coloured && p->appearance == 1) {
          /* c = sigmoid(z): dL/dz = g w c (1 - c) */
          double gz[3];
          for (int ch = 0; ch < 3; ++ch) gz[ch] = g[ch] * s->w * s->c[ch] * (1.0 - s->c[ch]);
          double uv[2], tw2[4];
          int64_t tp2[4];
          vto_oct(s->dsurf, uv);
          vto_bilinear_taps(sc->R, uv[0], uv[1], tp2, tw2);
          for (int tq = 0; tq < 4; ++tq)
            for (int ch = 0; ch < 3; ++ch) st |= emit(&cb, n4 + (i * RR + tp2[tq]) * 3 + ch, gz[ch] * tw2[tq]);
          double om[3] = {-drr[0], -drr[1], -drr[2]}, uvv[2];
          vto_oct(om, uvv);
          vto_bilinear_taps(sc->R, uvv[0], uvv[1], tp2, tw2);
          for (int tq = 0; tq < 4; ++tq)
            for (int ch = 0; ch < 3; ++ch) st |= emit(&cb, ntex + (i * RR + tp2[tq]) * 3 + ch, gz[ch] * tw2[tq]);
          /* through the surface direction: dsurf = (x - p)/|x - p|, x = o + t_x d */
          double dzdu[3], dzdv[3];
          bilinear_uv_grad(sc->R, sc->tex + i * RR * 3, uv[0], uv[1], dzdu, dzdv);
          double gu = 0.0, gv = 0.0;
          for (int ch = 0; ch < 3; ++ch) {
            gu += gz[ch] * dzdu[ch];
            gv += gz[ch] * dzdv[ch];
          }
          double gd[3];
          oct_vjp(s->dsurf, gu, gv, gd);
          if (s->rlen > 0.0) {
            double dd = dot3(gd, s->dsurf);
            double gx[3];
            for (int c3 = 0; c3 < 3; ++c3) gx[c3] = (gd[c3] - s->dsurf[c3] * dd) / s->rlen;
            for (int c3 = 0; c3 < 3; ++c3) st |= emit(&cb, 3 * i + c3, -gx[c3]);
            double gt = dot3(gx, drr);
            if (s->x_on == 0 && q > 0) xterm[q - 1] += gt;
            if (s->x_on == 1) xterm[q] += gt;
          }
        } else if (s->coloured) {
          for (int tq = 0; tq < 4; ++tq)
            for (int ch = 0; ch < 3; ++ch) st |= emit(&cb, n4 + (i * RR + taps[tq]) * 3 + ch, g[ch] * s->w * tw[tq]);
        }
      }
    }
    for (int64_t q = 0; q < sb.n && st == VTO_OK; ++q) {
      vto_seg* s = &sb.s[q];
      int64_t i = s->cell;
      /* crossing at the exit of this cell */
      int64_t j = s->next;
      double tb = s->t_out;
      if (j < 0 || !isfinite(tb)) continue;
      double dt_b = xterm[q];
      if (tb > t0 && tb < t1) {
        dt_b += sc->sigma[i] * dtau[q];
        if (q + 1 < sb.n) dt_b -= sc->sigma[j] * dtau[q + 1];
      }
      if (dt_b == 0.0) continue;
      const double* si = sc->sites + 3 * i;
      const double* sj = sc->sites + 3 * j;
      double n[3] = {sj[0] - si[0], sj[1] - si[1], sj[2] - si[2]};
      double nd = dot3(n, drr);
      double xb[3] = {orr[0] + tb * drr[0], orr[1] + tb * drr[1], orr[2] + tb * drr[2]};
      for (int c = 0; c < 3; ++c) {
        st |= emit(&cb, 3 * i + c, dt_b * (xb[c] - si[c]) / nd);
        st |= emit(&cb, 3 * j + c, dt_b * (sj[c] - xb[c]) / nd);
      }
    }
    if (st != VTO_OK) J->status = VTO_ERR_MEM;
    if (cb.n > (1 << 20)) flush_contribs(J, &cb);
  }
  flush_contribs(J, &cb);
  free(cb.c);
  free(sb.s);
  free(dtau);
  free(xterm);
  return NULL;
}

/* ------------------------------------------------------------------ */
/* Backward: gradient of L with respect to sites, densities and texels,
 * given dL/dC per ray; accumulates into the outputs (the caller zeroes them).
 *
 * With g = dL/dC, S_k = sum_{m>k} w_m c_m + T_final bg:
 *   dL/dtau_k   = g.(T_{k+1} c_k - S_k)              (tau_k = sigma delta_k)
 *   dL/dsigma_k = dL/dtau_k * delta_k                 (matches Eq. 3)
 *   dL/dc_k     = g * w_k  -> texels by bilinear weight
 *   crossing b between walked cells k, k+1 at t_b, t_near' < t_b < t_far':
 *     dL/dt_b = sigma_k dL/dtau_k - sigma_{k+1} dL/dtau_{k+1}
 *     dt_b/ds_k     = (x_b - s_k) / (n.d)
 *     dt_b/ds_{k+1} = (s_{k+1} - x_b) / (n.d),  n = s_{k+1} - s_k.
 * When the walk stopped by transmittance inside (t_near', t_far'), the exit
 * plane of the last cell still moves delta_K; its far side gets no dtau. */
int vto_render_bwd_dist(const vto_scene* sc, int64_t n_rays, const double* o, const double* d,
                        const vto_params* p, const double* grad_rgb, const double* grad_dist, double* g_sites,
                        double* g_sigma, double* g_tex, double* g_tex_vd, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_rays < n_threads) n_threads = n_rays > 0 ? (int)n_rays : 1;
  pthread_mutex_t mu;
  pthread_mutex_init(&mu, NULL);
  pthread_t th[256];
  bwd_job jobs[256];
  int64_t chunk = (n_rays + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].sc = sc;
    jobs[t].p = p;
    jobs[t].o = o;
    jobs[t].d = d;
    jobs[t].g = grad_rgb;
    jobs[t].gdist = grad_dist;
    jobs[t].g_sites = g_sites;
    jobs[t].g_sigma = g_sigma;
    jobs[t].g_tex = g_tex;
    jobs[t].g_tex_vd = g_tex_vd;
    jobs[t].mu = &mu;
    jobs[t].lo = t * chunk;
    jobs[t].hi = (t + 1) * chunk < n_rays ? (t + 1) * chunk : n_rays;
    jobs[t].status = VTO_OK;
    if (jobs[t].lo >= jobs[t].hi) continue;
    if (n_threads == 1)
      bwd_worker(&jobs[t]);
    else
      pthread_create(&th[t], NULL, bwd_worker, &jobs[t]);
  }
  int st = VTO_OK;
  for (int t = 0; t < n_threads; ++t) {
    if (jobs[t].lo >= jobs[t].hi) continue;
    if (n_threads > 1) pthread_join(th[t], NULL);
    if (jobs[t].status != VTO_OK) st = jobs[t].status;
  }
  pthread_mutex_destroy(&mu);
  return st;
}

int vto_render_bwd(const vto_scene* sc, int64_t n_rays, const double* o, const double* d,
                   const vto_params* p, const double* grad_rgb, double* g_sites, double* g_sigma,
                   double* g_tex, double* g_tex_vd, int n_threads) {
  return vto_render_bwd_dist(sc, n_rays, o, d, p, grad_rgb, NULL, g_sites, g_sigma, g_tex, g_tex_vd, n_threads);
}

/* Per-ray distortion loss L_dist (Eq. 2). */
typedef struct {
  const vto_scene* sc;
  const vto_params* p;
  const double *o, *d;
  double* L;
  int64_t lo, hi;
  int status;
} dist_job;

static void* dist_worker(void* arg) {
  dist_job* J = (dist_job*)arg;
  seg_buf b = {0, 0, 0};
  J->status = VTO_OK;
  for (int64_t r = J->lo; r < J->hi; ++r) {
    double C[3], T, lt;
    int32_t k, fl;
    int64_t ln;
    if (walk_ray(J->sc, J->p, J->o + 3 * r, J->d + 3 * r, &b, C, &T, &k, &fl, &ln, &lt) != VTO_OK) {
      J->status = VTO_ERR_MEM;
      break;
    }
    J->L[r] = ray_distortion(&b);
  }
  free(b.s);
  return NULL;
}

int vto_distortion(const vto_scene* sc, int64_t n_rays, const double* o, const double* d, const vto_params* p,
                   double* L, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_rays < n_threads) n_threads = n_rays > 0 ? (int)n_rays : 1;
  pthread_t th[256];
  dist_job jobs[256];
  int64_t chunk = (n_rays + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].sc = sc;
    jobs[t].p = p;
    jobs[t].o = o;
    jobs[t].d = d;
    jobs[t].L = L;
    jobs[t].lo = t * chunk;
    jobs[t].hi = (t + 1) * chunk < n_rays ? (t + 1) * chunk : n_rays;
    jobs[t].status = VTO_OK;
    if (jobs[t].lo >= jobs[t].hi) continue;
    if (n_threads == 1)
      dist_worker(&jobs[t]);
    else
      pthread_create(&th[t], NULL, dist_worker, &jobs[t]);
  }
  int st = VTO_OK;
  for (int t = 0; t < n_threads; ++t) {
    if (jobs[t].lo >= jobs[t].hi) continue;
    if (n_threads > 1) pthread_join(th[t], NULL);
    if (jobs[t].status != VTO_OK) st = jobs[t].status;
  }
  return st;
}

/* ------------------------------------------------------------------ */
/* Ray generation (Sec. 6.5: only the rays change between camera models).
 * Basis: f = fwd/|fwd|, r = (f x up)/|f x up|, u = r x f. Pixel (x, y) with
 * row 0 at the top, sample point at the pixel centre. Ray order:
 * [row][col][lens sample]. Directions are unit length.                      */
typedef struct {
  int32_t kind; /* 0 pinhole, 1 equidistant fisheye, 2 rolling shutter, 3 thin lens, 4 motion blur */
  int32_t w, h;
  double eye[3], fwd[3], up[3];
  double fov_y;         /* pinhole-type vertical field of view (radians)   */
  double fisheye_fov;   /* fisheye field of view across the width (rad)     */
  double rs_velocity[3];/* rolling shutter / motion blur: centre moves velocity*time */
  double lens_radius, focus_dist;
  int32_t lens_samples; /* samples per pixel: thin lens (a square number) or motion blur */
  uint64_t seed;
} vto_camera;

static void normalize3(double v[3]) {
  double l = sqrt(dot3(v, v));
  v[0] /= l;
  v[1] /= l;
  v[2] /= l;
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* SplitMix64 (Steele, Lea & Flood, 2014) as a counter-based generator: the
 * value for counter c under key s is mix(s ^ mix(c)); 24 high bits -> [0,1). */
uint64_t vto_mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double vto_uniform(uint64_t seed, uint64_t counter) {
  uint64_t h = vto_mix64(seed ^ vto_mix64(counter));
  return (double)(h >> 40) * (1.0 / 16777216.0);
}

/* Concentric square-to-disk map (Shirley & Chiu, 1997). */
void vto_concentric(double a, double b, double out[2]) {
  if (a == 0.0 && b == 0.0) {
    out[0] = out[1] = 0.0;
    return;
  }
  double r, phi;
  if (fabs(a) > fabs(b)) {
    r = a;
    phi = (M_PI / 4.0) * (b / a);
  } else {
    r = b;
    phi = M_PI / 2.0 - (M_PI / 4.0) * (a / b);
  }
  out[0] = r * cos(phi);
  out[1] = r * sin(phi);
}

int64_t vto_camera_rays(const vto_camera* c) {
  int64_t s = (c->kind == 3 || c->kind == 4) ? c->lens_samples : 1;
  return (int64_t)c->w * c->h * s;
}

int vto_raygen(const vto_camera* c, double* o, double* d, double* time) {
  if (c->w <= 0 || c->h <= 0) return VTO_ERR_ARG;
  double f[3] = {c->fwd[0], c->fwd[1], c->fwd[2]};
  normalize3(f);
  double r[3], u[3];
  cross3(f, c->up, r);
  normalize3(r);
  cross3(r, f, u);
  int32_t S = 1, m = 1;
  if (c->kind == 3) {
    S = c->lens_samples;
    m = (int32_t)floor(sqrt((double)S) + 0.5);
    if (S <= 0 || m * m != S) return VTO_ERR_ARG;
  } else if (c->kind == 4) {
    S = c->lens_samples;
    if (S <= 0) return VTO_ERR_ARG;
  }
  double ty = tan(0.5 * c->fov_y), tx = ty * (double)c->w / (double)c->h;
  double fpx = (0.5 * c->w) / (0.5 * c->fisheye_fov);
  for (int32_t y = 0; y < c->h; ++y)
    for (int32_t x = 0; x < c->w; ++x)
      for (int32_t s = 0; s < S; ++s) {
        int64_t ray = ((int64_t)y * c->w + x) * S + s;
        double oo[3] = {c->eye[0], c->eye[1], c->eye[2]};
        double dd[3];
        double tm = 0.0;
        if (c->kind == 1) {
          double px = x + 0.5 - 0.5 * c->w, py = 0.5 * c->h - (y + 0.5);
          double rr = sqrt(px * px + py * py);
          double th = rr / fpx;
          double cp = rr > 0.0 ? px / rr : 1.0, sp = rr > 0.0 ? py / rr : 0.0;
          double ct = cos(th), st = sin(th);
          for (int k = 0; k < 3; ++k) dd[k] = ct * f[k] + st * (cp * r[k] + sp * u[k]);
        } else {
          double px = (2.0 * (x + 0.5) / c->w - 1.0) * tx;
          double py = (1.0 - 2.0 * (y + 0.5) / c->h) * ty;
          double pd[3];
          for (int k = 0; k < 3; ++k) pd[k] = f[k] + px * r[k] + py * u[k];
          if (c->kind == 2) {
            tm = (double)y / (double)c->h;
            for (int k = 0; k < 3; ++k) oo[k] += tm * c->rs_velocity[k];
            for (int k = 0; k < 3; ++k) dd[k] = pd[k];
          } else if (c->kind == 3) {
            int32_t sx = s % m, sy = s / m;
            uint64_t pix = (uint64_t)y * c->w + x;
            double j1 = vto_uniform(c->seed, ((pix * S + s) << 1) | 0u);
            double j2 = vto_uniform(c->seed, ((pix * S + s) << 1) | 1u);
            double a = 2.0 * ((sx + j1) / m) - 1.0, b = 2.0 * ((sy + j2) / m) - 1.0;
            double disk[2];
            vto_concentric(a, b, disk);
            for (int k = 0; k < 3; ++k)
              oo[k] += c->lens_radius * (disk[0] * r[k] + disk[1] * u[k]);
            /* point on the plane of focus (pd.f == 1, so depth focus_dist) */
            for (int k = 0; k < 3; ++k) dd[k] = c->eye[k] + c->focus_dist * pd[k] - oo[k];
          } else if (c->kind == 4) {
            /* motion blur (Sec. 6.5): S stratified, jittered times over the
             * exposure [0,1), camera centre moved linearly */
            uint64_t pix = (uint64_t)y * c->w + x;
            tm = (s + vto_uniform(c->seed, (pix * S + s) << 1)) / S;
            for (int k = 0; k < 3; ++k) oo[k] += tm * c->rs_velocity[k];
            for (int k = 0; k < 3; ++k) dd[k] = pd[k];
          } else {
            for (int k = 0; k < 3; ++k) dd[k] = pd[k];
          }
        }
        normalize3(dd);
        for (int k = 0; k < 3; ++k) {
          o[3 * ray + k] = oo[k];
          d[3 * ray + k] = dd[k];
        }
        if (time) time[ray] = tm;
      }
  return VTO_OK;
}
