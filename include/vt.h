/*
 * vt.h -- C ABI of libvt.so: differentiable volume rendering by ray traversal
 * of a 3D Voronoi diagram, hand-written CUDA for sm_103a (GB300).
 *
 * Method (arXiv 2608.17682, "Differentiable Voronoi Ray Tracing Beyond
 * Rasterization Speeds"):
 *   - Sec. 3.1: a ray starts in the Voronoi cell containing its origin (one
 *     nearest-site query) and steps to the next cell across the nearest
 *     forward bisector-plane crossing with the cell's Delaunay neighbours:
 *       t_j = n.((s_i+s_j)/2 - o) / (n.d),  n = s_j - s_i,  over n.d > 0.
 *   - Sec. 3.2: piecewise-constant volume rendering, alpha_k = 1 -
 *     exp(-sigma_{i_k} delta_k), C = sum_k T_k alpha_k c_k, front to back,
 *     early termination once T falls below a threshold.
 *   - Sec. 5.1: per-cell R x R RGB octahedral texture, bilinear fetch. By
 *     default this library indexes it at the ray direction d (appearance 0);
 *     appearance 1 is the paper's model of Sec. 5.1-5.2 (a surface texture at
 *     the direction of the entry point from the site plus a view-dependent
 *     texture at -d, summed as logits, then a sigmoid).
 *   - Sec. 5.3, Eq. 2: the distortion loss of each ray, computed in the same
 *     walk (optional output of vt_render_fwd, optional input of vt_render_bwd).
 *   - Sec. 5.4, Eq. 4: sigma = exp(rho) and its adjoint.
 *   - Sec. 5.5 / Eq. 5: training-step helpers (ray sampling, Smooth-L1, the
 *     texture regularisers, Adam).
 *   - Sec. 5.6: RGB texels padded to RGBA for one aligned load, half-precision
 *     appearance storage, Morton-ordered cells, warp-coherent 4x8 ray tiles,
 *     optional low-contribution cell skip, optional FP16 neighbour offsets.
 *   - Eq. 3: dL/dsigma = dL/dalpha * delta * (1 - alpha) (the backward pass
 *     computes the same quantity as dL/dtau * delta, tau = sigma*delta).
 *   - Sec. 6.5: camera effects by ray generation only (pinhole, equidistant
 *     fisheye, rolling shutter, thin lens, motion blur).
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are caller-owned CUDA device pointers (for
 *     example torch tensors' data_ptr()); "host" pointers are ordinary CPU
 *     memory. Nothing is retained past the call unless stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All work is enqueued on it; calls return after enqueueing.
 *   - Errors are returned as vt_status; nothing throws across the ABI.
 *     Asynchronous faults of earlier work surface as VT_ERR_CUDA. Errors that
 *     kernels detect (step cap, trace capacity) are recorded on the scene and
 *     read with vt_scene_get_error().
 *   - Arrays are C-contiguous, FP32 unless stated; [N,3] means N rows of 3.
 *   - A scene owns its own reordered device copies; inputs given to
 *     vt_scene_create/vt_scene_update may be freed after the call returns
 *     and the stream has been synchronised.
 */
#ifndef VT_H
#define VT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VT_OK = 0,
  VT_ERR_INVALID_ARG = 1, /* bad size, null pointer, malformed CSR, NaN site ...   */
  VT_ERR_CUDA = 2,        /* a CUDA runtime call failed (incl. earlier async faults) */
  VT_ERR_OOM = 3,         /* device allocation failed                               */
  VT_ERR_MAX_STEPS = 4,   /* a ray walked more than max_steps cells (it was stopped) */
  VT_ERR_CAPACITY = 5,    /* a trace buffer was too small (output truncated)         */
  VT_ERR_UNSUPPORTED = 6  /* feature not available in this build                     */
} vt_status;

/* Storage precision of the octahedral textures (Sec. 5.6 stores appearance in
 * half precision); compositing and accumulation are always FP32.
 * FP16 and BF16 are rounded to nearest-even from the FP32 input. */
typedef enum { VT_F32 = 0, VT_F16 = 1, VT_BF16 = 2 } vt_dtype;

typedef struct vt_scene vt_scene; /* opaque, owned by the library */

/* Scene description (Sec. 3.1 sites and Delaunay graph, Sec. 3.2 densities,
 * Sec. 5.1 textures). All pointers are DEVICE pointers, user index order. */
typedef struct {
  int64_t n_sites;             /* N >= 1                                          */
  int32_t tex_res;             /* R >= 2: textures are R x R                      */
  int32_t tex_dtype;           /* vt_dtype of the internal texture copy           */
  const float* sites;          /* [N,3] site positions p_i, finite                */
  const float* sigma;          /* [N] densities sigma_i >= 0, finite              */
  const float* tex;            /* [N,R,R,3] RGB, row y then column x (see below)  */
  const int64_t* adj_offsets;  /* [N+1] CSR row offsets, adj_offsets[0] == 0     */
  const int32_t* adj_indices;  /* [E] neighbour ids; symmetric, no self loops,
                                  no duplicates within a row, E < 2^31; may be
                                  NULL when E == 0                                 */
  int32_t flags;               /* VT_SCENE_KEEP_ORDER: store cells in user order
                                  instead of Morton order (for ablations);
                                  VT_SCENE_HALF_OFFSETS: see below                */
  const float* tex_vd;         /* optional [N,R,R,3] view-dependent texture T_vd
                                  (Sec. 5.2), logits; required for appearance 1   */
} vt_scene_desc;

#define VT_SCENE_KEEP_ORDER 1
/* VT_SCENE_HALF_OFFSETS: also store each neighbour offset s_j - s_i as three
 * FP16 values (8-byte records, Sec. 5.6: the inference kernel's
 * half-precision neighbour vectors) and let vt_render_fwd / vt_trace_cells
 * search exits with them. The planes then pass through s_i + n_h/2 with
 * normal n_h = fp16(s_j - s_i), not exactly through the bisector, so cell
 * sequences can differ from the exact walk near Voronoi edges. Forward
 * only: vt_render_bwd, vt_render_bwd_static and the distortion output return
 * VT_ERR_UNSUPPORTED on such a scene. Offsets must be below 65504 in
 * magnitude (VT_ERR_INVALID_ARG otherwise). */
#define VT_SCENE_HALF_OFFSETS 2

/* Render parameters. Rays are r(t) = o + t d for t in [t_near, t_far],
 * optionally clipped to the box [clip_lo, clip_hi]. */
typedef struct {
  float t_near, t_far;     /* ray extent (in units of |d|); default 0, 20              */
  int32_t use_clip_box;    /* nonzero: also clip to the axis-aligned box               */
  float clip_lo[3], clip_hi[3];
  float T_eps;             /* early termination once T < T_eps (after compositing
                              that cell); 1e-4                                         */
  float skip_weight;       /* Sec. 5.6: if T*alpha < skip_weight the cell's colour is
                              not fetched (T still updated). 0 = exact                 */
  float bg[3];             /* background colour added as T_final * bg                  */
  int32_t img_w, img_h;    /* ray layout [n_images][img_h][img_w] -> 4x8 warp tiles;
                              0 = plain 1-D order                                      */
  int32_t n_images;        /* number of images when img_w > 0                          */
  int32_t max_steps;       /* cells a ray may visit (<= 0: min(4N, 2^20)); exceeding it
                              stops the ray and records VT_ERR_MAX_STEPS               */
  const int32_t* image_sizes; /* optional HOST [n_images][2] = (w, h) of each image when
                              the images differ in size (rays laid out image after image,
                              row-major); then img_w/img_h are ignored and n_images <= 64.
                              NULL: img_w/img_h/n_images as above                      */
  int32_t appearance;      /* 0: colour = tex at the ray direction (default).
                              1: the paper's model, Sec. 5.1-5.2:
                              c = sigmoid(T_vi(oct((x - p_i)/|x - p_i|)) + T_vd(oct(-d))),
                              T_vi = tex, T_vd = tex_vd (logits), x = where the ray
                              enters the cell (the cell holding the origin: where it
                              leaves it, or its segment end if it never leaves)      */
  void* walk_events[2];    /* optional cudaEvent_t pair: recorded on the call's stream
                              right before and right after the walk kernel of
                              vt_render_fwd / vt_render_bwd / vt_trace_cells, so a
                              caller can time that kernel alone. NULL: not recorded */
} vt_render_params;

/* Fill `p` with the defaults listed above. */
void vt_render_params_default(vt_render_params* p);

/* Build a scene (Sec. 5.6 one-time preprocessing, untimed in the paper):
 * validates the inputs (finite sites, sigma >= 0, CSR in range, symmetric,
 * no self loops, R >= 2), sorts cells by 63-bit Morton code over the sites'
 * bounding box (ties by user id; skipped with VT_SCENE_KEEP_ORDER, Sec. 6.3
 * ablates this ordering), permutes sites / densities / textures,
 * remaps the adjacency and stores each neighbour's position inline with its
 * CSR entry, pads texels RGB -> RGBA in the requested storage dtype.
 * On success *out receives a new scene; on error *out is NULL. Synchronises
 * `stream` before returning (validation result is read on the host). */
vt_status vt_scene_create(const vt_scene_desc* desc, void* stream, vt_scene** out);

/* Replace sites, densities and textures (device pointers, user order, same
 * N, R and adjacency as at creation; any may be NULL to keep the old one;
 * tex_vd only if the scene was created with one). The Morton order of
 * creation is kept. Validates like vt_scene_create. */
vt_status vt_scene_update(vt_scene* s, const float* sites, const float* sigma, const float* tex,
                          const float* tex_vd, void* stream);

/* Free a scene. NULL is ignored. Synchronises the device first. */
void vt_scene_destroy(vt_scene* s);

/* Scene facts: n_sites, tex_res, tex_dtype, number of CSR entries. */
vt_status vt_scene_info(const vt_scene* s, int64_t* n_sites, int32_t* tex_res, int32_t* tex_dtype,
                        int64_t* n_edges);

/* Synchronise `stream`, return the first kernel-detected error recorded on the
 * scene since the last call (VT_ERR_MAX_STEPS, VT_ERR_CAPACITY) or VT_OK,
 * and clear it. Also returns VT_ERR_CUDA for an asynchronous CUDA fault.
 * If n_fp64 is not NULL it receives the number of FP64 plane rechecks done
 * since the last call: planes of a walked cell with |n.d| <= 1e-6 |d| max|n|,
 * the maximum over that cell's neighbours (a superset of the planes with
 * |n.d| <= 1e-6 |n| |d|). */
vt_status vt_scene_get_error(vt_scene* s, void* stream, int64_t* n_fp64);

/* ---------------------------------------------------------------------- */
/* Cameras (Sec. 6.5 / application appendix: only ray generation changes).
 * Basis: f = fwd/|fwd|, r = (f x up)/|f x up|, u = r x f. Pixel (x,y), row 0
 * at the top, rays through pixel centres. Rays are written in the order
 * [camera][row][col][lens sample]; directions are unit length.
 *   PINHOLE:          d ~ f + px r + py u, px = (2(x+.5)/w - 1) tan(fov_y/2) w/h,
 *                     py = (1 - 2(y+.5)/h) tan(fov_y/2).
 *   FISHEYE_EQUIDIST: angle to f = rho / F, rho = pixel-centre distance from the
 *                     image centre in pixels, F = (w/2)/(fisheye_fov/2);
 *                     azimuth = atan2(py, px) in the (r, u) plane.
 *   ROLLING_SHUTTER:  pinhole directions; row y has time y/h and origin
 *                     eye + (y/h) * rs_velocity (linear motion per frame).
 *   MOTION_BLUR:      pinhole directions; lens_samples = S time samples per
 *                     pixel, sample s at time (s + j)/S with j a SplitMix64
 *                     counter hash of (seed, pixel, s) as below, origin
 *                     eye + time * rs_velocity (linear motion over the exposure).
 *   THIN_LENS:        lens_samples = m*m stratified samples per pixel; sample s
 *                     = (sy*m + sx) is jittered in its stratum by a SplitMix64
 *                     counter hash of (seed, pixel, s), mapped to the disk by
 *                     Shirley-Chiu's concentric map, origin eye + lens_radius
 *                     (lx r + ly u); the ray aims at the pinhole ray's point at
 *                     depth focus_dist along f.
 * `time` is 0 except for rolling shutter and motion blur. Average the samples
 * of a pixel with vt_average_samples. */
typedef enum {
  VT_CAM_PINHOLE = 0,
  VT_CAM_FISHEYE_EQUIDIST = 1,
  VT_CAM_ROLLING_SHUTTER = 2,
  VT_CAM_THIN_LENS = 3,
  VT_CAM_MOTION_BLUR = 4
} vt_cam_kind;

typedef struct {
  int32_t kind; /* vt_cam_kind */
  int32_t w, h;
  float eye[3], fwd[3], up[3];
  float fov_y;          /* radians                                   */
  float fisheye_fov;    /* radians across the width (pi = 180 deg)   */
  float rs_velocity[3]; /* world units per frame (rolling shutter, motion blur) */
  float lens_radius, focus_dist;
  int32_t lens_samples; /* samples per pixel: thin lens (a square number) or
                           motion blur (>= 1)                        */
  uint64_t seed;
} vt_camera;

/* Number of rays camera `c` produces (w*h, times lens_samples for thin lens
 * and motion blur). */
int64_t vt_camera_n_rays(const vt_camera* c);

/* Generate rays for n_cams cameras (HOST array of descriptions) into DEVICE
 * buffers o [R,3], d [R,3], time [R] (time may be NULL), R = sum of
 * vt_camera_n_rays. */
vt_status vt_generate_rays(const vt_camera* cams, int32_t n_cams, float* o, float* d, float* time,
                           void* stream);

/* ---------------------------------------------------------------------- */
/* Forward render (Sec. 3.1 walk + Sec. 3.2 compositing + Sec. 5.1 colour).
 *   o, d   : DEVICE [n_rays,3] ray origins and directions (|d| > 0; t is in
 *            units of |d|; the colour uses d's direction).
 *   time   : DEVICE [n_rays] or NULL; accepted and ignored (static scene).
 *   rgb_out: DEVICE [n_rays,3] C = sum_k T_k alpha_k c_k + T_final bg
 *            (accumulated in float-float, rounded to FP32).
 *   T_out  : DEVICE [n_rays] final transmittance (NULL allowed).
 *   steps_out: DEVICE [n_rays] int32 cells visited by the walk (NULL allowed).
 *   rgb_residual: DEVICE [n_rays,3] or NULL: the rounding residual C - rgb_out
 *            of the float-float colour. Passing it to vt_render_bwd lets the
 *            backward form the suffix sums C - sum_{m<=k} w_m c_m without the
 *            FP32 rounding of C (which limits deep-ray gradients to ~1e-3).
 *   dist_out: DEVICE [n_rays,3] or NULL: the distortion loss of Mip-NeRF 360
 *            (Sec. 5.3, Eq. 2) of each ray, computed in the same pass:
 *              dist_out[3r]   = L_dist(r) = sum_{k,l} w_k w_l |sbar_k - sbar_l|
 *                                           + 1/3 sum_k w_k^2 ds_k,
 *            w_k = T_k alpha_k over the composited intervals [a_k, b_k],
 *            s(t) = 1 - 1/(1+t) of the ray parameter t, sbar_k = (s(a_k) +
 *            s(b_k))/2, ds_k = s(b_k) - s(a_k);
 *              dist_out[3r+1] = sum_k w_k, dist_out[3r+2] = sum_k w_k (sbar_k -
 *            sbar_first): totals that vt_render_bwd reads back. Requires
 *            t_near >= 0 (VT_ERR_INVALID_ARG otherwise).
 * The start cell of each ray is found by an exact nearest-site search for one
 * anchor origin per image (per 4096 rays in 1-D layout) followed by a greedy
 * walk over the Delaunay graph to the ray's own origin. */
vt_status vt_render_fwd(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                        const vt_render_params* p, float* rgb_out, float* T_out, int32_t* steps_out,
                        float* rgb_residual, float* dist_out, void* stream);

/* Backward render: re-traverses every ray with decisions identical to
 * vt_render_fwd (no per-ray cell lists are stored) and accumulates
 *   grad_sites [N,3] (through the bisector-plane crossings),
 *   grad_sigma [N]   (dL/dtau * delta, Eq. 3),
 *   grad_tex   [N,R,R,3] (bilinear weights * T alpha * dL/dC),
 * all DEVICE FP32 in USER index order, OVERWRITTEN (the call zero-fills them).
 * rgb_out is the forward's output for the same rays and parameters and
 * rgb_residual (NULL allowed) its residual output; grad_rgb is dL/dC [n_rays,3].
 * grad_dist (DEVICE [n_rays] or NULL) is dL/dL_dist per ray; when given, the
 * gradients include the distortion loss and dist_out must be the forward's
 * dist_out for the same rays (VT_ERR_INVALID_ARG if NULL). Any of the gradient
 * pointers may be NULL to skip that output; grad_tex_vd is for appearance 1.
 * Library-owned scratch (one float4 per cell and per texel, one byte per
 * cell) is allocated on first use and kept with the scene; the call leaves the
 * texel scratch zeroed for the next one (only the cells this call touched are
 * rewritten). Backward calls on one scene share that scratch: order them on
 * one stream. */
vt_status vt_render_bwd(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                        const vt_render_params* p, const float* rgb_out, const float* rgb_residual,
                        const float* dist_out, const float* grad_rgb, const float* grad_dist, float* grad_sites,
                        float* grad_sigma, float* grad_tex, float* grad_tex_vd, void* stream);

/* Backward render that leaves the gradients in the scene's own cell order
 * (the Morton order of vt_scene_create; Sec. 5.6 keeps cells in that order)
 * instead of permuting them to user order: same walk, arguments and numerics
 * as vt_render_bwd, minus the permute, which writes the dense user-order
 * arrays (about 1 ms and 4 GB of traffic for 3M cells with 8x8 textures). On
 * success it sets *grad_cell, *grad_tex and (if not NULL) *grad_tex_vd to
 * DEVICE arrays owned by the scene:
 *   grad_cell [N][4]      {dL/ds_x, dL/ds_y, dL/ds_z, dL/dsigma} of cell k,
 *   grad_tex  [N][R][R][4] RGBA texel gradients (A is 0), grad_tex_vd the same
 *                         for the view-dependent texture (appearance 1; NULL
 *                         when the scene has none),
 * where cell k is the user's site vt_scene_permutation()[k]. They hold this
 * call's gradients until the next backward call on the scene (of either
 * kind) or its destruction; the next call re-zeroes only the texel blocks
 * this one wrote. Read them on `stream` (or after synchronising it).
 * grad_cell and grad_tex must not be NULL (VT_ERR_INVALID_ARG); the other
 * errors are those of vt_render_bwd. On any error the three pointers are set
 * to NULL (grad_tex_vd only if it was given). */
vt_status vt_render_bwd_scene_order(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                                    const vt_render_params* p, const float* rgb_out, const float* rgb_residual,
                                    const float* dist_out, const float* grad_rgb, const float* grad_dist,
                                    const float** grad_cell, const float** grad_tex, const float** grad_tex_vd,
                                    void* stream);

/* The scene's cell order: perm [N] DEVICE int32, perm[k] = user id of cell k
 * (copied on `stream`). */
vt_status vt_scene_permutation(const vt_scene* s, int32_t* perm, void* stream);

/* Allocation-free backward (no counterpart in the paper). Same arguments,
 * outputs and numerics as vt_render_bwd without a colour residual or distortion
 * loss, appearance 0 only (appearance 1 returns VT_ERR_UNSUPPORTED), for callers that may not allocate
 * device memory at the time of the call: vt_render_bwd allocates its gradient
 * scratch with cudaMalloc on its first call for a scene, and cudaMalloc can
 * synchronise the device and bypasses an application's own memory pool or
 * budget (for example a framework's caching allocator). This entry point
 * calls no cudaMalloc, cudaFree or other allocating routine; its scratch is a
 * fixed device array of VT_STATIC_SCRATCH_BYTES (32 MiB) compiled into
 * libvt.so, which every GPU that loads the library holds until the process
 * exits. The scene needs n_sites * (1 + R*R) * 16 bytes of it (for R = 8,
 * up to 32,263 sites); a larger scene returns VT_ERR_CAPACITY and does nothing.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. All calls share the one array and clear the part they
 * use at the start: calls whose work overlaps on the GPU (other streams, other
 * threads, or vt_render_bwd_static on two scenes concurrently) race and give
 * wrong gradients -- order them on one stream. */
#define VT_STATIC_SCRATCH_BYTES (32ll * 1024 * 1024)
vt_status vt_render_bwd_static(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                               const vt_render_params* p, const float* rgb_out, const float* grad_rgb,
                               float* grad_sites, float* grad_sigma, float* grad_tex, void* stream);

/* Debug / parity: visited cells of each ray (walk order, USER ids) and the
 * exit parameter of each visited cell (+inf if unbounded), up to max_cells
 * per ray: cells [n_rays,max_cells] int32, t_exit [n_rays,max_cells] (NULL
 * allowed), n_cells [n_rays] = true count. Overflow records VT_ERR_CAPACITY. */
vt_status vt_trace_cells(vt_scene* s, int64_t n_rays, const float* o, const float* d,
                         const vt_render_params* p, int32_t max_cells, int32_t* cells, float* t_exit,
                         int32_t* n_cells, void* stream);

/* L2 photometric loss of the benchmark workloads: L = mean((C - Y)^2) over
 * n*3 values; grad = dL/dC = 2 (C - Y) / (3 n). DEVICE pointers; loss_out is
 * one float (overwritten). */
vt_status vt_l2_loss(int64_t n, const float* rgb, const float* target, float* grad_out, float* loss_out,
                     void* stream);

/* Pixel = mean of spp consecutive rays (depth of field, Sec. 6.5):
 * out [n_pixels,3] from rays [n_pixels*spp,3]; the backward spreads
 * grad_px / spp to every sample. DEVICE pointers. */
vt_status vt_average_samples(int64_t n_pixels, int32_t spp, const float* rgb_rays, float* rgb_px,
                             void* stream);
vt_status vt_average_samples_bwd(int64_t n_pixels, int32_t spp, const float* grad_px, float* grad_rays,
                                 void* stream);

/* Scale-invariant density parameterisation (Sec. 5.4): sigma = exp(rho), and
 * its adjoint grad_rho = grad_sigma * sigma (Eq. 4). DEVICE [n] FP32 arrays;
 * the output may alias the input. */
vt_status vt_sigma_from_rho(int64_t n, const float* rho, float* sigma, void* stream);
vt_status vt_sigma_from_rho_bwd(int64_t n, const float* sigma, const float* grad_sigma, float* grad_rho,
                                void* stream);

/* ---- training step helpers (Sec. 5.5, Eq. 5, and the appendix's training
 * settings). All pointers DEVICE, FP32, caller-owned. */

/* Stratified ray sampling: from a pool of n_pool rays (o_pool, d_pool
 * [n_pool,3], optional colours y_pool [n_pool,3]) draw n <= n_pool rays, one
 * uniformly inside each stratum [k n_pool/n, (k+1) n_pool/n) (SplitMix64
 * counter hash of (seed, k)), and gather them into o, d, y [n,3] (y NULL to
 * skip) and their pool indices idx_out [n] (NULL allowed). The indices are
 * increasing, so rays of one camera stay together; every pool ray is drawn
 * with probability n/n_pool. */
vt_status vt_sample_rays(int64_t n_pool, const float* o_pool, const float* d_pool, const float* y_pool, int64_t n,
                         uint64_t seed, float* o, float* d, float* y, int64_t* idx_out, void* stream);

/* Smooth-L1 photometric loss (L_rgb of Eq. 5): mean over the 3n channels of
 * 0.5 r^2/beta (|r| < beta) else |r| - 0.5 beta, r = rgb - target; grad_out
 * [n,3] (NULL allowed) receives dL/drgb, loss_out one float (overwritten). */
vt_status vt_smooth_l1_loss(int64_t n, const float* rgb, const float* target, float beta, float* grad_out,
                            float* loss_out, void* stream);

/* Texture regularisers of Eq. 5 on [n_cells, R, R, 3] maps:
 *   L_vd   = 1/(N R^2) sum_i |T_i^vd|^2,
 *   L_mean = 1/(N R^2) sum_{i,u} |T_{i,u}^vi - 1/R^2 sum_v T_{i,v}^vi|^2;
 * loss_out = lambda_vd L_vd + lambda_mean L_mean (overwritten); the weighted
 * gradients are ADDED to grad_tex / grad_tex_vd (NULL to skip). */
vt_status vt_texture_regularizers(int64_t n_cells, int32_t tex_res, const float* tex, const float* tex_vd,
                                  float lambda_vd, float lambda_mean, float* grad_tex, float* grad_tex_vd,
                                  float* loss_out, void* stream);

/* One Adam step (Kingma & Ba) with bias correction at step >= 1:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   param -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * param, m, v updated in place. */
vt_status vt_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                       float beta2, float eps, int64_t step, void* stream);

/* ---- measurement aids (no counterpart in the paper) */

/* Number of kernels this library has launched in the process so far (all
 * devices and threads). A caller takes the difference around a region to
 * count the library's launches in it. */
uint64_t vt_kernel_launches(void);

/* Bandwidth probe: read the DEVICE buffer `buf` (16-byte aligned, `bytes` a
 * multiple of 16) `reps` times in one kernel, through the L2 only (the loads
 * bypass L1). With a buffer that fits in L2 and many repetitions, bytes*reps
 * over the kernel's time is the L2 read bandwidth; with a buffer larger than
 * L2 it is the HBM read bandwidth. `sink` is one DEVICE float that is written
 * only on a value the data never produces. VT_ERR_INVALID_ARG on a bad
 * pointer, size or count. */
vt_status vt_stream_read(const void* buf, int64_t bytes, int32_t reps, float* sink, void* stream);

/* Adam steps that take the gradients of vt_render_bwd_scene_order directly
 * (scene cell order, float4 records) and update user-order parameters, so a
 * training step needs no user-order gradient arrays. perm [N] is
 * vt_scene_permutation (scene cell k = user cell perm[k]; an entry outside
 * [0, N) is skipped); Adam as in vt_adam_step (bias correction at `step`);
 * all pointers DEVICE, FP32.
 *
 * Texture map: grad_tex_scene [N][R][R][4] (RGBA, A ignored); tex, m, v
 * [N][R][R][3] user order, updated in place. The map's regulariser of Eq. 5
 * is fused in: regularizer 0 adds lambda * L_mean (for T_vi), 1 adds lambda *
 * L_vd (for T_vd), both normalised by N R^2 as in vt_texture_regularizers;
 * its gradient is taken at the parameters before the update and its loss is
 * ADDED to *loss_out (one float; NULL allowed when lambda == 0). With lr == 0
 * the parameters and moments are left as they are and only the loss is
 * added. VT_ERR_INVALID_ARG on a bad size, regulariser id, Adam constant or a
 * missing pointer. */
vt_status vt_adam_step_tex_scene_order(int64_t n_cells, int32_t tex_res, const int32_t* perm,
                                      const float* grad_tex_scene, float* tex, float* m, float* v, int32_t regularizer,
                                      float lambda, float lr, float beta1, float beta2, float eps, int64_t step,
                                      float* loss_out, void* stream);

/* Sites and log-densities: grad_cell_scene [N][4] = {dL/ds, dL/dsigma} in
 * scene order; sites [N,3], rho [N] (sigma = exp(rho), Sec. 5.4) and their
 * moments in user order; sigma [N] user order, the densities the gradients
 * were taken at. dL/drho = dL/dsigma * sigma (Eq. 4). A rate of 0 skips that
 * parameter (its pointers may then be NULL). */
vt_status vt_adam_step_cells_scene_order(int64_t n_cells, const int32_t* perm, const float* grad_cell_scene,
                                        float* sites, float* rho, const float* sigma, float* m_sites, float* v_sites,
                                        float* m_rho, float* v_rho, float lr_sites, float lr_rho, float beta1,
                                        float beta2, float eps, int64_t step, void* stream);

/* Human-readable status name (static string). */
const char* vt_status_str(vt_status s);

#ifdef __cplusplus
}
#endif
#endif /* VT_H */
