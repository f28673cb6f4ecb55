// vt_render.cu -- start-cell search, Voronoi walk, compositing, adjoint.
//
// One thread per ray; a warp covers a 4 x 8 tile of an image (the warp-coherent
// tiling of Sec. 5.6, 8 pixels wide, 4 tall) and a 128-thread block a
// 16 x 8-pixel patch of such tiles, so neighbouring threads walk similar
// cells and share cache lines. Forward, backward and trace are one templated
// kernel whose walk is the same inline code, so their decisions are identical.
//
// Exit test (Sec. 3.1): from cell i, entered at ray parameter t, the exit is
// the nearest forward crossing over the Delaunay neighbours j of
//   dt_j = n.(r + n/2) / (n.d),   n = s_j - s_i,  r = s_i - (o + t d),
// which is t_j - t for t_j = n.((s_i+s_j)/2 - o)/(n.d). r is formed with
// compensated (float-float) arithmetic, so the comparison error scales with
// the cell size instead of the distance from the origin. Candidates are
// compared by cross-multiplication (no division in the loop). A plane with
// |n.d| <= 1e-6 |n||d| (grazing; FP32 cannot fix the sign of n.d) is
// re-evaluated in FP64 from the FP32 site positions, in a second pass over the
// cell that runs only when the loop met such a plane.
//
// Compositing (Sec. 3.2): alpha = 1 - exp(-sigma delta), w = T alpha,
// C += w c, T *= (1 - alpha); stop once T < T_eps after compositing a cell.
// Colour (Sec. 5.1): bilinear fetch of the cell's octahedral texture at the
// ray direction; the four taps are fixed per ray. Appearance 1 is the paper's
// model (Sec. 5.1-5.2): a surface texture at the entry point's direction from
// the site plus a view-dependent texture at -d, summed as logits, sigmoid.
// The distortion loss (Eq. 2) can ride in the same walk (template DIST).
// Backward gradients go to Morton-ordered scratch through warp-aggregated
// vector atomics and are permuted to the caller's order by k_grad_out.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "vt_internal.cuh"

namespace {

enum Mode { FWD = 0, BWD = 1, TRACE = 2 };

// minimum resident warps per SM requested for the walk kernels (more warps
// hide the walk's dependent loads; the appearance-1 and distortion backwards
// keep more registers for their adjoint state); the launch bounds convert
// them to blocks of VT_WPB warps. On 3M sites / 4 views with 4-warp blocks:
// forward 36 warps (56 registers) 3.01 ms, 32 (64) 3.07 ms, 40 (48) spills
// twice as much; plain backward 24 warps (80 registers) 4.88 ms, 28 (72)
// 4.88 ms, 20 (96, no spills) 5.08 ms; with 8-warp blocks the plain backward
// ran 5.11 ms at 24 warps and 5.31 ms at 32.
#ifndef VT_FWD_WARPS
#define VT_FWD_WARPS 36
#endif
#ifndef VT_FWD_WARPS_EXT
#define VT_FWD_WARPS_EXT 32  // forward with the paper's appearance model or the distortion loss
#endif
#ifndef VT_BWD_WARPS
#define VT_BWD_WARPS 24
#endif
#ifndef VT_BWD_WARPS_EXT
#define VT_BWD_WARPS_EXT 24  // backward with the paper's appearance model or the distortion loss
#endif
// 1: issue a cell's texel loads before its exit search (latency overlapped,
// more live registers); 0: after it
#ifndef VT_TEX_EARLY
#define VT_TEX_EARLY 0
#endif
// warp aggregation of gradient atomics by pairwise key-matched shuffles:
// 0 none, 1 site/sigma gradients, 2 also texel gradients. The lanes of a 4x8
// tile mostly sit in the same cell at the same step, so 2 removes most of the
// atomics; on 3M sites / 4 views the backward drops from 13.3 to 8.8 ms
// (1: 12.8 ms).
#ifndef VT_AGG
#define VT_AGG 2
#endif
// 1: the backward re-reads the previous cell's position from its record
// instead of keeping it in registers across the neighbour loop
#ifndef VT_BWD_RELOAD_PREV
#define VT_BWD_RELOAD_PREV 1
#endif
// tiles per row of the patch a walk block renders (with 8-warp blocks, 8: a
// 64x4 pixel strip; 2: a 16x16 square; on 3M sites / 4 views: 8 327.6, 4
// 337.5, 1 341.0, 2 346.0 Mrays/s fwd+bwd -- the squarest patch shares the
// most cells)
#ifndef VT_ST_W
#define VT_ST_W 2
#endif
// warps per walk block (each warp a 4x8 tile; the block a patch of tiles).
// On 3M sites / 4 views, walk kernels fwd / bwd in ms: 8 warps (16x16-pixel
// patch) 3.16 / 5.11; 4 (16x8) 3.06 / 4.88; 2 (8x8) 3.08 / 4.91; 2 (16x4)
// 3.14 / 5.01; 1 3.17 / 6.41: a smaller block leaves fewer lanes idle while
// its slowest tile finishes.
#ifndef VT_WPB
#define VT_WPB 4
#endif
constexpr int kWpb = VT_WPB;
constexpr int kPatchH = kWpb / VT_ST_W;  // tile rows of a patch
// unroll factor of the neighbour loop
#ifndef VT_NBR_UNROLL
#define VT_NBR_UNROLL 8
#endif
constexpr int kNbrUnroll = VT_NBR_UNROLL;
// 1: stage the neighbour records of a cell that all 32 lanes of a warp share
// in shared memory (kStageCap records at most per warp)
#ifndef VT_STAGE
#define VT_STAGE 0
#endif
constexpr int kStageCap = 64;

struct Scene {
  const vt_cell* __restrict__ cell;
  const float4* __restrict__ nbr;
  const uint2* __restrict__ nbr_h;  // FP16 offsets (VT_SCENE_HALF_OFFSETS) or null
  const void* __restrict__ tex;
  const void* __restrict__ tex_vd;
  int64_t n;
  int32_t R, RR;
  unsigned long long* err;
};

// one image of a launch whose images differ in size
struct ImgEnt {
  int64_t first_ray, first_tile;
  int w, h, tiles_x, st_x;  // st_x: tile patches per row
};

struct RP {  // render parameters, device copy
  float t_near, t_far;
  int clip;
  float3 lo, hi;
  float T_eps, skip;
  float3 bg;
  int img_w, img_h, n_images, tiles_x, tiles_per_img, st_x;
  int max_steps;
  int64_t n_rays;
  int64_t anchor_stride;
  int appearance;
  // ray layout: 0 plain 1-D, 1 n_images equal images, 2 table of images
  int layout, n_tab;
  int64_t total_tiles;
  ImgEnt img[VT_MAX_ANCHORS];
};

// first ray of anchor a (its origin is the anchor point)
__device__ __forceinline__ int64_t anchor_ray(const RP& P, int a) {
  return P.layout == 2 ? P.img[a].first_ray : (int64_t)a * P.anchor_stride;
}

struct Grad {
  float4* g_cell;
  float4* g_tex;
  float4* g_tex_vd;
  const float* rgb;
  const float* rgb_lo;  // optional residual of the forward colour
  const float* grad;
  // distortion loss (Eq. 2): per-ray {L_dist, sum w, sum w sbar'} written by
  // the forward, read by the backward; dL/dL_dist per ray (backward)
  float* dist;
  const float* gdist;
  uint8_t* touched;  // per cell: texel scratch written (null: not tracked)
};

struct Trace {
  int32_t* cells;
  float* t_exit;
  int32_t* n_cells;
  int max_cells;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float dist2(float3 q, float x, float y, float z) {
  float dx = __fsub_rn(q.x, x), dy = __fsub_rn(q.y, y), dz = __fsub_rn(q.z, z);
  return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s - (o + (th + tl) d), compensated per component
__device__ __forceinline__ float rel1(float s, float o, float d, float th, float tl) {
  float ah, al;
  two_sum(s, -o, ah, al);
  float ph = __fmul_rn(th, d);
  float pl = __fmaf_rn(th, d, -ph);
  pl = __fmaf_rn(tl, d, pl);
  return __fadd_rn(__fsub_rn(ah, ph), __fsub_rn(al, pl));
}
__device__ __forceinline__ float3 rel_pos(float3 s, float3 o, float3 d, float th, float tl) {
  return make_float3(rel1(s.x, o.x, d.x, th, tl), rel1(s.y, o.y, d.y, th, tl), rel1(s.z, o.z, d.z, th, tl));
}

// (th, tl) + x  -> renormalised float-float
__device__ __forceinline__ void ff_add(float& th, float& tl, float x) {
  float s, e;
  two_sum(th, x, s, e);
  e = __fadd_rn(e, tl);
  th = __fadd_rn(s, e);
  tl = __fsub_rn(e, __fsub_rn(th, s));
}
// float-float strictly greater / greater-or-equal than a float
__device__ __forceinline__ bool ff_gt(float th, float tl, float x) { return th > x || (th == x && tl > 0.f); }
__device__ __forceinline__ bool ff_ge(float th, float tl, float x) { return th > x || (th == x && tl >= 0.f); }

// Raw texel (RGBA): FP32 as float4, FP16/BF16 as 4 x 16 bits in a uint2 (kept
// packed until use to save registers).
template <int DT>
struct TexRaw {
  uint2 v;
};
template <>
struct TexRaw<VT_F32> {
  float4 v;
};

template <int DT>
__device__ __forceinline__ TexRaw<DT> load_texel(const void* tex, int64_t e) {
  TexRaw<DT> t;
  if constexpr (DT == VT_F32)
    t.v = __ldg(reinterpret_cast<const float4*>(tex) + e);
  else
    t.v = __ldg(reinterpret_cast<const uint2*>(tex) + e);
  return t;
}

template <int DT>
__device__ __forceinline__ float3 texel_rgb(const TexRaw<DT>& t) {
  if constexpr (DT == VT_F32) {
    return make_float3(t.v.x, t.v.y, t.v.z);
  } else if constexpr (DT == VT_F16) {
    uint2 u = t.v;
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    return make_float3(a.x, a.y, __half2float(*reinterpret_cast<const __half*>(&u.y)));
  } else {
    return make_float3(__uint_as_float(t.v.x << 16), __uint_as_float(t.v.x & 0xffff0000u),
                       __uint_as_float(t.v.y << 16));
  }
}

// Octahedral map (Sec. 5.1) + bilinear taps, texel index y*R + x, clamp to
// edge. Returned compactly: base texel, x / y steps (0 at the clamped edge)
// and the fractional offsets; taps are base, base+sx, base+sy, base+sx+sy.
struct Taps {
  int base, sx, sy;
  float fx, fy;
  float gxs, gys;  // d(texel x, y)/d(u, v): R/2 inside, 0 where clamped
};

// FAST: q = d * approx(1/l1) (per-step surface directions of appearance 1);
// else correctly rounded quotients (once per ray)
template <bool FAST = false>
__device__ __forceinline__ Taps taps_for(float3 d, int R) {
  float l1 = __fadd_rn(__fadd_rn(fabsf(d.x), fabsf(d.y)), fabsf(d.z));
  float qx, qy;
  if (FAST) {
    const float il = __fdividef(1.f, l1);
    qx = d.x * il;
    qy = d.y * il;
  } else {
    qx = __fdiv_rn(d.x, l1);
    qy = __fdiv_rn(d.y, l1);
  }
  float u, v;
  if (d.z >= 0.f) {
    u = qx;
    v = qy;
  } else {
    u = copysignf(__fsub_rn(1.f, fabsf(qy)), qx >= 0.f ? 1.f : -1.f);
    v = copysignf(__fsub_rn(1.f, fabsf(qx)), qy >= 0.f ? 1.f : -1.f);
  }
  float x = __fsub_rn(__fmul_rn(__fmul_rn(__fadd_rn(u, 1.f), 0.5f), (float)R), 0.5f);
  float y = __fsub_rn(__fmul_rn(__fmul_rn(__fadd_rn(v, 1.f), 0.5f), (float)R), 0.5f);
  Taps t;
  t.gxs = (x >= 0.f && x <= (float)(R - 1)) ? 0.5f * (float)R : 0.f;
  t.gys = (y >= 0.f && y <= (float)(R - 1)) ? 0.5f * (float)R : 0.f;
  x = fminf(fmaxf(x, 0.f), (float)(R - 1));
  y = fminf(fmaxf(y, 0.f), (float)(R - 1));
  int x0 = min((int)floorf(x), R - 1), y0 = min((int)floorf(y), R - 1);
  t.base = y0 * R + x0;
  t.sx = x0 + 1 < R ? 1 : 0;
  t.sy = y0 + 1 < R ? R : 0;
  t.fx = __fsub_rn(x, (float)x0);
  t.fy = __fsub_rn(y, (float)y0);
  return t;
}

__device__ __forceinline__ void tap_weights(const Taps& t, float w[4]) {
  const float gx = __fsub_rn(1.f, t.fx), gy = __fsub_rn(1.f, t.fy);
  w[0] = __fmul_rn(gx, gy);
  w[1] = __fmul_rn(t.fx, gy);
  w[2] = __fmul_rn(gx, t.fy);
  w[3] = __fmul_rn(t.fx, t.fy);
}

// (gu, gv) . d(u, v)/d(dir) for the octahedral map (Sec. 5.1) of `dir`
__device__ __forceinline__ float3 oct_vjp(float3 dir, float gu, float gv) {
  const float l1 = fabsf(dir.x) + fabsf(dir.y) + fabsf(dir.z);
  const float il = __fdividef(1.f, l1);
  const float qx = dir.x * il, qy = dir.y * il;
  const float sx = dir.x >= 0.f ? 1.f : -1.f, sy = dir.y >= 0.f ? 1.f : -1.f, sz = dir.z >= 0.f ? 1.f : -1.f;
  // dq_a/ddir_j = (delta_aj - q_a sgn(dir_j)) / l1
  float ax, ay;  // coefficients on dq_x and dq_y
  if (dir.z >= 0.f) {
    ax = gu;
    ay = gv;
  } else {
    ax = -sy * sx * gv;
    ay = -sx * sy * gu;
  }
  const float dot = ax * qx + ay * qy;
  return make_float3((ax - dot * sx) * il, (ay - dot * sy) * il, -dot * sz * il);
}

// n.d for n = sj - si: plain FP32 when the crossing is not near grazing
// (|n.d| > 1e-2 |n||d|, relative error < 2e-5), else the compensated form.
__device__ __forceinline__ float exact_nd(float3 si, float3 sj, float3 d);
__device__ __forceinline__ float crossing_nd(float3 si, float3 sj, float3 d, float dd) {
  const float nx = __fsub_rn(sj.x, si.x), ny = __fsub_rn(sj.y, si.y), nz = __fsub_rn(sj.z, si.z);
  const float nd = __fmaf_rn(nx, d.x, __fmaf_rn(ny, d.y, __fmul_rn(nz, d.z)));
  const float nn = __fmaf_rn(nx, nx, __fmaf_rn(ny, ny, __fmul_rn(nz, nz)));
  if (__fmul_rn(nd, nd) > __fmul_rn(1e-4f, __fmul_rn(nn, dd))) return nd;
  return exact_nd(si, sj, d);
}

// Exact n.d for n = sj - si (FP32 inputs): n is split into rounded part and
// rounding error (TwoSum), products are split by FMA (TwoProd) and summed with
// compensation -- accurate to about FP32 rounding of the exact value even for
// grazing crossings, where the plain FP32 dot product loses all digits.
__device__ __forceinline__ float exact_nd(float3 si, float3 sj, float3 d) {
  float h0, l0, h1, l1, h2, l2;
  two_sum(sj.x, -si.x, h0, l0);
  two_sum(sj.y, -si.y, h1, l1);
  two_sum(sj.z, -si.z, h2, l2);
  const float p0 = __fmul_rn(h0, d.x), p1 = __fmul_rn(h1, d.y), p2 = __fmul_rn(h2, d.z);
  float e = __fmaf_rn(h0, d.x, -p0);
  e = __fadd_rn(e, __fmaf_rn(h1, d.y, -p1));
  e = __fadd_rn(e, __fmaf_rn(h2, d.z, -p2));
  e = __fmaf_rn(l0, d.x, __fmaf_rn(l1, d.y, __fmaf_rn(l2, d.z, e)));
  float s, c1, c2;
  two_sum(p0, p1, s, c1);
  float s2;
  two_sum(s, p2, s2, c2);
  return __fadd_rn(s2, __fadd_rn(__fadd_rn(c1, c2), e));
}

// A cell record is two 16-byte halves: {x, y, z, sigma} and {begin, end, uid, 0}.
__device__ __forceinline__ float4 cell_pos(const vt_cell* c, int i) {
  return __ldg(reinterpret_cast<const float4*>(c + i));
}
__device__ __forceinline__ int4 cell_csr(const vt_cell* c, int i) {
  return __ldg(reinterpret_cast<const int4*>(c + i) + 1);
}

// neighbour record p: {n = s_j - s_i, j}; with FP16 offsets {n, p} (the id is
// read from the FP32 record when needed)
template <int HALF>
__device__ __forceinline__ float4 nbr_record(const Scene& S, int p) {
  if constexpr (HALF) {
    const uint2 h = __ldg(S.nbr_h + p);
    const float2 xy = __half22float2(*reinterpret_cast<const __half2*>(&h.x));
    return make_float4(xy.x, xy.y, __low2float(*reinterpret_cast<const __half2*>(&h.y)), __int_as_float(p));
  } else {
    return __ldg(S.nbr + p);
  }
}

// FP64 re-evaluation of a grazing plane from the FP32 inputs (exact site
// positions, not the rounded offset): returns false if the plane is not
// crossed forward, else the step dt to it.
__device__ __noinline__ bool grazing_fp64(const vt_cell* cells, int j, float3 si, float3 o, float3 d, float th,
                                          float tl, float* dt) {
  const float4 sj = cell_pos(cells, j);
  const double t64 = (double)th + (double)tl;
  const double n0 = (double)sj.x - (double)si.x, n1 = (double)sj.y - (double)si.y,
               n2 = (double)sj.z - (double)si.z;
  const double den64 = n0 * (double)d.x + n1 * (double)d.y + n2 * (double)d.z;
  if (!(den64 > 0.0)) return false;
  const double r0 = (double)si.x - ((double)o.x + t64 * (double)d.x),
               r1 = (double)si.y - ((double)o.y + t64 * (double)d.y),
               r2 = (double)si.z - ((double)o.z + t64 * (double)d.z);
  const double num64 = n0 * r0 + n1 * r1 + n2 * r2 + 0.5 * (n0 * n0 + n1 * n1 + n2 * n2);
  *dt = (float)(num64 / den64);
  return true;
}

// Greedy descent on the Delaunay graph to the site nearest q, ordering sites
// by (FP32 squared distance, user id). Each move strictly decreases that key,
// so it ends; a local minimum over the Delaunay neighbours is the nearest
// site (Delaunay property).
__device__ int greedy_nearest(const Scene& S, int cell, float3 q, int max_steps, bool& ok) {
  const float4 s0 = cell_pos(S.cell, cell);
  float best = dist2(q, s0.x, s0.y, s0.z);
  int best_uid = cell_csr(S.cell, cell).z;
  for (int it = 0; it < max_steps; ++it) {
    const int4 m = cell_csr(S.cell, cell);
    int bc = cell;
    for (int p = m.x; p < m.y; ++p) {
      const int j = __float_as_int(__ldg(&S.nbr[p].w));
      const float4 sj = cell_pos(S.cell, j);
      const float dd = dist2(q, sj.x, sj.y, sj.z);
      if (dd <= best) {
        const int uid = cell_csr(S.cell, j).z;
        if (dd < best || uid < best_uid) {
          best = dd;
          best_uid = uid;
          bc = j;
        }
      }
    }
    if (bc == cell) return cell;
    cell = bc;
  }
  ok = false;
  return cell;
}

// ---------------------------------------------------------------- anchors
// Exact nearest site of each anchor point: packed (distance bits, user id)
// atomicMin over all sites. Each thread reads a site record once for a group
// of up to kAnchorGroup anchors (blockIdx.y selects the group) and keeps the
// group's minima in registers; warps reduce them before the atomics.
constexpr int kAnchorGroup = 16;
__global__ void k_anchor_nn(Scene S, RP P, const float* __restrict__ o, int n_anchors, unsigned long long* key) {
  const int a0 = blockIdx.y * kAnchorGroup;
  const int na = min(kAnchorGroup, n_anchors - a0);
  float3 q[kAnchorGroup];
  unsigned long long best[kAnchorGroup];
#pragma unroll
  for (int a = 0; a < kAnchorGroup; ++a) {
    const int64_t ar = anchor_ray(P, a0 + min(a, na - 1));
    q[a] = make_float3(o[3 * ar], o[3 * ar + 1], o[3 * ar + 2]);
    best[a] = ~0ull;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 s = cell_pos(S.cell, (int)i);
    const unsigned uid = (unsigned)cell_csr(S.cell, (int)i).z;
#pragma unroll
    for (int a = 0; a < kAnchorGroup; ++a) {
      const unsigned long long k = ((unsigned long long)__float_as_uint(dist2(q[a], s.x, s.y, s.z)) << 32) | uid;
      best[a] = k < best[a] ? k : best[a];
    }
  }
#pragma unroll
  for (int a = 0; a < kAnchorGroup; ++a) {
    unsigned long long b = best[a];
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, off);
      b = v < b ? v : b;
    }
    if ((threadIdx.x & 31) == 0 && a < na) atomicMin(key + a0 + a, b);
  }
}

// One warp per anchor: the greedy descent of greedy_nearest with the
// neighbours of the current cell examined by the 32 lanes at once and the
// smallest (distance bits, user id) key kept, which is the same order as the
// sequential scan, so the same cell results.
__global__ void k_anchor_refine(Scene S, RP P, const float* __restrict__ o, int n_anchors,
                                const int32_t* __restrict__ inv, const unsigned long long* key, int32_t* cell,
                                int max_steps) {
  const int a = blockIdx.x;
  const int lane = threadIdx.x & 31;
  if (a >= n_anchors) return;
  const int64_t ar = anchor_ray(P, a);
  const float3 q = make_float3(o[3 * ar], o[3 * ar + 1], o[3 * ar + 2]);
  int c = inv[(int)(key[a] & 0xffffffffu)];
  auto key_of = [&](int j) {
    const float4 sj = cell_pos(S.cell, j);
    return ((unsigned long long)__float_as_uint(dist2(q, sj.x, sj.y, sj.z)) << 32) |
           (unsigned)cell_csr(S.cell, j).z;
  };
  unsigned long long kc = key_of(c);
  bool moved = true;
  int it = 0;
  for (; it < max_steps && moved; ++it) {
    const int4 m = cell_csr(S.cell, c);
    unsigned long long best = ~0ull;
    int bj = -1;
    for (int p = m.x + lane; p < m.y; p += 32) {
      const int j = __float_as_int(__ldg(&S.nbr[p].w));
      const unsigned long long kj = key_of(j);
      if (kj < best) {
        best = kj;
        bj = j;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
      if (ob < best) {
        best = ob;
        bj = oj;
      }
    }
    moved = best < kc;  // the same on every lane
    if (moved) {
      kc = best;
      c = bj;
    }
  }
  if (lane == 0) {
    if (moved) atomicOr(S.err, (unsigned long long)VT_EBIT_MAX_STEPS);
    cell[a] = c;
  }
}

// ---------------------------------------------------------------- ray mapping
// thread -> ray (-1: none) and its anchor. In image layouts a warp covers a
// 4 x 8 tile (8 columns, 4 rows) of one image.
__device__ __forceinline__ int64_t ray_of_thread(const RP& P, int64_t tid, int& anchor) {
  if (P.layout == 0) {
    if (tid >= P.n_rays) return -1;
    anchor = (int)(tid / P.anchor_stride);
    return tid;
  }
  const int64_t warp = tid >> 5;
  const int lane = (int)(tid & 31);
  int64_t img, t, first;
  int w, h, tiles_x;
  if (P.layout == 1) {
    img = warp / P.tiles_per_img;
    if (img >= P.n_images) return -1;
    t = warp - img * P.tiles_per_img;
    w = P.img_w;
    h = P.img_h;
    tiles_x = P.tiles_x;
    first = img * (int64_t)P.img_w * P.img_h;
  } else {
    if (warp >= P.total_tiles) return -1;
    int lo = 0, hi = P.n_tab - 1;  // last image with first_tile <= warp
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.img[mid].first_tile <= warp)
        lo = mid;
      else
        hi = mid - 1;
    }
    img = lo;
    t = warp - P.img[lo].first_tile;
    w = P.img[lo].w;
    h = P.img[lo].h;
    tiles_x = P.img[lo].tiles_x;
    first = P.img[lo].first_ray;
  }
  // the kWpb warps of a block take a VT_ST_W x kPatchH patch of tiles
  const int st_x = P.layout == 1 ? P.st_x : P.img[img].st_x;
  const int st = (int)(t / kWpb), k = (int)(t % kWpb);
  const int sy = st / st_x, sx = st - sy * st_x;
  const int tx = sx * VT_ST_W + k % VT_ST_W, ty = sy * kPatchH + k / VT_ST_W;
  if (tx >= tiles_x) return -1;
  const int x = tx * 8 + (lane & 7), y = ty * 4 + (lane >> 3);
  if (x >= w || y >= h) return -1;
  const int64_t ray = first + (int64_t)y * w + x;
  anchor = P.layout == 2 ? (int)img : (int)(ray / P.anchor_stride);
  return ray;
}

// ---------------------------------------------------------------- gradient atomics
// Warp aggregation: lanes of `act` holding the same non-negative key combine
// their N values pairwise (butterfly over lane ^ 1, 2, 4, 8, 16; the lower
// lane of a matching pair keeps the sum, the upper one is zeroed); a round
// with no matching pair anywhere is skipped. Values only move, so the sum
// over lanes is unchanged; afterwards the lanes still holding values issue
// the atomics.
template <int N>
__device__ __forceinline__ void warp_combine(unsigned act, int key, float (&v)[N]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int ko = __shfl_xor_sync(act, key, off);
    const bool same = ((act >> (lane ^ off)) & 1u) && ko == key && key >= 0;
    if (__any_sync(act, same)) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float vo = __shfl_xor_sync(act, v[i], off);
        if (same) v[i] = (lane & off) ? 0.f : v[i] + vo;
      }
    }
  }
}

// dL/d(site, sigma) of cell c += (gx, gy, gz, gsig)
__device__ __forceinline__ void add_cell_grad(float4* g_cell, int c, float gx, float gy, float gz, float gsig) {
#if VT_AGG >= 1
  float v[4] = {gx, gy, gz, gsig};
  warp_combine<4>(__activemask(), c, v);
  if (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f) atomicAdd(g_cell + c, make_float4(v[0], v[1], v[2], v[3]));
#else
  atomicAdd(g_cell + c, make_float4(gx, gy, gz, gsig));
#endif
}

// texel gradients of the four bilinear taps: g * w * tap weight
__device__ __forceinline__ void add_tex_grad(float4* g_tex, int64_t b0, int sx, int sy, float g0, float g1, float g2,
                                             float w, const float (&tw)[4], bool agg, uint8_t* touched, int cell) {
  const float a0 = w * tw[0], a1 = w * tw[1], a2 = w * tw[2], a3 = w * tw[3];
  float v[12] = {g0 * a0, g1 * a0, g2 * a0, g0 * a1, g1 * a1, g2 * a1,
                 g0 * a2, g1 * a2, g2 * a2, g0 * a3, g1 * a3, g2 * a3};
#if VT_AGG >= 2
  if (agg) warp_combine<12>(__activemask(), (int)b0, v);
#endif
  const int64_t e[4] = {b0, b0 + sx, b0 + sy, b0 + sx + sy};
  bool any = false;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (v[3 * q] != 0.f || v[3 * q + 1] != 0.f || v[3 * q + 2] != 0.f) {
      atomicAdd(g_tex + e[q], make_float4(v[3 * q], v[3 * q + 1], v[3 * q + 2], 0.f));
      any = true;
    }
  if (any && touched) touched[cell] = 1;  // every writer stores the same value
}

// ---------------------------------------------------------------- the walk
// (hi, lo) -= w * c exactly up to the float-float rounding (TwoProd + TwoSum)
__device__ __forceinline__ void ff_fma_acc(float& hi, float& lo, float w, float c, float sign) {
  const float p = __fmul_rn(w, c);
  const float pe = __fmaf_rn(w, c, -p);
  float s, e;
  two_sum(hi, sign * p, s, e);
  lo = __fadd_rn(lo, __fmaf_rn(sign, pe, e));
  hi = s;
}

template <int MODE, int APP, int DIST>
struct WalkBounds {
  static constexpr int warps = MODE == FWD   ? ((APP || DIST) ? VT_FWD_WARPS_EXT : VT_FWD_WARPS)
                               : MODE == BWD ? ((APP || DIST) ? VT_BWD_WARPS_EXT : VT_BWD_WARPS)
                                             : 16;
  static constexpr int blocks = warps / kWpb;  // resident blocks per SM requested
};

template <int MODE, int DT, int APP, int DIST, int HALF>
__global__ void __launch_bounds__(kWpb * 32, WalkBounds<MODE, APP, DIST>::blocks)
    k_walk(Scene S, RP P, const float* __restrict__ O, const float* __restrict__ D,
           const int32_t* __restrict__ anchor_cell, float* __restrict__ rgb_out, float* __restrict__ T_out,
           int32_t* __restrict__ steps_out, Grad G, Trace TR) {
#if VT_STAGE
  __shared__ float4 stage[kWpb][kStageCap];  // per warp: neighbour records of its shared cell
#endif
  int anchor = 0;
  const int64_t ray = ray_of_thread(P, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, anchor);
  if (ray < 0) return;
  const float3 o = make_float3(O[3 * ray], O[3 * ray + 1], O[3 * ray + 2]);
  const float3 d = make_float3(D[3 * ray], D[3 * ray + 1], D[3 * ray + 2]);
  const float dd = __fmaf_rn(d.x, d.x, __fmaf_rn(d.y, d.y, __fmul_rn(d.z, d.z)));
  // colour (FWD) as float-float: C = Ch + Cl
  float Ch0 = 0.f, Ch1 = 0.f, Ch2 = 0.f, Cl0 = 0.f, Cl1 = 0.f, Cl2 = 0.f;
  float T = 1.f;
  int k = 0;
  // distortion loss (Eq. 2) in the coordinate s(t) = 1 - 1/(1+t). Composited
  // intervals are contiguous, so sbar_k - sbar_{k-1} = (ds_{k-1} + ds_k)/2 with
  // ds = s(b) - s(a) = (b - a)/((1+a)(1+b)); sbar' = sbar - sbar_first. Sums
  // in the order of the walk: W = sum w, Q = sum w sbar',
  // A_k = sum_{l<k} w_l (sbar_k - sbar_l) = A_{k-1} + W_{<k} gap_k,
  // L = sum_k w_k (2 A_k + w_k ds_k / 3).
  float dW = 0.f, dQ = 0.f, dA = 0.f, dL = 0.f, dsb = 0.f, dsp = -1.f;
  // backward: forward totals, dL/dL_dist, sum_{l<k} G_l w_l, pending exit term
  float dLt = 0.f, dWt = 0.f, dQt = 0.f, gdd = 0.f, dP = 0.f, p_db = 0.f;
  if (DIST && MODE == BWD) {
    dLt = G.dist[3 * ray];
    dWt = G.dist[3 * ray + 1];
    dQt = G.dist[3 * ray + 2];
    gdd = G.gdist[ray];
  }
  const bool bad = !(dd > 0.f) || !isfinite(dd) || !isfinite(o.x) || !isfinite(o.y) || !isfinite(o.z);
  // clip [t_near, t_far] to the optional box (slab test)
  float t0 = P.t_near, t1 = P.t_far;
  if (P.clip && !bad) {
    const float ov[3] = {o.x, o.y, o.z}, dv[3] = {d.x, d.y, d.z};
    const float lv[3] = {P.lo.x, P.lo.y, P.lo.z}, hv[3] = {P.hi.x, P.hi.y, P.hi.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (dv[a] != 0.f) {
        float ta = __fdiv_rn(__fsub_rn(lv[a], ov[a]), dv[a]), tb = __fdiv_rn(__fsub_rn(hv[a], ov[a]), dv[a]);
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
      } else if (ov[a] < lv[a] || ov[a] > hv[a]) {
        t1 = t0;
      }
    }
  }
  if (bad) {
    atomicOr(S.err, (unsigned long long)VT_EBIT_BAD_RAY);
  } else if (t1 > t0) {
    // taps of the ray direction (appearance 0) / of the view direction -d (T_vd, appearance 1)
    const Taps tp = taps_for(APP ? make_float3(-d.x, -d.y, -d.z) : d, S.R);
    const float Gd = __fmul_rn(1e-6f, sqrtf(dd));  // grazing scale 1e-6 |d|
    // BWD: g = dL/dC and the suffix S_k = C_out - sum_{m<=k} w_m c_m as float-float
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, Sh0 = 0.f, Sh1 = 0.f, Sh2 = 0.f, Sl0 = 0.f, Sl1 = 0.f, Sl2 = 0.f;
    if (MODE == BWD) {
      g0 = G.grad[3 * ray];
      g1 = G.grad[3 * ray + 1];
      g2 = G.grad[3 * ray + 2];
      Sh0 = G.rgb[3 * ray];
      Sh1 = G.rgb[3 * ray + 1];
      Sh2 = G.rgb[3 * ray + 2];
      if (G.rgb_lo) {
        Sl0 = G.rgb_lo[3 * ray];
        Sl1 = G.rgb_lo[3 * ray + 1];
        Sl2 = G.rgb_lo[3 * ray + 2];
      }
    }
    // start cell: the anchor's cell if the origin is the anchor point, else a
    // greedy walk from it to the origin
    int cell;
    {
      const int64_t ar = anchor_ray(P, anchor);
      cell = anchor_cell[anchor];
      if (O[3 * ar] != o.x || O[3 * ar + 1] != o.y || O[3 * ar + 2] != o.z) {
        bool ok = true;
        cell = greedy_nearest(S, cell, o, P.max_steps, ok);
        if (!ok) atomicOr(S.err, (unsigned long long)VT_EBIT_MAX_STEPS);
      }
    }
    float th = 0.f, tl = 0.f;  // entry parameter of the current cell (float-float)
    // BWD carry: previous cell, its sigma * dL/dtau, its dL/dsigma, site
    // gradient so far and position; whether the entry crossing is differentiable
    int pc = -1;
    float p_sdtau = 0.f, p_gsig = 0.f;
    float3 p_gs = make_float3(0.f, 0.f, 0.f), p_s = make_float3(0.f, 0.f, 0.f);
    bool cross_valid = false;
    float p_xt = 0.f;  // appearance 1: colour term dL/dt pending on the previous cell's exit crossing
    for (;;) {
      if (k >= P.max_steps) {
        atomicOr(S.err, (unsigned long long)VT_EBIT_MAX_STEPS);
        break;
      }
      const float4 cp = cell_pos(S.cell, cell);
      const int4 m = cell_csr(S.cell, cell);
      const float3 si = make_float3(cp.x, cp.y, cp.z);
      const float sig = cp.w;
      // texels of this cell (independent of the exit search)
      TexRaw<DT> tx0, tx1, tx2, tx3;
      const int64_t tb0 = (int64_t)cell * S.RR + tp.base;
      if (MODE != TRACE && VT_TEX_EARLY && !APP) {
        tx0 = load_texel<DT>(S.tex, tb0);
        tx1 = load_texel<DT>(S.tex, tb0 + tp.sx);
        tx2 = load_texel<DT>(S.tex, tb0 + tp.sy);
        tx3 = load_texel<DT>(S.tex, tb0 + tp.sx + tp.sy);
      }
      const float3 r = rel_pos(si, o, d, th, tl);
      // ---- exit search over the Delaunay neighbours (offset records n = s_j - s_i)
      // grazing bound for this cell: |n.d| <= 1e-6 |d| max_j |n_j| (a superset
      // of the planes with |n.d| <= 1e-6 |n||d|)
      const float Gc = __fmul_rn(Gd, __int_as_float(m.w));
      float bn = 1.f, bd = 0.f;  // best dt = bn / bd (bd == 0: none yet)
      int bj = -1;
      // grazing planes (|n.d| <= Gc) are only noted in the hot loop, through
      // the running minimum of |n.d|; their FP64 recheck runs in a second pass
      // over the cell when there is one (rare). Keeping the FP64 call out of
      // the unrolled loop: 350.5 -> 379.3 Mrays/s fwd+bwd on 3M sites / 4 views.
      float mind = INFINITY;
      // One neighbour record q = {n, j}: keep its forward crossing if nearer.
      // The body has no branch: every plane's numerator n.(r + n/2) is formed
      // and the candidate kept by a predicated select. On 3M sites / 4 views
      // this cut the forward walk from 4.21 to 3.18 ms and the backward from
      // 6.29 to 5.30 ms against a body that branched on n.d first and noted
      // grazing planes in an else branch (the branches inside the unrolled
      // loop had cost more than the arithmetic they skipped).
      auto consider = [&](const float4 q) {
        const float den = __fmaf_rn(q.x, d.x, __fmaf_rn(q.y, d.y, __fmul_rn(q.z, d.z)));
        const float num = __fmaf_rn(q.x, __fmaf_rn(0.5f, q.x, r.x),
                                    __fmaf_rn(q.y, __fmaf_rn(0.5f, q.y, r.y), __fmul_rn(q.z, __fmaf_rn(0.5f, q.z, r.z))));
        if (den > Gc && __fmul_rn(num, bd) < __fmul_rn(bn, den)) {
          bn = num;
          bd = den;
          bj = __float_as_int(q.w);
        }
        mind = fminf(mind, fabsf(den));
      };
#if VT_STAGE
      // Warp-shared cell (Sec. 5.6 warp-coherent tiles): when all 32 lanes of
      // the warp are in the same cell, its neighbour records are read once
      // into shared memory with one coalesced load and every lane searches
      // them there. The test is warp-uniform (all lanes active and equal), so
      // the whole warp takes the same branch and the __syncwarp()s are
      // reached by all 32 lanes. Same arithmetic on the same values as the
      // other branch: the decisions do not depend on which branch ran.
      bool staged = false;
      if (!HALF && __activemask() == 0xffffffffu)
        staged = __match_any_sync(0xffffffffu, cell) == 0xffffffffu && m.y - m.x <= kStageCap;
      if (staged) {
        float4* buf = stage[threadIdx.x >> 5];
        const int deg = m.y - m.x;
        for (int q = threadIdx.x & 31; q < deg; q += 32) buf[q] = __ldg(S.nbr + m.x + q);
        __syncwarp();
#pragma unroll kNbrUnroll
        for (int p = 0; p < deg; ++p) consider(buf[p]);
        __syncwarp();  // every lane has read buf before the next step refills it
      } else
#endif
      {
#pragma unroll kNbrUnroll
        for (int p = m.x; p < m.y; ++p) consider(nbr_record<HALF>(S, p));
      }
      // grazing planes (|n.d| <= Gc) of this cell
      const bool grazed = mind <= Gc;
      if (grazed) {
        for (int p = m.x; p < m.y; ++p) {
          const float4 q = nbr_record<HALF>(S, p);
          const float den = __fmaf_rn(q.x, d.x, __fmaf_rn(q.y, d.y, __fmul_rn(q.z, d.z)));
          if (!(fabsf(den) <= Gc)) continue;
          atomicAdd(S.err + 1, 1ull);
          const int jg = HALF ? __ldg(reinterpret_cast<const int*>(S.nbr + p) + 3) : __float_as_int(q.w);
          float num;
          if (!grazing_fp64(S.cell, jg, si, o, d, th, tl, &num)) continue;
          if (__fmul_rn(num, bd) < bn) {  // den = 1
            bn = num;
            bd = 1.f;
            bj = __float_as_int(q.w);
          }
        }
      }
      if (HALF && bj >= 0) bj = __ldg(reinterpret_cast<const int*>(S.nbr + bj) + 3);
      ++k;
      if (MODE != TRACE && !VT_TEX_EARLY && !APP) {
        tx0 = load_texel<DT>(S.tex, tb0);
        tx1 = load_texel<DT>(S.tex, tb0 + tp.sx);
        tx2 = load_texel<DT>(S.tex, tb0 + tp.sy);
        tx3 = load_texel<DT>(S.tex, tb0 + tp.sx + tp.sy);
      }
      const float dt = bj >= 0 ? __fdividef(bn, bd) : INFINITY;
      float eh = th, el = tl;  // exit parameter
      if (bj >= 0)
        ff_add(eh, el, dt);
      else
        eh = INFINITY, el = 0.f;
      const bool exit_beyond = bj < 0 || ff_ge(eh, el, t1);
      if (MODE == TRACE) {
        const int64_t slot = ray * (int64_t)TR.max_cells + (k - 1);
        if (k <= TR.max_cells) {
          TR.cells[slot] = m.z;
          if (TR.t_exit) TR.t_exit[slot] = bj >= 0 ? __fadd_rn(eh, el) : INFINITY;
        }
      }
      // ---- segment [max(t_in, t0), min(t_exit, t1)]
      const bool start_clip = !ff_ge(th, tl, t0);
      float delta;
      if (!start_clip && !exit_beyond) {
        delta = dt;
      } else {
        float ah = th, al = tl, bh = eh, bl = el;
        if (start_clip) ah = t0, al = 0.f;
        if (exit_beyond) bh = t1, bl = 0.f;
        delta = __fadd_rn(__fsub_rn(bh, ah), __fsub_rn(bl, al));
      }
      float dist_da = 0.f, dist_db = 0.f;  // distortion: direct dL/da, dL/db of this interval
      bool stop = false;
      float dtau = 0.f, w = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
      bool coloured = false;
      float tw[4];
      // appearance 1: surface direction, its taps, and the colour gradient terms
      float3 dsurf = make_float3(0.f, 0.f, 0.f);
      float rinv = 0.f, gt_col = 0.f;  // rinv: 1/|x - p| of the surface point (0: none)
      float3 gx_col = make_float3(0.f, 0.f, 0.f);
      Taps tv{0, 0, 0, 0.f, 0.f, 0.f, 0.f};
      float wv[4] = {0.f, 0.f, 0.f, 0.f};
      int64_t tbv = 0;
      float gz0 = 0.f, gz1 = 0.f, gz2 = 0.f;
      if (delta > 0.f) {
        const float e = __expf(-__fmul_rn(sig, delta));
        const float alpha = __fsub_rn(1.f, e);
        w = __fmul_rn(T, alpha);
        const float Tn = __fmul_rn(T, e);
        if (MODE != TRACE && (!(P.skip > 0.f) || w >= P.skip)) {
          coloured = true;
          tap_weights(tp, tw);
          if constexpr (APP == 0) {
            const float3 a0 = texel_rgb<DT>(tx0), a1 = texel_rgb<DT>(tx1), a2 = texel_rgb<DT>(tx2),
                         a3 = texel_rgb<DT>(tx3);
            c0 = __fmaf_rn(tw[3], a3.x, __fmaf_rn(tw[2], a2.x, __fmaf_rn(tw[1], a1.x, __fmul_rn(tw[0], a0.x))));
            c1 = __fmaf_rn(tw[3], a3.y, __fmaf_rn(tw[2], a2.y, __fmaf_rn(tw[1], a1.y, __fmul_rn(tw[0], a0.y))));
            c2 = __fmaf_rn(tw[3], a3.z, __fmaf_rn(tw[2], a2.z, __fmaf_rn(tw[1], a1.z, __fmul_rn(tw[0], a0.z))));
          } else {
            // Sec. 5.1-5.2: x = entry point (origin cell: exit point, or segment end)
            float3 vs;
            if (k > 1) {
              vs = make_float3(-r.x, -r.y, -r.z);
            } else {
              const float tx = bj >= 0 ? dt : __fsub_rn(t1, th);
              vs = make_float3(__fmaf_rn(tx, d.x, -r.x), __fmaf_rn(tx, d.y, -r.y), __fmaf_rn(tx, d.z, -r.z));
            }
            const float ss = vs.x * vs.x + vs.y * vs.y + vs.z * vs.z;
            rinv = ss > 0.f ? rsqrtf(ss) : 0.f;  // 1/|x - p|
            const float il = ss > 0.f ? rinv : rsqrtf(dd);
            dsurf = ss > 0.f ? make_float3(vs.x * il, vs.y * il, vs.z * il) : make_float3(d.x * il, d.y * il, d.z * il);
            tv = taps_for<true>(dsurf, S.R);
            tap_weights(tv, wv);
            tbv = (int64_t)cell * S.RR + tv.base;
            const int64_t tbd = tb0;  // view-dependent taps of this cell
            const float3 a0 = texel_rgb<DT>(load_texel<DT>(S.tex, tbv));
            const float3 a1 = texel_rgb<DT>(load_texel<DT>(S.tex, tbv + tv.sx));
            const float3 a2 = texel_rgb<DT>(load_texel<DT>(S.tex, tbv + tv.sy));
            const float3 a3 = texel_rgb<DT>(load_texel<DT>(S.tex, tbv + tv.sx + tv.sy));
            const float3 b0 = texel_rgb<DT>(load_texel<DT>(S.tex_vd, tbd));
            const float3 b1 = texel_rgb<DT>(load_texel<DT>(S.tex_vd, tbd + tp.sx));
            const float3 b2 = texel_rgb<DT>(load_texel<DT>(S.tex_vd, tbd + tp.sy));
            const float3 b3 = texel_rgb<DT>(load_texel<DT>(S.tex_vd, tbd + tp.sx + tp.sy));
            const float z0 = wv[0] * a0.x + wv[1] * a1.x + wv[2] * a2.x + wv[3] * a3.x + tw[0] * b0.x + tw[1] * b1.x +
                             tw[2] * b2.x + tw[3] * b3.x;
            const float z1 = wv[0] * a0.y + wv[1] * a1.y + wv[2] * a2.y + wv[3] * a3.y + tw[0] * b0.y + tw[1] * b1.y +
                             tw[2] * b2.y + tw[3] * b3.y;
            const float z2 = wv[0] * a0.z + wv[1] * a1.z + wv[2] * a2.z + wv[3] * a3.z + tw[0] * b0.z + tw[1] * b1.z +
                             tw[2] * b2.z + tw[3] * b3.z;
            c0 = __fdividef(1.f, 1.f + __expf(-z0));
            c1 = __fdividef(1.f, 1.f + __expf(-z1));
            c2 = __fdividef(1.f, 1.f + __expf(-z2));
            if (MODE == BWD) {
              // dL/dz = g w c (1 - c); through the bilinear fetch and the octahedral
              // map into the surface direction, then into x and the site
              gz0 = g0 * w * c0 * (1.f - c0);
              gz1 = g1 * w * c1 * (1.f - c1);
              gz2 = g2 * w * c2 * (1.f - c2);
              const float gu = tv.gxs * (gz0 * ((1.f - tv.fy) * (a1.x - a0.x) + tv.fy * (a3.x - a2.x)) +
                                         gz1 * ((1.f - tv.fy) * (a1.y - a0.y) + tv.fy * (a3.y - a2.y)) +
                                         gz2 * ((1.f - tv.fy) * (a1.z - a0.z) + tv.fy * (a3.z - a2.z)));
              const float gv = tv.gys * (gz0 * ((1.f - tv.fx) * (a2.x - a0.x) + tv.fx * (a3.x - a1.x)) +
                                         gz1 * ((1.f - tv.fx) * (a2.y - a0.y) + tv.fx * (a3.y - a1.y)) +
                                         gz2 * ((1.f - tv.fx) * (a2.z - a0.z) + tv.fx * (a3.z - a1.z)));
              const float3 gd = oct_vjp(dsurf, gu, gv);
              if (rinv > 0.f) {
                const float dg = gd.x * dsurf.x + gd.y * dsurf.y + gd.z * dsurf.z;
                gx_col = make_float3((gd.x - dsurf.x * dg) * rinv, (gd.y - dsurf.y * dg) * rinv,
                                     (gd.z - dsurf.z * dg) * rinv);
                gt_col = gx_col.x * d.x + gx_col.y * d.y + gx_col.z * d.z;
              }
            }
          }
          if (MODE == FWD) {
            ff_fma_acc(Ch0, Cl0, w, c0, 1.f);
            ff_fma_acc(Ch1, Cl1, w, c1, 1.f);
            ff_fma_acc(Ch2, Cl2, w, c2, 1.f);
          } else if (MODE == BWD) {
            ff_fma_acc(Sh0, Sl0, w, c0, -1.f);
            ff_fma_acc(Sh1, Sl1, w, c1, -1.f);
            ff_fma_acc(Sh2, Sl2, w, c2, -1.f);
          }
        }
        if (MODE == BWD) {
          // dL/dtau_k = g . (T_{k+1} c_k - S_k)
          dtau = g0 * ((Tn * c0 - Sh0) - Sl0) + g1 * ((Tn * c1 - Sh1) - Sl1) + g2 * ((Tn * c2 - Sh2) - Sl2);
        }
        if (DIST && MODE != TRACE) {
          const float a = start_clip ? t0 : __fadd_rn(th, tl);
          const float b = exit_beyond ? t1 : __fadd_rn(eh, el);
          const float ia = __fdividef(1.f, 1.f + a), ib = __fdividef(1.f, 1.f + b);
          const float ds = delta * ia * ib;
          if (dsp >= 0.f) {
            const float gap = 0.5f * (dsp + ds);
            dsb += gap;
            dA = __fmaf_rn(dW, gap, dA);
          }
          dsp = ds;
          if (MODE == FWD) {
            dL = __fmaf_rn(w, __fmaf_rn(w * ds, 1.f / 3.f, 2.f * dA), dL);
          } else {
            // G_k = dL/dw_k = 2 (A_k + B_k) + 2/3 w_k ds_k,
            // B_k = sum_{l>k} w_l (sbar_l - sbar_k) = Q_{>k} - sbar'_k W_{>k}
            const float Wg = dWt - dW - w, Qg = dQt - dQ - w * dsb;
            const float Gk = 2.f * (dA + (Qg - dsb * Wg)) + (2.f / 3.f) * w * ds;
            // dw_k/dtau_k = T_{k+1}; dw_m/dtau_k = -w_m (m > k); sum_m G_m w_m = 2 L
            const float suffix = 2.f * dLt - dP - Gk * w;
            dtau = __fmaf_rn(gdd, Gk * Tn - suffix, dtau);
            dP = __fmaf_rn(Gk, w, dP);
            // interval ends: sbar = (s(a)+s(b))/2, ds = s(b)-s(a), s' = 1/(1+t)^2
            const float dsbar = 2.f * w * (dW - Wg), ddsk = w * w * (1.f / 3.f);
            dist_da = gdd * ia * ia * (0.5f * dsbar - ddsk);
            dist_db = gdd * ib * ib * (0.5f * dsbar + ddsk);
          }
          dQ = __fmaf_rn(w, dsb, dQ);
          dW += w;
        }
        T = Tn;
        if (T < P.T_eps) stop = true;
      }
      if (MODE == BWD) {
        // crossing between the previous cell and this one (entry face):
        // dL/dt_b = sigma_prev dtau_prev - sigma dtau (inside the extent)
        //           + colour terms of surface points on this face (appearance 1);
        // x_b - s_prev = n - r, s_cur - x_b = r
        float3 gs = make_float3(0.f, 0.f, 0.f);
        float dLdt = cross_valid ? p_sdtau - sig * dtau : 0.f;
        if (DIST && cross_valid) dLdt += p_db + dist_da;
        if (APP) dLdt += p_xt + (k > 1 ? gt_col : 0.f);
        if (pc >= 0 && dLdt != 0.f) {
#if VT_BWD_RELOAD_PREV
          {  // previous site from its record (L1-resident) instead of a live register triple
            const float4 pp = cell_pos(S.cell, pc);
            p_s = make_float3(pp.x, pp.y, pp.z);
          }
#endif
          const float nd = crossing_nd(p_s, si, d, dd);
          const float dtb = __fdividef(dLdt, nd);
          const float nx = __fsub_rn(si.x, p_s.x), ny = __fsub_rn(si.y, p_s.y), nz = __fsub_rn(si.z, p_s.z);
          p_gs.x += dtb * (nx - r.x);
          p_gs.y += dtb * (ny - r.y);
          p_gs.z += dtb * (nz - r.z);
          gs = make_float3(dtb * r.x, dtb * r.y, dtb * r.z);
        }
        if (APP) {  // the site itself moves the surface direction
          gs.x -= gx_col.x;
          gs.y -= gx_col.y;
          gs.z -= gx_col.z;
        }
        if (pc >= 0) add_cell_grad(G.g_cell, pc, p_gs.x, p_gs.y, p_gs.z, p_gsig);
        if (coloured && w > 0.f) {
          if constexpr (APP == 0) {
            add_tex_grad(G.g_tex, tb0, tp.sx, tp.sy, g0, g1, g2, w, tw, S.n * S.RR < ((int64_t)1 << 31), G.touched,
                         cell);
          } else {
            add_tex_grad(G.g_tex, tbv, tv.sx, tv.sy, gz0, gz1, gz2, 1.f, wv, S.n * S.RR < ((int64_t)1 << 31), G.touched,
                         cell);
            add_tex_grad(G.g_tex_vd, tb0, tp.sx, tp.sy, gz0, gz1, gz2, 1.f, tw, S.n * S.RR < ((int64_t)1 << 31),
                         G.touched, cell);
          }
        }
        pc = cell;
        p_sdtau = sig * dtau;
        p_gsig = dtau * delta;
        p_gs = gs;
#if !VT_BWD_RELOAD_PREV
        p_s = si;
#endif
        // will the crossing at this cell's exit be differentiable?
        cross_valid = (bj >= 0) && !exit_beyond && ff_gt(eh, el, t0);
        // appearance 1: the origin cell's colour sits on its exit crossing
        const float xt_exit = (APP && k == 1 && bj >= 0) ? gt_col : 0.f;
        const float dLdt_exit = (stop && cross_valid ? p_sdtau + (DIST ? dist_db : 0.f) : 0.f) + xt_exit;
        if ((stop || exit_beyond) && bj >= 0 && dLdt_exit != 0.f) {
          // the walk ends in this cell but its exit plane still moves delta_K
          // (terminated inside the extent) and/or its surface point
          const float4 q4 = cell_pos(S.cell, bj);
          const float3 sj = make_float3(q4.x, q4.y, q4.z);
          const float3 re = rel_pos(si, o, d, eh, el);  // s_K - x_out
          const float nd = crossing_nd(si, sj, d, dd);
          const float dtb = __fdividef(dLdt_exit, nd);
          const float nx = __fsub_rn(sj.x, si.x), ny = __fsub_rn(sj.y, si.y), nz = __fsub_rn(sj.z, si.z);
          p_gs.x -= dtb * re.x;
          p_gs.y -= dtb * re.y;
          p_gs.z -= dtb * re.z;
          add_cell_grad(G.g_cell, bj, dtb * (re.x + nx), dtb * (re.y + ny), dtb * (re.z + nz), 0.f);
        }
        p_xt = xt_exit;
        if (DIST) p_db = dist_db;
      }
      if (stop || exit_beyond) break;
      cell = bj;
      th = eh;
      tl = el;
    }
    if (MODE == BWD && pc >= 0) add_cell_grad(G.g_cell, pc, p_gs.x, p_gs.y, p_gs.z, p_gsig);
    if (MODE == FWD) {
      ff_fma_acc(Ch0, Cl0, T, P.bg.x, 1.f);
      ff_fma_acc(Ch1, Cl1, T, P.bg.y, 1.f);
      ff_fma_acc(Ch2, Cl2, T, P.bg.z, 1.f);
    }
  } else {
    Ch0 = P.bg.x;
    Ch1 = P.bg.y;
    Ch2 = P.bg.z;
  }
  if (MODE == FWD) {
    const float r0 = __fadd_rn(Ch0, Cl0), r1 = __fadd_rn(Ch1, Cl1), r2 = __fadd_rn(Ch2, Cl2);
    rgb_out[3 * ray] = r0;
    rgb_out[3 * ray + 1] = r1;
    rgb_out[3 * ray + 2] = r2;
    if (G.rgb_lo) {  // forward: residual output (C - rounded C), Fast2Sum
      float* lo = const_cast<float*>(G.rgb_lo);
      lo[3 * ray] = __fsub_rn(Cl0, __fsub_rn(r0, Ch0));
      lo[3 * ray + 1] = __fsub_rn(Cl1, __fsub_rn(r1, Ch1));
      lo[3 * ray + 2] = __fsub_rn(Cl2, __fsub_rn(r2, Ch2));
    }
    if (T_out) T_out[ray] = T;
    if (steps_out) steps_out[ray] = k;
    if (DIST) {
      G.dist[3 * ray] = dL;
      G.dist[3 * ray + 1] = dW;
      G.dist[3 * ray + 2] = dQ;
    }
  } else if (MODE == TRACE) {
    TR.n_cells[ray] = k;
    if (k > TR.max_cells) atomicOr(S.err, (unsigned long long)VT_EBIT_CAPACITY);
  }
}

// user-order gradients from the Morton-ordered scratch (overwrites outputs)
// Gradient scratch (Morton order, RGBA float4 per texel) -> caller's FP32
// arrays in user order. One warp per cell: the warp writes the cell's R*R*3
// output floats contiguously (coalesced 128-B stores) and gathers them from
// the cell's scratch block. With `touched` (the backward walk flags the cells
// it added texel gradients to), cells not flagged are known to be zero: their
// outputs are written as zeros without reading the scratch, and the flagged
// cells' scratch is re-zeroed here, so the next backward needs no clear.
__device__ __forceinline__ void copy_tex_grad(int lane, int RR, bool hot, float4* __restrict__ src, float* dst,
                                              bool rezero) {
  const float* s = reinterpret_cast<const float*>(src);
  if (dst)
    for (int f = lane; f < RR * 3; f += 32) {
      const int t = f / 3, c = f - 3 * t;
      dst[f] = hot ? s[4 * t + c] : 0.f;
    }
  if (hot && rezero) {
    __syncwarp();  // every lane has read the block
    for (int t = lane; t < RR; t += 32) src[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void k_grad_out(int64_t n, int RR, const vt_cell* __restrict__ cells, const float4* __restrict__ g_cell,
                           float4* g_tex, float* gs, float* gsig, float* gtex, float4* g_tex_vd, float* gtex_vd,
                           uint8_t* touched) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int64_t u = cell_csr(cells, (int)i).z;
    const bool hot = !touched || touched[i];
    if (gtex || touched) copy_tex_grad(lane, RR, hot, g_tex + i * RR, gtex ? gtex + u * RR * 3 : nullptr, touched);
    if (g_tex_vd && (gtex_vd || touched))
      copy_tex_grad(lane, RR, hot, g_tex_vd + i * RR, gtex_vd ? gtex_vd + u * RR * 3 : nullptr, touched);
    if (lane == 0) {
      if (touched && hot) touched[i] = 0;
      const float4 c = g_cell[i];
      if (gs) {
        gs[3 * u] = c.x;
        gs[3 * u + 1] = c.y;
        gs[3 * u + 2] = c.z;
      }
      if (gsig) gsig[u] = c.w;
    }
  }
}

// the permute launch (measured alternatives, 3M cells: loops unrolled for 8x8
// textures, +0.26 ms per call; outputs walked in user order, -0.02 ms, within
// noise; neither kept)
void launch_grad_out(int64_t n, int RR, const vt_cell* cells, const float4* g_cell, float4* g_tex, float* gs,
                     float* gsig, float* gtex, float4* g_tex_vd, float* gtex_vd, uint8_t* touched, cudaStream_t st) {
  vt_note_launch();
  k_grad_out<<<vt_grid(n * 32, 256, 152 * 16), 256, 0, st>>>(n, RR, cells, g_cell, g_tex, gs, gsig, gtex, g_tex_vd,
                                                              gtex_vd, touched);
}

// ---------------------------------------------------------------- host side
vt_status make_rp(const vt_scene* s, int64_t n_rays, const vt_render_params* p, RP& P) {
  if (!p) return VT_ERR_INVALID_ARG;
  P.t_near = p->t_near;
  P.t_far = p->t_far;
  P.clip = p->use_clip_box != 0;
  P.lo = make_float3(p->clip_lo[0], p->clip_lo[1], p->clip_lo[2]);
  P.hi = make_float3(p->clip_hi[0], p->clip_hi[1], p->clip_hi[2]);
  P.T_eps = p->T_eps;
  P.skip = p->skip_weight;
  P.bg = make_float3(p->bg[0], p->bg[1], p->bg[2]);
  P.appearance = p->appearance;
  if (p->appearance != 0 && p->appearance != 1) return VT_ERR_INVALID_ARG;
  if (p->appearance == 1 && !s->tex_vd) return VT_ERR_INVALID_ARG;
  P.img_w = p->img_w;
  P.img_h = p->img_h;
  P.n_images = p->n_images;
  P.n_rays = n_rays;
  int64_t ms = p->max_steps > 0 ? p->max_steps : (s->n * 4 < (1 << 20) ? s->n * 4 : (1 << 20));
  if (ms < 4) ms = 4;
  P.max_steps = (int)ms;
  if (!(p->t_far >= p->t_near) || !isfinite(p->t_near) || !(p->T_eps >= 0.f)) return VT_ERR_INVALID_ARG;
  int64_t per_image;
  P.layout = 0;
  P.n_tab = 0;
  P.total_tiles = 0;
  if (p->image_sizes) {
    // images of different sizes, one anchor each
    if (p->n_images <= 0 || p->n_images > VT_MAX_ANCHORS) return VT_ERR_INVALID_ARG;
    int64_t ray0 = 0, tile0 = 0;
    for (int i = 0; i < p->n_images; ++i) {
      const int w = p->image_sizes[2 * i], h = p->image_sizes[2 * i + 1];
      if (w <= 0 || h <= 0) return VT_ERR_INVALID_ARG;
      ImgEnt& e = P.img[i];
      e.first_ray = ray0;
      e.first_tile = tile0;
      e.w = w;
      e.h = h;
      e.tiles_x = (w + 7) / 8;
      e.st_x = (e.tiles_x + VT_ST_W - 1) / VT_ST_W;
      ray0 += (int64_t)w * h;
      // warps of this image: 8 per tile patch
      tile0 += (int64_t)e.st_x * (((h + 3) / 4 + kPatchH - 1) / kPatchH) * kWpb;
    }
    if (ray0 != n_rays) return VT_ERR_INVALID_ARG;
    P.layout = 2;
    P.n_tab = p->n_images;
    P.total_tiles = tile0;
    P.tiles_x = P.tiles_per_img = 0;
    P.anchor_stride = 1;
    return VT_OK;
  }
  if (p->img_w > 0) {
    P.layout = 1;
    if (p->img_h <= 0 || p->n_images <= 0) return VT_ERR_INVALID_ARG;
    per_image = (int64_t)p->img_w * p->img_h;
    if (per_image * p->n_images != n_rays) return VT_ERR_INVALID_ARG;
    P.tiles_x = (p->img_w + 7) / 8;
    // warps per image: kWpb per patch of VT_ST_W x kPatchH tiles (ragged
    // patches at the right and bottom edges have idle warps)
    P.st_x = (P.tiles_x + VT_ST_W - 1) / VT_ST_W;
    P.tiles_per_img = P.st_x * (((p->img_h + 3) / 4 + kPatchH - 1) / kPatchH) * kWpb;
    int64_t groups = (p->n_images + VT_MAX_ANCHORS - 1) / VT_MAX_ANCHORS;
    P.anchor_stride = per_image * groups;
  } else {
    P.tiles_x = P.tiles_per_img = 0;
    int64_t st = (n_rays + VT_MAX_ANCHORS - 1) / VT_MAX_ANCHORS;
    P.anchor_stride = st < 4096 ? 4096 : st;
  }
  return VT_OK;
}

int64_t walk_threads(const RP& P) {
  if (P.layout == 0) return P.n_rays;
  if (P.layout == 2) return P.total_tiles * 32;
  return (int64_t)P.n_images * P.tiles_per_img * 32;
}

int n_anchors(const RP& P) {
  if (P.layout == 2) return P.n_tab;
  return (int)((P.n_rays + P.anchor_stride - 1) / P.anchor_stride);
}

Scene scene_view(vt_scene* s) {
  Scene S;
  S.cell = s->cell;
  S.nbr = s->nbr;
  S.nbr_h = s->nbr_h;
  S.tex = s->tex;
  S.tex_vd = s->tex_vd;
  S.n = s->n;
  S.R = s->R;
  S.RR = s->R * s->R;
  S.err = s->d_err;
  return S;
}

vt_status anchors(vt_scene* s, const Scene& S, const RP& P, const float* o, cudaStream_t st) {
  const int na = n_anchors(P);
  if (na < 1 || na > VT_MAX_ANCHORS) return VT_ERR_INVALID_ARG;
  VT_CUDA_TRY(cudaMemsetAsync(s->anchor_key, 0xff, na * sizeof(unsigned long long), st));
  dim3 g(vt_grid(s->n, 256, 152 * 4), (na + kAnchorGroup - 1) / kAnchorGroup);
  vt_note_launch();
  k_anchor_nn<<<g, 256, 0, st>>>(S, P, o, na, s->anchor_key);
  vt_note_launch();
  k_anchor_refine<<<na, 32, 0, st>>>(S, P, o, na, s->inv, s->anchor_key, s->anchor_cell, P.max_steps);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

template <int MODE, int APP, int DIST, int HALF = 0>
void launch_walk_app(vt_scene* s, const Scene& S, const RP& P, const float* o, const float* d, float* rgb, float* T,
                     int32_t* steps, Grad G, Trace TR, cudaStream_t st, int g) {
  vt_note_launch();
  if (s->dtype == VT_F32)
    k_walk<MODE, VT_F32, APP, DIST, HALF><<<g, kWpb * 32, 0, st>>>(S, P, o, d, s->anchor_cell, rgb, T, steps, G, TR);
  else if (s->dtype == VT_F16)
    k_walk<MODE, VT_F16, APP, DIST, HALF><<<g, kWpb * 32, 0, st>>>(S, P, o, d, s->anchor_cell, rgb, T, steps, G, TR);
  else
    k_walk<MODE, VT_BF16, APP, DIST, HALF><<<g, kWpb * 32, 0, st>>>(S, P, o, d, s->anchor_cell, rgb, T, steps, G, TR);
}

template <int MODE>
vt_status launch_walk_kernel(vt_scene* s, const Scene& S, const RP& P, const float* o, const float* d, float* rgb,
                             float* T, int32_t* steps, Grad G, Trace TR, cudaStream_t st) {
  int64_t nt = walk_threads(P);
  if (nt == 0) return VT_OK;
  int g = vt_grid(nt, kWpb * 32, ((int64_t)1 << 31) - 1);
  constexpr int F = MODE == TRACE ? 0 : 1;  // no appearance / distortion variants of the trace
  const bool dist = MODE != TRACE && G.dist != nullptr;
  if (S.nbr_h) {
    // FP16 neighbour offsets: forward (no distortion) and trace only
    if (MODE == BWD || dist) return VT_ERR_UNSUPPORTED;
    constexpr int H = MODE == BWD ? 0 : 1;
    if (P.appearance == 1)
      launch_walk_app<MODE, F, 0, H>(s, S, P, o, d, rgb, T, steps, G, TR, st, g);
    else
      launch_walk_app<MODE, 0, 0, H>(s, S, P, o, d, rgb, T, steps, G, TR, st, g);
  } else if (P.appearance == 1 && dist)
    launch_walk_app<MODE, F, F>(s, S, P, o, d, rgb, T, steps, G, TR, st, g);
  else if (P.appearance == 1)
    launch_walk_app<MODE, F, 0>(s, S, P, o, d, rgb, T, steps, G, TR, st, g);
  else if (dist)
    launch_walk_app<MODE, 0, F>(s, S, P, o, d, rgb, T, steps, G, TR, st, g);
  else
    launch_walk_app<MODE, 0, 0>(s, S, P, o, d, rgb, T, steps, G, TR, st, g);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

// the walk launch, bracketed by the caller's timing events if it gave any
template <int MODE>
vt_status launch_walk(vt_scene* s, const Scene& S, const RP& P, const float* o, const float* d, float* rgb,
                      float* T, int32_t* steps, Grad G, Trace TR, cudaStream_t st, const vt_render_params* p) {
  if (p && p->walk_events[0]) VT_CUDA_TRY(cudaEventRecord((cudaEvent_t)p->walk_events[0], st));
  vt_status r = launch_walk_kernel<MODE>(s, S, P, o, d, rgb, T, steps, G, TR, st);
  if (r != VT_OK) return r;
  if (p && p->walk_events[1]) VT_CUDA_TRY(cudaEventRecord((cudaEvent_t)p->walk_events[1], st));
  return VT_OK;
}

// Gradient scratch of a scene, ready for a backward walk: allocated on first
// use; cell gradients cleared; texel scratch zero everywhere (fully cleared
// after first use or an interrupted call, else only the blocks a scene-order
// backward left holding sums, see vt_render_bwd_scene_order).
__global__ void k_rezero(int64_t n, int RR, float4* g_tex, float4* g_tex_vd, uint8_t* touched) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    if (!touched[i]) continue;  // warp-uniform
    for (int t = lane; t < RR; t += 32) {
      g_tex[i * RR + t] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (g_tex_vd) g_tex_vd[i * RR + t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    if (lane == 0) touched[i] = 0;
  }
}

vt_status prepare_scratch(vt_scene* s, cudaStream_t st) {
  const int64_t RR = (int64_t)s->R * s->R;
  if (!s->g_cell) VT_CUDA_TRY(cudaMalloc(&s->g_cell, s->n * sizeof(float4)));
  if (!s->g_tex) {
    s->g_tex_clean = false;
    VT_CUDA_TRY(cudaMalloc(&s->g_tex, s->n * RR * sizeof(float4)));
  }
  if (s->tex_vd && !s->g_tex_vd) {
    s->g_tex_clean = false;
    VT_CUDA_TRY(cudaMalloc(&s->g_tex_vd, s->n * RR * sizeof(float4)));
  }
  if (!s->g_touched) {
    s->g_tex_clean = false;
    VT_CUDA_TRY(cudaMalloc(&s->g_touched, s->n));
  }
  VT_CUDA_TRY(cudaMemsetAsync(s->g_cell, 0, s->n * sizeof(float4), st));
  if (!s->g_tex_clean) {
    // first use, or a previous call stopped before its permute: clear everything
    VT_CUDA_TRY(cudaMemsetAsync(s->g_tex, 0, s->n * RR * sizeof(float4), st));
    if (s->g_tex_vd) VT_CUDA_TRY(cudaMemsetAsync(s->g_tex_vd, 0, s->n * RR * sizeof(float4), st));
    VT_CUDA_TRY(cudaMemsetAsync(s->g_touched, 0, s->n, st));
  } else if (s->g_held) {
    vt_note_launch();
    k_rezero<<<vt_grid(s->n * 32, 256, 152 * 16), 256, 0, st>>>(s->n, (int)RR, s->g_tex, s->g_tex_vd, s->g_touched);
    VT_CUDA_TRY(cudaGetLastError());
  }
  s->g_tex_clean = false;  // until the call that follows finishes enqueueing
  s->g_held = false;
  return VT_OK;
}

// The backward walk shared by vt_render_bwd and vt_render_bwd_scene_order:
// checks, scratch preparation, start cells and the re-traversal into the
// Morton-ordered scratch (cells it adds texel gradients to are flagged).
vt_status backward_walk(vt_scene* s, int64_t n_rays, const float* o, const float* d, const vt_render_params* p,
                        const float* rgb_out, const float* rgb_residual, const float* dist_out, const float* grad_rgb,
                        const float* grad_dist, cudaStream_t st) {
  if (!s || n_rays < 0 || (n_rays > 0 && (!o || !d || !rgb_out || !grad_rgb))) return VT_ERR_INVALID_ARG;
  if (grad_dist && !dist_out) return VT_ERR_INVALID_ARG;
  if (s->nbr_h) return VT_ERR_UNSUPPORTED;  // FP16-offset scenes are forward only
  RP P;
  vt_status r = make_rp(s, n_rays > 0 ? n_rays : 0, p, P);
  if (r != VT_OK && n_rays > 0) return r;
  if (grad_dist && n_rays > 0 && !(P.t_near >= 0.f)) return VT_ERR_INVALID_ARG;
  r = prepare_scratch(s, st);
  if (r != VT_OK) return r;
  if (n_rays == 0) return VT_OK;
  Scene S = scene_view(s);
  r = anchors(s, S, P, o, st);
  if (r != VT_OK) return r;
  Grad G{s->g_cell, s->g_tex, s->g_tex_vd, rgb_out, rgb_residual, grad_rgb, nullptr, nullptr, s->g_touched};
  if (grad_dist) {
    G.dist = const_cast<float*>(dist_out);  // read only in the backward
    G.gdist = grad_dist;
  }
  return launch_walk<BWD>(s, S, P, o, d, nullptr, nullptr, nullptr, G, Trace{}, st, p);
}

}  // namespace

extern "C" {

vt_status vt_render_fwd(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                        const vt_render_params* p, float* rgb_out, float* T_out, int32_t* steps_out,
                        float* rgb_residual, float* dist_out, void* stream) {
  (void)time;
  if (!s || n_rays < 0 || (n_rays > 0 && (!o || !d || !rgb_out))) return VT_ERR_INVALID_ARG;
  if (n_rays == 0) return VT_OK;
  RP P;
  vt_status r = make_rp(s, n_rays, p, P);
  if (r != VT_OK) return r;
  if (dist_out && !(P.t_near >= 0.f)) return VT_ERR_INVALID_ARG;  // s(t) needs t > -1
  if (dist_out && s->nbr_h) return VT_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  Scene S = scene_view(s);
  r = anchors(s, S, P, o, st);
  if (r != VT_OK) return r;
  Grad G{};
  G.rgb_lo = rgb_residual;
  G.dist = dist_out;
  return launch_walk<FWD>(s, S, P, o, d, rgb_out, T_out, steps_out, G, Trace{}, st, p);
}

vt_status vt_render_bwd(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                        const vt_render_params* p, const float* rgb_out, const float* rgb_residual,
                        const float* dist_out, const float* grad_rgb, const float* grad_dist, float* grad_sites,
                        float* grad_sigma, float* grad_tex, float* grad_tex_vd, void* stream) {
  (void)time;
  if (grad_tex_vd && s && !s->tex_vd) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  vt_status r = backward_walk(s, n_rays, o, d, p, rgb_out, rgb_residual, dist_out, grad_rgb, grad_dist, st);
  if (r != VT_OK) return r;
  // always launched: it also re-zeroes the flagged cells' texel scratch
  launch_grad_out(s->n, (int)(s->R * s->R), s->cell, s->g_cell, s->g_tex, grad_sites, grad_sigma, grad_tex,
                  s->g_tex_vd, grad_tex_vd, s->g_touched, st);
  VT_CUDA_TRY(cudaGetLastError());
  s->g_tex_clean = true;
  s->g_held = false;
  return VT_OK;
}

vt_status vt_render_bwd_scene_order(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                                    const vt_render_params* p, const float* rgb_out, const float* rgb_residual,
                                    const float* dist_out, const float* grad_rgb, const float* grad_dist,
                                    const float** grad_cell, const float** grad_tex, const float** grad_tex_vd,
                                    void* stream) {
  (void)time;
  if (!grad_cell || !grad_tex) return VT_ERR_INVALID_ARG;
  *grad_cell = *grad_tex = nullptr;
  if (grad_tex_vd) *grad_tex_vd = nullptr;
  vt_status r = backward_walk(s, n_rays, o, d, p, rgb_out, rgb_residual, dist_out, grad_rgb, grad_dist,
                              (cudaStream_t)stream);
  if (r != VT_OK) return r;
  // the flagged cells' blocks now hold this call's sums; the next backward
  // call on the scene re-zeroes them first
  s->g_tex_clean = true;
  s->g_held = true;
  *grad_cell = reinterpret_cast<const float*>(s->g_cell);
  *grad_tex = reinterpret_cast<const float*>(s->g_tex);
  if (grad_tex_vd) *grad_tex_vd = reinterpret_cast<const float*>(s->g_tex_vd);
  return VT_OK;
}

vt_status vt_scene_permutation(const vt_scene* s, int32_t* perm, void* stream) {
  if (!s || !perm) return VT_ERR_INVALID_ARG;
  VT_CUDA_TRY(cudaMemcpyAsync(perm, s->perm, s->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return VT_OK;
}

vt_status vt_trace_cells(vt_scene* s, int64_t n_rays, const float* o, const float* d, const vt_render_params* p,
                         int32_t max_cells, int32_t* cells, float* t_exit, int32_t* n_cells, void* stream) {
  if (!s || n_rays < 0 || max_cells < 0 || (n_rays > 0 && (!o || !d || !n_cells || (max_cells > 0 && !cells))))
    return VT_ERR_INVALID_ARG;
  if (n_rays == 0) return VT_OK;
  RP P;
  vt_status r = make_rp(s, n_rays, p, P);
  if (r != VT_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  Scene S = scene_view(s);
  r = anchors(s, S, P, o, st);
  if (r != VT_OK) return r;
  Trace TR{cells, t_exit, n_cells, max_cells};
  return launch_walk<TRACE>(s, S, P, o, d, nullptr, nullptr, nullptr, Grad{}, TR, st, p);
}

// ---------------------------------------------------------------- allocation-free backward
// Backward pass for callers that cannot allocate device memory at the time of
// the call. vt_render_bwd allocates its gradient scratch with cudaMalloc on the
// first call for a scene; this variant instead accumulates into one fixed
// array compiled into the library (VT_STATIC_SCRATCH_BYTES, resident on every
// GPU that loads libvt.so until the process exits). It has no counterpart in
// the paper.
}  // extern "C"

namespace {
constexpr int64_t kStaticScratchFloat4 = VT_STATIC_SCRATCH_BYTES / 16;
static __device__ __align__(256) float4 g_static_scratch[kStaticScratchFloat4];

// Device address of g_static_scratch per device. The host-side name is only a
// stand-in for the symbol, so the address is looked up once per device, with
// that device current, and cached.
std::mutex g_static_mu;
void* g_static_addr[256] = {nullptr};

vt_status static_scratch_addr(float4** out) {
  int dev = -1;
  VT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return VT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    VT_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_static_scratch));
    if (!ptr) return VT_ERR_CUDA;
    g_static_addr[dev] = ptr;
  }
  *out = reinterpret_cast<float4*>(g_static_addr[dev]);
  return VT_OK;
}
}  // namespace

extern "C" {

vt_status vt_render_bwd_static(vt_scene* s, int64_t n_rays, const float* o, const float* d, const float* time,
                               const vt_render_params* p, const float* rgb_out, const float* grad_rgb,
                               float* grad_sites, float* grad_sigma, float* grad_tex, void* stream) {
  (void)time;
  if (!s || n_rays < 0 || (n_rays > 0 && (!o || !d || !rgb_out || !grad_rgb))) return VT_ERR_INVALID_ARG;
  if ((p && p->appearance != 0) || s->nbr_h) return VT_ERR_UNSUPPORTED;
  const int64_t RR = (int64_t)s->R * s->R;
  const int64_t need = s->n * (1 + RR);  // one float4 per cell + one per texel
  if (need > kStaticScratchFloat4) return VT_ERR_CAPACITY;
  RP P;
  vt_status r = make_rp(s, n_rays > 0 ? n_rays : 0, p, P);
  if (r != VT_OK && n_rays > 0) return r;
  float4* base = nullptr;
  r = static_scratch_addr(&base);
  if (r != VT_OK) return r;
  float4* g_cell = base;
  float4* g_tex = base + s->n;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's sums: clear the part this call uses
  VT_CUDA_TRY(cudaMemsetAsync(base, 0, need * sizeof(float4), st));
  Scene S = scene_view(s);
  if (n_rays > 0) {
    r = anchors(s, S, P, o, st);
    if (r != VT_OK) return r;
    Grad G{g_cell, g_tex, nullptr, rgb_out, nullptr, grad_rgb, nullptr, nullptr, nullptr};
    r = launch_walk<BWD>(s, S, P, o, d, nullptr, nullptr, nullptr, G, Trace{}, st, p);
    if (r != VT_OK) return r;
  }
  if (grad_sites || grad_sigma || grad_tex) {
    launch_grad_out(s->n, (int)RR, s->cell, g_cell, g_tex, grad_sites, grad_sigma, grad_tex, nullptr, nullptr,
                    nullptr, st);
    VT_CUDA_TRY(cudaGetLastError());
  }
  return VT_OK;
}

}  // extern "C"
