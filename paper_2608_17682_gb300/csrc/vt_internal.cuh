// vt_internal.cuh -- internal layout of a scene and helpers shared by the
// translation units of libvt.so (never installed, never seen by callers).
//
// Device layout of a scene (all arrays in Morton order of the sites):
//   cell [N]    32-byte record {x, y, z, sigma, csr begin, csr end, user id,
//               nmax}: one sector holds everything a walk step needs about a
//               cell; nmax (float bits) = max over its neighbours of |s_j - s_i|
//   nbr  [E]    float4 {n_x, n_y, n_z, int bits of j}: the offset
//               n = s_j - s_i (each component rounded to FP32) to neighbour j,
//               stored beside the CSR entry so the exit test needs no second load
//   tex  [N*R*R] RGBA texel: float4 (FP32) or 4 x 16-bit (FP16 / BF16)
//   perm [N]    Morton index -> user id,  inv [N] user id -> Morton index
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "vt.h"

#define VT_MAX_ANCHORS 64

// error bits recorded on the device (scene->d_err[0])
#define VT_EBIT_MAX_STEPS 1u
#define VT_EBIT_CAPACITY 2u
#define VT_EBIT_BAD_RAY 4u

struct __align__(32) vt_cell {
  float x, y, z, sigma;
  int beg, end, uid, pad;
};

struct vt_scene {
  int64_t n = 0;
  int64_t E = 0;
  int32_t R = 0;
  int32_t dtype = VT_F32;
  vt_cell* cell = nullptr;
  float4* nbr = nullptr;
  uint2* nbr_h = nullptr;  // optional FP16 offsets {x,y | z,0} (VT_SCENE_HALF_OFFSETS)
  void* tex = nullptr;
  void* tex_vd = nullptr;  // view-dependent texture (appearance 1), same layout as tex
  int32_t* perm = nullptr;
  int32_t* inv = nullptr;
  // kernel-detected errors [0], FP64 recheck counter [1]
  unsigned long long* d_err = nullptr;
  // anchors of the start-cell search
  unsigned long long* anchor_key = nullptr;
  int32_t* anchor_cell = nullptr;
  // backward scratch: per-cell {dL/ds_x, dL/ds_y, dL/ds_z, dL/dsigma}, per-texel RGBA
  float4* g_cell = nullptr;
  float4* g_tex = nullptr;
  float4* g_tex_vd = nullptr;
  // cells whose texel scratch holds sums (set by the backward walk, cleared
  // by the gradient permute, which also re-zeroes those cells' scratch);
  // g_tex_clean: the texel scratch is zero outside the flagged cells
  uint8_t* g_touched = nullptr;
  bool g_tex_clean = false;
  // g_held: the flagged cells' blocks hold the sums of a scene-order backward
  // (vt_render_bwd_scene_order) that the caller may still read
  bool g_held = false;
};

// Kernels this library has launched since the process started (all devices
// and threads), read with vt_kernel_launches(); every launch site adds one.
extern std::atomic<unsigned long long> g_vt_launches;
static inline void vt_note_launch() { g_vt_launches.fetch_add(1, std::memory_order_relaxed); }

static inline size_t vt_texel_bytes(int32_t dtype) { return dtype == VT_F32 ? 16 : 8; }

#define VT_CUDA_TRY(expr)                     \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) {                  \
      if (e_ == cudaErrorMemoryAllocation) {  \
        cudaGetLastError();                   \
        return VT_ERR_OOM;                    \
      }                                       \
      return VT_ERR_CUDA;                     \
    }                                         \
  } while (0)

static inline int vt_grid(int64_t n, int block, int64_t cap = 1 << 30) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}
