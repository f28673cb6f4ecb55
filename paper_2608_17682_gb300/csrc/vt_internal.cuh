// vt_internal.cuh -- internal layout of a scene and helpers shared by the
// translation units of libvt.so (never installed, never seen by callers).
//
// Device layout of a scene (all arrays in Morton order of the sites):
//   site [N]    float4 {x, y, z, sigma}
//   meta [N]    int4   {csr begin, csr end, sigma bits, user id}
//   nbr  [E]    float4 {x_j, y_j, z_j, int bits of j}   neighbour records
//               inlined beside the CSR so the exit test needs no second load
//   tex  [N*R*R] RGBA texel: float4 (FP32) or 4 x 16-bit (FP16 / BF16)
//   perm [N]    Morton index -> user id,  inv [N] user id -> Morton index
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vt.h"

#define VT_MAX_ANCHORS 64

// error bits recorded on the device (scene->d_err[0])
#define VT_EBIT_MAX_STEPS 1u
#define VT_EBIT_CAPACITY 2u
#define VT_EBIT_BAD_RAY 4u

struct vt_scene {
  int64_t n = 0;
  int64_t E = 0;
  int32_t R = 0;
  int32_t dtype = VT_F32;
  float4* site = nullptr;
  int4* meta = nullptr;
  float4* nbr = nullptr;
  void* tex = nullptr;
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
};

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
