// vt_scene.cu -- scene preparation (the paper's one-time preprocessing,
// Sec. 5.6): input validation, Morton reordering of the cells, CSR remap with
// neighbour positions inlined beside the adjacency, RGB -> RGBA texel packing
// in FP32 / FP16 / BF16 storage.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "vt_internal.cuh"

namespace {

// ------------------------------------------------------------------ validation
// bits of the validation word
enum : unsigned {
  BAD_SITE = 1,
  BAD_SIGMA = 2,
  BAD_OFFSETS = 4,
  BAD_INDEX = 8,
  SELF_LOOP = 16,
  ASYMMETRIC = 32,
  DUPLICATE = 64
};

__global__ void k_validate_nodes(int64_t n, const float* __restrict__ sites, const float* __restrict__ sigma,
                                 const int64_t* __restrict__ off, int64_t E, unsigned* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned b = 0;
    if (sites) {
      float x = sites[3 * i], y = sites[3 * i + 1], z = sites[3 * i + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) b |= BAD_SITE;
    }
    if (sigma) {
      float s = sigma[i];
      if (!isfinite(s) || !(s >= 0.f)) b |= BAD_SIGMA;
    }
    if (off) {
      int64_t a = off[i], c = off[i + 1];
      if (a < 0 || c < a || c > E) b |= BAD_OFFSETS;
    }
    if (b) atomicOr(bad, b);
  }
}

// one thread per CSR row: range, self loop, duplicate and symmetry checks
__global__ void k_validate_rows(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                                unsigned* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned b = 0;
    int64_t a = off[i], c = off[i + 1];
    for (int64_t p = a; p < c; ++p) {
      int32_t j = idx[p];
      if (j < 0 || j >= n) {
        b |= BAD_INDEX;
        continue;
      }
      if (j == i) b |= SELF_LOOP;
      for (int64_t q = a; q < p; ++q)
        if (idx[q] == j) b |= DUPLICATE;
      bool found = false;
      for (int64_t q = off[j]; q < off[j + 1]; ++q)
        if (idx[q] == (int32_t)i) {
          found = true;
          break;
        }
      if (!found) b |= ASYMMETRIC;
    }
    if (b) atomicOr(bad, b);
  }
}

// ------------------------------------------------------------------ Morton order
__global__ void k_bbox(int64_t n, const float* __restrict__ sites, float* __restrict__ part) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      float v = sites[3 * i + k];
      lo[k] = fminf(lo[k], v);
      hi[k] = fmaxf(hi[k], v);
    }
  __shared__ float s[6][256];
  for (int k = 0; k < 3; ++k) {
    s[k][threadIdx.x] = lo[k];
    s[3 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = fminf(s[k][threadIdx.x], s[k][threadIdx.x + w]);
        s[3 + k][threadIdx.x] = fmaxf(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) part[6 * blockIdx.x + k] = s[k][0];
}

__device__ __forceinline__ uint64_t spread21(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__global__ void k_morton(int64_t n, const float* __restrict__ sites, float3 lo, float3 scale,
                         uint64_t* __restrict__ code, int32_t* __restrict__ ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float m = 2097151.f;  // 2^21 - 1
    float q[3] = {(sites[3 * i] - lo.x) * scale.x, (sites[3 * i + 1] - lo.y) * scale.y,
                  (sites[3 * i + 2] - lo.z) * scale.z};
    uint64_t c = 0;
    for (int k = 0; k < 3; ++k) {
      float v = fminf(fmaxf(q[k] * m, 0.f), m);
      c |= spread21((uint64_t)v) << (2 - k);
    }
    code[i] = c;
    ids[i] = (int32_t)i;
  }
}

__global__ void k_inverse(int64_t n, const int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inv[perm[i]] = (int32_t)i;
}

__global__ void k_degree(int64_t n, const int32_t* __restrict__ perm, const int64_t* __restrict__ off,
                         int32_t* __restrict__ deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = perm[i];
    deg[i] = (int32_t)(off[u + 1] - off[u]);
  }
}

// cell records (position, sigma, CSR range, user id) in Morton order
__global__ void k_fill_cells(int64_t n, const int32_t* __restrict__ perm, const float* __restrict__ sites,
                             const float* __restrict__ sigma, const int32_t* __restrict__ beg,
                             const int32_t* __restrict__ deg, vt_cell* __restrict__ cell, int keep_csr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = perm[i];
    vt_cell c = cell[i];
    if (sites) {
      c.x = sites[3 * (int64_t)u];
      c.y = sites[3 * (int64_t)u + 1];
      c.z = sites[3 * (int64_t)u + 2];
    }
    if (sigma) c.sigma = sigma[u];
    if (!keep_csr) {
      c.beg = beg[i];
      c.end = beg[i] + deg[i];
      c.uid = u;
      c.pad = 0;
    }
    cell[i] = c;
  }
}

// neighbour records {s_j - s_i, j} in the user's CSR order of each row
__global__ void k_fill_nbr(int64_t n, const vt_cell* __restrict__ cell, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ idx, const int32_t* __restrict__ inv,
                           float4* __restrict__ nbr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const vt_cell c = cell[i];
    int64_t ub = off[c.uid];
    for (int p = c.beg; p < c.end; ++p) {
      int32_t j = inv[idx[ub + (p - c.beg)]];
      const vt_cell cj = cell[j];
      nbr[p] = make_float4(__fsub_rn(cj.x, c.x), __fsub_rn(cj.y, c.y), __fsub_rn(cj.z, c.z), __int_as_float(j));
    }
  }
}

// FP16 copies of the offsets (round to nearest even); flags an offset that
// does not fit FP16's range
__global__ void k_fill_nbr_h(int64_t E, const float4* __restrict__ nbr, uint2* __restrict__ nbr_h,
                             unsigned long long* err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
    const float4 q = nbr[p];
    if (!(fabsf(q.x) < 65504.f && fabsf(q.y) < 65504.f && fabsf(q.z) < 65504.f)) atomicOr(err, 1ull);
    const __half2 xy = __floats2half2_rn(q.x, q.y);
    const __half2 z0 = __floats2half2_rn(q.z, 0.f);
    nbr_h[p] = make_uint2(*reinterpret_cast<const unsigned int*>(&xy), *reinterpret_cast<const unsigned int*>(&z0));
  }
}

vt_status fill_half_offsets(vt_scene* s, cudaStream_t st) {
  if (!s->nbr_h || s->E == 0) return VT_OK;
  unsigned long long* bad = nullptr;
  VT_CUDA_TRY(cudaMalloc(&bad, sizeof(unsigned long long)));
  unsigned long long hbad = 0;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    vt_note_launch();
    k_fill_nbr_h<<<vt_grid(s->E, 256, 152 * 32), 256, 0, st>>>(s->E, s->nbr, s->nbr_h, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(bad);
  if (e != cudaSuccess) return VT_ERR_CUDA;
  return hbad ? VT_ERR_INVALID_ARG : VT_OK;
}

// largest neighbour offset |n| of each cell (bound for the grazing test)
__global__ void k_cell_nmax(int64_t n, vt_cell* __restrict__ cell, const float4* __restrict__ nbr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = cell[i].beg, e = cell[i].end;
    float m = 0.f;
    for (int p = b; p < e; ++p) {
      const float4 q = nbr[p];
      m = fmaxf(m, sqrtf(q.x * q.x + q.y * q.y + q.z * q.z));
    }
    cell[i].pad = __float_as_int(m * 1.0001f);
  }
}

// texel packing: [N,R,R,3] FP32 user order -> Morton-ordered RGBA in storage dtype
template <int DT>
__global__ void k_pack_tex(int64_t n, int32_t RR, const int32_t* __restrict__ perm, const float* __restrict__ tex,
                           void* __restrict__ out) {
  int64_t total = n * RR;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / RR, t = e - i * RR;
    const float* src = tex + ((int64_t)perm[i] * RR + t) * 3;
    float r = src[0], g = src[1], b = src[2];
    if (DT == VT_F32) {
      reinterpret_cast<float4*>(out)[e] = make_float4(r, g, b, 0.f);
    } else if (DT == VT_F16) {
      __half h[4] = {__float2half_rn(r), __float2half_rn(g), __float2half_rn(b), __float2half_rn(0.f)};
      reinterpret_cast<uint2*>(out)[e] = *reinterpret_cast<uint2*>(h);
    } else {
      __nv_bfloat16 h[4] = {__float2bfloat16_rn(r), __float2bfloat16_rn(g), __float2bfloat16_rn(b),
                            __float2bfloat16_rn(0.f)};
      reinterpret_cast<uint2*>(out)[e] = *reinterpret_cast<uint2*>(h);
    }
  }
}

vt_status pack_tex(vt_scene* s, const float* tex, cudaStream_t st, void* dst = nullptr) {
  int64_t total = s->n * (int64_t)s->R * s->R;
  int g = vt_grid(total, 256, 152 * 64);
  void* out = dst ? dst : s->tex;
  vt_note_launch();
  if (s->dtype == VT_F32)
    k_pack_tex<VT_F32><<<g, 256, 0, st>>>(s->n, s->R * s->R, s->perm, tex, out);
  else if (s->dtype == VT_F16)
    k_pack_tex<VT_F16><<<g, 256, 0, st>>>(s->n, s->R * s->R, s->perm, tex, out);
  else
    k_pack_tex<VT_BF16><<<g, 256, 0, st>>>(s->n, s->R * s->R, s->perm, tex, out);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

template <class T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

vt_status validate(int64_t n, const float* sites, const float* sigma, const int64_t* off, const int32_t* idx,
                   int64_t E, cudaStream_t st) {
  unsigned* bad = nullptr;
  VT_CUDA_TRY(cudaMalloc(&bad, sizeof(unsigned)));
  unsigned hbad = 0;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
  int g = vt_grid(n, 256, 152 * 32);
  if (e == cudaSuccess) {
    vt_note_launch();
    k_validate_nodes<<<g, 256, 0, st>>>(n, sites, sigma, off, E, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && hbad == 0 && off && (idx || E == 0)) {
    vt_note_launch();
    k_validate_rows<<<g, 256, 0, st>>>(n, off, idx, bad);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(bad);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VT_ERR_OOM : VT_ERR_CUDA;
  return hbad ? VT_ERR_INVALID_ARG : VT_OK;
}

void free_scene(vt_scene* s) {
  if (!s) return;
  cudaFree(s->cell);
  cudaFree(s->nbr);
  cudaFree(s->nbr_h);
  cudaFree(s->tex);
  cudaFree(s->tex_vd);
  cudaFree(s->perm);
  cudaFree(s->inv);
  cudaFree(s->d_err);
  cudaFree(s->anchor_key);
  cudaFree(s->anchor_cell);
  cudaFree(s->g_cell);
  cudaFree(s->g_tex);
  cudaFree(s->g_tex_vd);
  cudaFree(s->g_touched);
  delete s;
}

vt_status create_impl(const vt_scene_desc* dsc, cudaStream_t st, vt_scene* s) {
  const int64_t n = dsc->n_sites;
  int64_t E = 0;
  VT_CUDA_TRY(cudaMemcpyAsync(&E, dsc->adj_offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  int64_t off0 = -1;
  VT_CUDA_TRY(cudaMemcpyAsync(&off0, dsc->adj_offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  VT_CUDA_TRY(cudaStreamSynchronize(st));
  if (off0 != 0 || E < 0 || E >= (int64_t)INT32_MAX || (E > 0 && !dsc->adj_indices)) return VT_ERR_INVALID_ARG;
  vt_status v = validate(n, dsc->sites, dsc->sigma, dsc->adj_offsets, dsc->adj_indices, E, st);
  if (v != VT_OK) return v;
  s->n = n;
  s->E = E;
  s->R = dsc->tex_res;
  s->dtype = dsc->tex_dtype;
  const int64_t RR = (int64_t)s->R * s->R;
  VT_CUDA_TRY(dmalloc(&s->cell, n));
  VT_CUDA_TRY(dmalloc(&s->nbr, E > 0 ? E : 1));
  if (dsc->flags & VT_SCENE_HALF_OFFSETS) VT_CUDA_TRY(dmalloc(&s->nbr_h, E > 0 ? E : 1));
  VT_CUDA_TRY(cudaMalloc(&s->tex, n * RR * vt_texel_bytes(s->dtype) + 16));
  if (dsc->tex_vd) VT_CUDA_TRY(cudaMalloc(&s->tex_vd, n * RR * vt_texel_bytes(s->dtype) + 16));
  VT_CUDA_TRY(dmalloc(&s->perm, n));
  VT_CUDA_TRY(dmalloc(&s->inv, n));
  VT_CUDA_TRY(dmalloc(&s->d_err, 4));
  VT_CUDA_TRY(dmalloc(&s->anchor_key, VT_MAX_ANCHORS));
  VT_CUDA_TRY(dmalloc(&s->anchor_cell, VT_MAX_ANCHORS));
  VT_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, 4 * sizeof(unsigned long long), st));
  VT_CUDA_TRY(cudaMemsetAsync(s->cell, 0, n * sizeof(vt_cell), st));

  // bounding box
  const int nb = 256;
  float* part = nullptr;
  VT_CUDA_TRY(cudaMalloc(&part, nb * 6 * sizeof(float)));
  vt_note_launch();
  k_bbox<<<nb, 256, 0, st>>>(n, dsc->sites, part);
  float hp[nb * 6];
  cudaError_t e = cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(part);
  VT_CUDA_TRY(e);
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], hp[6 * b + k]);
      hi[k] = fmaxf(hi[k], hp[6 * b + 3 + k]);
    }
  float3 lo3 = make_float3(lo[0], lo[1], lo[2]);
  float ext[3];
  for (int k = 0; k < 3; ++k) ext[k] = hi[k] > lo[k] ? 1.f / (hi[k] - lo[k]) : 0.f;
  float3 sc3 = make_float3(ext[0], ext[1], ext[2]);

  // Morton codes, stable radix sort of (code, user id)
  uint64_t *code = nullptr, *code2 = nullptr;
  int32_t *ids = nullptr, *deg = nullptr, *beg = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0, scan_bytes = 0;
  vt_status rs = VT_OK;
  do {
    if (cudaMalloc(&code, n * sizeof(uint64_t)) != cudaSuccess || cudaMalloc(&code2, n * sizeof(uint64_t)) ||
        cudaMalloc(&ids, n * sizeof(int32_t)) || cudaMalloc(&deg, n * sizeof(int32_t)) ||
        cudaMalloc(&beg, n * sizeof(int32_t))) {
      rs = VT_ERR_OOM;
      break;
    }
    int g = vt_grid(n, 256, 152 * 32);
    vt_note_launch();
    k_morton<<<g, 256, 0, st>>>(n, dsc->sites, lo3, sc3, code, ids);
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, code, code2, ids, s->perm, (int)n, 0, 63, st);
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, deg, beg, (int)n, st);
    if (scan_bytes > tmp_bytes) tmp_bytes = scan_bytes;
    if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) {
      rs = VT_ERR_OOM;
      break;
    }
    if (dsc->flags & VT_SCENE_KEEP_ORDER) {
      if (cudaMemcpyAsync(s->perm, ids, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        rs = VT_ERR_CUDA;
        break;
      }
    } else if (cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, code, code2, ids, s->perm, (int)n, 0, 63, st) !=
               cudaSuccess) {
      rs = VT_ERR_CUDA;
      break;
    }
    vt_note_launch();
    k_inverse<<<g, 256, 0, st>>>(n, s->perm, s->inv);
    vt_note_launch();
    k_degree<<<g, 256, 0, st>>>(n, s->perm, dsc->adj_offsets, deg);
    if (cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, deg, beg, (int)n, st) != cudaSuccess) {
      rs = VT_ERR_CUDA;
      break;
    }
    vt_note_launch();
    k_fill_cells<<<g, 256, 0, st>>>(n, s->perm, dsc->sites, dsc->sigma, beg, deg, s->cell, 0);
    vt_note_launch();
    k_fill_nbr<<<g, 256, 0, st>>>(n, s->cell, dsc->adj_offsets, dsc->adj_indices, s->inv, s->nbr);
    vt_note_launch();
    k_cell_nmax<<<g, 256, 0, st>>>(n, s->cell, s->nbr);
    rs = fill_half_offsets(s, st);
    if (rs != VT_OK) break;
    rs = pack_tex(s, dsc->tex, st);
    if (rs != VT_OK) break;
    if (dsc->tex_vd) {
      rs = pack_tex(s, dsc->tex_vd, st, s->tex_vd);
      if (rs != VT_OK) break;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) rs = VT_ERR_CUDA;
  } while (0);
  cudaFree(code);
  cudaFree(code2);
  cudaFree(ids);
  cudaFree(deg);
  cudaFree(beg);
  cudaFree(tmp);
  return rs;
}

__global__ void k_refresh_nbr(int64_t n, const vt_cell* __restrict__ cell, float4* __restrict__ nbr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const vt_cell c = cell[i];
    for (int p = c.beg; p < c.end; ++p) {
      float4 q = nbr[p];
      const vt_cell cj = cell[__float_as_int(q.w)];
      nbr[p] = make_float4(__fsub_rn(cj.x, c.x), __fsub_rn(cj.y, c.y), __fsub_rn(cj.z, c.z), q.w);
    }
  }
}

}  // namespace

extern "C" {

void vt_render_params_default(vt_render_params* p) {
  if (!p) return;
  *p = vt_render_params{};
  p->t_near = 0.f;
  p->t_far = 20.f;
  p->use_clip_box = 0;
  for (int k = 0; k < 3; ++k) {
    p->clip_lo[k] = 0.f;
    p->clip_hi[k] = 1.f;
    p->bg[k] = 1.f;
  }
  p->T_eps = 1e-4f;
  p->skip_weight = 0.f;
  p->img_w = p->img_h = p->n_images = 0;
  p->max_steps = 0;
}

vt_status vt_scene_create(const vt_scene_desc* dsc, void* stream, vt_scene** out) {
  if (!out) return VT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dsc || dsc->n_sites < 1 || dsc->n_sites >= (int64_t)INT32_MAX || dsc->tex_res < 2 ||
      dsc->tex_res > 64 || !dsc->sites || !dsc->sigma || !dsc->tex || !dsc->adj_offsets)
    return VT_ERR_INVALID_ARG;
  if (dsc->tex_dtype != VT_F32 && dsc->tex_dtype != VT_F16 && dsc->tex_dtype != VT_BF16) return VT_ERR_INVALID_ARG;
  if ((__int128)dsc->n_sites * dsc->tex_res * dsc->tex_res >= ((__int128)1 << 40)) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  vt_scene* s = new vt_scene();
  vt_status r = create_impl(dsc, st, s);
  if (r != VT_OK) {
    cudaStreamSynchronize(st);
    free_scene(s);
    return r;
  }
  *out = s;
  return VT_OK;
}

vt_status vt_scene_update(vt_scene* s, const float* sites, const float* sigma, const float* tex,
                          const float* tex_vd, void* stream) {
  if (!s || (tex_vd && !s->tex_vd)) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (sites || sigma) {
    vt_status v = validate(s->n, sites, sigma, nullptr, nullptr, 0, st);
    if (v != VT_OK) return v;
    int g = vt_grid(s->n, 256, 152 * 32);
    vt_note_launch();
    k_fill_cells<<<g, 256, 0, st>>>(s->n, s->perm, sites, sigma, nullptr, nullptr, s->cell, 1);
    if (sites) {
      vt_note_launch();
      k_refresh_nbr<<<g, 256, 0, st>>>(s->n, s->cell, s->nbr);
      vt_note_launch();
      k_cell_nmax<<<g, 256, 0, st>>>(s->n, s->cell, s->nbr);
    }
    VT_CUDA_TRY(cudaGetLastError());
    if (sites) {
      vt_status h = fill_half_offsets(s, st);
      if (h != VT_OK) return h;
    }
  }
  if (tex) {
    vt_status v = pack_tex(s, tex, st);
    if (v != VT_OK) return v;
  }
  if (tex_vd) {
    vt_status v = pack_tex(s, tex_vd, st, s->tex_vd);
    if (v != VT_OK) return v;
  }
  return VT_OK;
}

void vt_scene_destroy(vt_scene* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  free_scene(s);
}

vt_status vt_scene_info(const vt_scene* s, int64_t* n_sites, int32_t* tex_res, int32_t* tex_dtype,
                        int64_t* n_edges) {
  if (!s) return VT_ERR_INVALID_ARG;
  if (n_sites) *n_sites = s->n;
  if (tex_res) *tex_res = s->R;
  if (tex_dtype) *tex_dtype = s->dtype;
  if (n_edges) *n_edges = s->E;
  return VT_OK;
}

vt_status vt_scene_get_error(vt_scene* s, void* stream, int64_t* n_fp64) {
  if (!s) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[4] = {0, 0, 0, 0};
  VT_CUDA_TRY(cudaStreamSynchronize(st));
  VT_CUDA_TRY(cudaMemcpy(h, s->d_err, sizeof(h), cudaMemcpyDeviceToHost));
  VT_CUDA_TRY(cudaMemset(s->d_err, 0, sizeof(h)));
  if (n_fp64) *n_fp64 = (int64_t)h[1];
  if (h[0] & VT_EBIT_MAX_STEPS) return VT_ERR_MAX_STEPS;
  if (h[0] & VT_EBIT_CAPACITY) return VT_ERR_CAPACITY;
  if (h[0] & VT_EBIT_BAD_RAY) return VT_ERR_INVALID_ARG;
  return VT_OK;
}

const char* vt_status_str(vt_status s) {
  switch (s) {
    case VT_OK: return "VT_OK";
    case VT_ERR_INVALID_ARG: return "VT_ERR_INVALID_ARG";
    case VT_ERR_CUDA: return "VT_ERR_CUDA";
    case VT_ERR_OOM: return "VT_ERR_OOM";
    case VT_ERR_MAX_STEPS: return "VT_ERR_MAX_STEPS";
    case VT_ERR_CAPACITY: return "VT_ERR_CAPACITY";
    case VT_ERR_UNSUPPORTED: return "VT_ERR_UNSUPPORTED";
  }
  return "VT_ERR_UNKNOWN";
}

}  // extern "C"
