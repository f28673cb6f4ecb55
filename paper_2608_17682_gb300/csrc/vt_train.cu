// vt_train.cu -- the pieces of a training step around the renderer (Sec. 5.5
// and the training details of the appendix): stratified ray sampling from
// pre-generated camera rays, the Smooth-L1 photometric loss, the two texture
// regularisers of Eq. 5 (L_vd and L_mean), and an Adam update.
#include "vt_internal.cuh"

namespace {

// SplitMix64 counter hash (Steele, Lea & Flood 2014); top 24 bits -> [0,1)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform24(uint64_t seed, uint64_t c) {
  return (double)(mix64(seed ^ mix64(c)) >> 40) * (1.0 / 16777216.0);
}

// one sample per stratum [k N/B, (k+1) N/B): sorted, distinct indices, each
// pool entry drawn with probability B/N
__global__ void k_sample(int64_t n_pool, int64_t n, uint64_t seed, const float* __restrict__ o_pool,
                         const float* __restrict__ d_pool, const float* __restrict__ y_pool, float* __restrict__ o,
                         float* __restrict__ d, float* __restrict__ y, int64_t* __restrict__ idx_out) {
  const double stride = (double)n_pool / (double)n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = (int64_t)(((double)k + uniform24(seed, (uint64_t)k)) * stride);
    const int64_t hi = (int64_t)((double)(k + 1) * stride);
    if (i >= hi) i = hi - 1;  // rounding at the top of the stratum
    if (i >= n_pool) i = n_pool - 1;
    if (i < 0) i = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o[3 * k + c] = o_pool[3 * i + c];
      d[3 * k + c] = d_pool[3 * i + c];
      if (y) y[3 * k + c] = y_pool[3 * i + c];
    }
    if (idx_out) idx_out[k] = i;
  }
}

__device__ __forceinline__ double block_sum(double acc) {
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
  return t;
}

// Smooth-L1 (Huber with transition beta) averaged over all n3 channels
__global__ void k_smooth_l1(int64_t n3, float inv_n3, float beta, const float* __restrict__ C,
                            const float* __restrict__ Y, float* __restrict__ g, float* loss) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
    const float r = C[e] - Y[e], a = fabsf(r);
    float l, dl;
    if (a < beta) {
      l = 0.5f * r * r / beta;
      dl = r / beta;
    } else {
      l = a - 0.5f * beta;
      dl = r > 0.f ? 1.f : -1.f;
    }
    if (g) g[e] = dl * inv_n3;
    acc += (double)l;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(loss, (float)(t * inv_n3));
}

// One warp per cell. L_vd = 1/(N R^2) sum_i |T_i^vd|^2 and
// L_mean = 1/(N R^2) sum_{i,u} |T_{i,u} - mean_v T_{i,v}|^2, weighted by
// lam_vd, lam_mean; gradients are ADDED to grad_vi / grad_vd.
__global__ void k_tex_reg(int64_t n, int RR, float lam_vd, float lam_mean, const float* __restrict__ tvi,
                          const float* __restrict__ tvd, float* __restrict__ gvi, float* __restrict__ gvd, float* loss) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float scale = 1.f / ((float)n * (float)RR);
  double acc = 0.0;
  for (int64_t i = warp0; i < n; i += warps) {
    const int64_t base = i * RR * 3;
    if (tvi && lam_mean != 0.f) {
      float m0 = 0.f, m1 = 0.f, m2 = 0.f;
      for (int u = lane; u < RR; u += 32) {
        m0 += tvi[base + 3 * u];
        m1 += tvi[base + 3 * u + 1];
        m2 += tvi[base + 3 * u + 2];
      }
      for (int off = 16; off > 0; off >>= 1) {
        m0 += __shfl_xor_sync(0xffffffffu, m0, off);
        m1 += __shfl_xor_sync(0xffffffffu, m1, off);
        m2 += __shfl_xor_sync(0xffffffffu, m2, off);
      }
      m0 /= (float)RR;
      m1 /= (float)RR;
      m2 /= (float)RR;
      for (int u = lane; u < RR; u += 32) {
        const float r0 = tvi[base + 3 * u] - m0, r1 = tvi[base + 3 * u + 1] - m1, r2 = tvi[base + 3 * u + 2] - m2;
        acc += (double)lam_mean * scale * (r0 * r0 + r1 * r1 + r2 * r2);
        // the mean's own derivative sums to zero over u
        if (gvi) {
          gvi[base + 3 * u] += 2.f * lam_mean * scale * r0;
          gvi[base + 3 * u + 1] += 2.f * lam_mean * scale * r1;
          gvi[base + 3 * u + 2] += 2.f * lam_mean * scale * r2;
        }
      }
    }
    if (tvd && lam_vd != 0.f) {
      for (int e = lane; e < RR * 3; e += 32) {
        const float t = tvd[base + e];
        acc += (double)lam_vd * scale * t * t;
        if (gvd) gvd[base + e] += 2.f * lam_vd * scale * t;
      }
    }
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(loss, (float)t);
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Adam on a user-order texture map from scene-order gradients, with the
// map's regulariser of Eq. 5 fused in. One warp per scene cell k (user cell
// u = perm[k]): the warp reads the cell's R^2 x 3 parameters, forms the
// regulariser gradient from them (reg 0: L_mean = 1/(N R^2) sum |T_u -
// mean_v T_v|^2; reg 1: L_vd = 1/(N R^2) sum |T|^2), adds the RGB part of the
// scene-order RGBA render gradient, and updates parameter and moments in place
// (no update when lr == 0; the regulariser's loss is still added to *loss).
__global__ void k_adam_tex_scene(int64_t n, int RR, const int32_t* __restrict__ perm,
                                 const float4* __restrict__ gsc, float* __restrict__ tex, float* __restrict__ m,
                                 float* __restrict__ v, int reg, float lam, float lr, float b1, float b2, float eps,
                                 float c1, float c2, float* loss) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float scale = 1.f / ((float)n * (float)RR);
  double acc = 0.0;
  for (int64_t k = warp0; k < n; k += warps) {
    const int32_t uk = perm[k];
    if (uk < 0 || (int64_t)uk >= n) continue;  // not a permutation entry: skipped (warp-uniform)
    const int64_t base = (int64_t)uk * RR * 3;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
    if (reg == 0 && lam != 0.f) {
      for (int t = lane; t < RR; t += 32) {
        m0 += tex[base + 3 * t];
        m1 += tex[base + 3 * t + 1];
        m2 += tex[base + 3 * t + 2];
      }
      for (int off = 16; off > 0; off >>= 1) {
        m0 += __shfl_xor_sync(0xffffffffu, m0, off);
        m1 += __shfl_xor_sync(0xffffffffu, m1, off);
        m2 += __shfl_xor_sync(0xffffffffu, m2, off);
      }
      m0 /= (float)RR;
      m1 /= (float)RR;
      m2 /= (float)RR;
    }
    for (int e = lane; e < RR * 3; e += 32) {
      const int t = e / 3, c = e - 3 * t;
      const float p = tex[base + e];
      float rg = 0.f;
      if (lam != 0.f) {
        const float r = reg == 0 ? p - (c == 0 ? m0 : (c == 1 ? m1 : m2)) : p;
        acc += (double)lam * scale * r * r;
        rg = 2.f * lam * scale * r;
      }
      if (lr != 0.f) {
        const float4 gq = gsc[k * RR + t];
        const float gi = (c == 0 ? gq.x : (c == 1 ? gq.y : gq.z)) + rg;
        const float mi = b1 * m[base + e] + (1.f - b1) * gi;
        const float vi = b2 * v[base + e] + (1.f - b2) * gi * gi;
        m[base + e] = mi;
        v[base + e] = vi;
        tex[base + e] = p - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
      }
    }
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, (float)t);
}

// Adam on user-order sites and log-densities from the scene-order cell
// gradients {dL/ds, dL/dsigma}: dL/drho = dL/dsigma * sigma (Eq. 4).
__global__ void k_adam_cells_scene(int64_t n, const int32_t* __restrict__ perm, const float4* __restrict__ gc,
                                   float* __restrict__ sites, float* __restrict__ rho, const float* __restrict__ sigma,
                                   float* __restrict__ ms, float* __restrict__ vs, float* __restrict__ mr,
                                   float* __restrict__ vr, float lr_s, float lr_r, float b1, float b2, float eps,
                                   float c1, float c2) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = perm[k];
    if (u < 0 || u >= n) continue;  // not a permutation entry: skipped
    const float4 g = gc[k];
    if (lr_s != 0.f) {
      const float gs[3] = {g.x, g.y, g.z};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int64_t e = 3 * u + a;
        const float mi = b1 * ms[e] + (1.f - b1) * gs[a];
        const float vi = b2 * vs[e] + (1.f - b2) * gs[a] * gs[a];
        ms[e] = mi;
        vs[e] = vi;
        sites[e] -= lr_s * (mi / c1) / (sqrtf(vi / c2) + eps);
      }
    }
    if (lr_r != 0.f) {
      const float gi = g.w * sigma[u];
      const float mi = b1 * mr[u] + (1.f - b1) * gi;
      const float vi = b2 * vr[u] + (1.f - b2) * gi * gi;
      mr[u] = mi;
      vr[u] = vi;
      rho[u] -= lr_r * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
  }
}

bool adam_args_ok(float beta1, float beta2, float eps, int64_t step) {
  return step >= 1 && beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f;
}

}  // namespace

extern "C" {

vt_status vt_sample_rays(int64_t n_pool, const float* o_pool, const float* d_pool, const float* y_pool, int64_t n,
                         uint64_t seed, float* o, float* d, float* y, int64_t* idx_out, void* stream) {
  if (n_pool < 0 || n < 0 || n > n_pool) return VT_ERR_INVALID_ARG;
  if (n == 0) return VT_OK;
  if (!o_pool || !d_pool || !o || !d || (y && !y_pool)) return VT_ERR_INVALID_ARG;
  vt_note_launch();
  k_sample<<<vt_grid(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(n_pool, n, seed, o_pool, d_pool, y_pool, o,
                                                                         d, y, idx_out);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_smooth_l1_loss(int64_t n, const float* rgb, const float* target, float beta, float* grad_out,
                            float* loss_out, void* stream) {
  if (n < 0 || (n > 0 && (!rgb || !target)) || !loss_out || !(beta > 0.f)) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  VT_CUDA_TRY(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
  if (n == 0) return VT_OK;
  vt_note_launch();
  k_smooth_l1<<<vt_grid(3 * n, 256, 152 * 8), 256, 0, st>>>(3 * n, 1.0f / (float)(3 * n), beta, rgb, target,
                                                            grad_out, loss_out);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_texture_regularizers(int64_t n_cells, int32_t tex_res, const float* tex, const float* tex_vd,
                                  float lambda_vd, float lambda_mean, float* grad_tex, float* grad_tex_vd,
                                  float* loss_out, void* stream) {
  if (n_cells < 0 || tex_res < 1 || !loss_out) return VT_ERR_INVALID_ARG;
  if ((lambda_mean != 0.f && !tex) || (lambda_vd != 0.f && !tex_vd)) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  VT_CUDA_TRY(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
  if (n_cells == 0) return VT_OK;
  vt_note_launch();
  k_tex_reg<<<vt_grid(n_cells * 32, 256, 152 * 8), 256, 0, st>>>(n_cells, tex_res * tex_res, lambda_vd, lambda_mean,
                                                                  tex, tex_vd, grad_tex, grad_tex_vd, loss_out);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                       float beta2, float eps, int64_t step, void* stream) {
  if (n < 0 || step < 1 || (n > 0 && (!param || !grad || !m || !v))) return VT_ERR_INVALID_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f)) return VT_ERR_INVALID_ARG;
  if (n == 0) return VT_OK;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  vt_note_launch();
  k_adam<<<vt_grid(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(n, param, grad, m, v, lr, beta1, beta2, eps,
                                                                       c1, c2);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_adam_step_tex_scene_order(int64_t n_cells, int32_t tex_res, const int32_t* perm,
                                      const float* grad_tex_scene, float* tex, float* m, float* v, int32_t regularizer,
                                      float lambda, float lr, float beta1, float beta2, float eps, int64_t step,
                                      float* loss_out, void* stream) {
  if (n_cells < 0 || tex_res < 1 || (regularizer != 0 && regularizer != 1)) return VT_ERR_INVALID_ARG;
  if (!adam_args_ok(beta1, beta2, eps, step)) return VT_ERR_INVALID_ARG;
  if (n_cells > 0 && (!perm || !tex || (lr != 0.f && (!grad_tex_scene || !m || !v)) || (lambda != 0.f && !loss_out)))
    return VT_ERR_INVALID_ARG;
  if (n_cells == 0) return VT_OK;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  vt_note_launch();
  k_adam_tex_scene<<<vt_grid(n_cells * 32, 256, 152 * 8), 256, 0, (cudaStream_t)stream>>>(
      n_cells, tex_res * tex_res, perm, reinterpret_cast<const float4*>(grad_tex_scene), tex, m, v, regularizer, lambda,
      lr, beta1, beta2, eps, c1, c2, loss_out);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_adam_step_cells_scene_order(int64_t n_cells, const int32_t* perm, const float* grad_cell_scene,
                                        float* sites, float* rho, const float* sigma, float* m_sites, float* v_sites,
                                        float* m_rho, float* v_rho, float lr_sites, float lr_rho, float beta1,
                                        float beta2, float eps, int64_t step, void* stream) {
  if (n_cells < 0 || !adam_args_ok(beta1, beta2, eps, step)) return VT_ERR_INVALID_ARG;
  if (n_cells > 0 && (!perm || !grad_cell_scene || (lr_sites != 0.f && (!sites || !m_sites || !v_sites)) ||
                      (lr_rho != 0.f && (!rho || !sigma || !m_rho || !v_rho))))
    return VT_ERR_INVALID_ARG;
  if (n_cells == 0) return VT_OK;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  vt_note_launch();
  k_adam_cells_scene<<<vt_grid(n_cells, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(
      n_cells, perm, reinterpret_cast<const float4*>(grad_cell_scene), sites, rho, sigma, m_sites, v_sites, m_rho,
      v_rho, lr_sites, lr_rho, beta1, beta2, eps, c1, c2);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

}  // extern "C"
