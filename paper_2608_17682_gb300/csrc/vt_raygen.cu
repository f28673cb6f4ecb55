// vt_raygen.cu -- ray generation for the camera models of Sec. 6.5 (pinhole,
// equidistant fisheye, rolling shutter, thin lens, motion blur), the L2
// photometric loss of the benchmark workloads, the per-pixel average of lens
// and time samples, and the sigma = exp(rho) density map of Sec. 5.4.
#include "vt_internal.cuh"

namespace {

constexpr int kCamsPerLaunch = 64;

struct CamBatch {
  vt_camera cam[kCamsPerLaunch];
  int64_t first[kCamsPerLaunch + 1];  // first ray of each camera
  int n;
};

// SplitMix64 finaliser (Steele, Lea & Flood 2014) used as a counter hash:
// value(seed, c) = mix(seed ^ mix(c)); the top 24 bits give a float in [0,1).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t c) {
  return (float)(mix64(seed ^ mix64(c)) >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ float3 f3(const float* v) { return make_float3(v[0], v[1], v[2]); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 mul(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 unit(float3 a) {
  float inv = 1.0f / sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
  return mul(inv, a);
}

__global__ void k_raygen(CamBatch B, int64_t n_rays, float* __restrict__ O, float* __restrict__ D,
                         float* __restrict__ Tm) {
  for (int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ray < n_rays;
       ray += (int64_t)gridDim.x * blockDim.x) {
    int c = 0;
    while (c + 1 < B.n && ray >= B.first[c + 1]) ++c;
    const vt_camera& cam = B.cam[c];
    int64_t local = ray - B.first[c];
    int S = (cam.kind == VT_CAM_THIN_LENS || cam.kind == VT_CAM_MOTION_BLUR) ? cam.lens_samples : 1;
    int s = (int)(local % S);
    int64_t pix = local / S;
    int y = (int)(pix / cam.w), x = (int)(pix - (int64_t)y * cam.w);
    float3 f = unit(f3(cam.fwd));
    float3 r = unit(cross(f, f3(cam.up)));
    float3 u = cross(r, f);
    float3 o = f3(cam.eye), d;
    float tm = 0.f;
    if (cam.kind == VT_CAM_FISHEYE_EQUIDIST) {
      float px = (x + 0.5f) - 0.5f * cam.w, py = 0.5f * cam.h - (y + 0.5f);
      float rho = sqrtf(px * px + py * py);
      float F = (0.5f * cam.w) / (0.5f * cam.fisheye_fov);
      float th = rho / F;
      float cp = rho > 0.f ? px / rho : 1.f, sp = rho > 0.f ? py / rho : 0.f;
      float st, ct;
      sincosf(th, &st, &ct);
      d = add(mul(ct, f), mul(st, add(mul(cp, r), mul(sp, u))));
    } else {
      float ty = tanf(0.5f * cam.fov_y), tx = ty * (float)cam.w / (float)cam.h;
      float px = (2.f * (x + 0.5f) / cam.w - 1.f) * tx;
      float py = (1.f - 2.f * (y + 0.5f) / cam.h) * ty;
      float3 pd = add(f, add(mul(px, r), mul(py, u)));
      d = pd;
      if (cam.kind == VT_CAM_ROLLING_SHUTTER) {
        tm = (float)y / (float)cam.h;
        o = add(o, mul(tm, f3(cam.rs_velocity)));
      } else if (cam.kind == VT_CAM_THIN_LENS) {
        int m = (int)floorf(sqrtf((float)S) + 0.5f);
        int sx = s % m, sy = s / m;
        uint64_t cnt = (uint64_t)pix * S + s;
        float j1 = uniform24(cam.seed, cnt << 1), j2 = uniform24(cam.seed, (cnt << 1) | 1u);
        float a = 2.f * ((sx + j1) / m) - 1.f, b = 2.f * ((sy + j2) / m) - 1.f;
        // Shirley-Chiu concentric square-to-disk map
        float lx = 0.f, ly = 0.f;
        if (a != 0.f || b != 0.f) {
          float rr, phi;
          const float q = 0.78539816339744831f;  // pi/4
          if (fabsf(a) > fabsf(b)) {
            rr = a;
            phi = q * (b / a);
          } else {
            rr = b;
            phi = 2.f * q - q * (a / b);
          }
          float sp2, cp2;
          sincosf(phi, &sp2, &cp2);
          lx = rr * cp2;
          ly = rr * sp2;
        }
        float3 eye = o;
        o = add(eye, mul(cam.lens_radius, add(mul(lx, r), mul(ly, u))));
        float3 P = add(eye, mul(cam.focus_dist, pd));  // pd.f == 1: depth focus_dist
        d = make_float3(P.x - o.x, P.y - o.y, P.z - o.z);
      } else if (cam.kind == VT_CAM_MOTION_BLUR) {
        // stratified jittered time over the exposure, linear camera motion
        const uint64_t cnt = (uint64_t)pix * S + s;
        tm = ((float)s + uniform24(cam.seed, cnt << 1)) / (float)S;
        o = add(o, mul(tm, f3(cam.rs_velocity)));
      }
    }
    d = unit(d);
    O[3 * ray] = o.x;
    O[3 * ray + 1] = o.y;
    O[3 * ray + 2] = o.z;
    D[3 * ray] = d.x;
    D[3 * ray + 1] = d.y;
    D[3 * ray + 2] = d.z;
    if (Tm) Tm[ray] = tm;
  }
}

__global__ void k_l2(int64_t n3, float inv_n3, const float* __restrict__ C, const float* __restrict__ Y,
                     float* __restrict__ g, float* loss) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
    float r = C[e] - Y[e];
    if (g) g[e] = 2.f * r * inv_n3;
    acc += (double)r * r;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(loss, (float)(t * inv_n3));
  }
}

__global__ void k_avg(int64_t n, int spp, const float* __restrict__ in, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * 3; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e / 3, c = e - p * 3;
    float s = 0.f;
    for (int k = 0; k < spp; ++k) s += in[(p * spp + k) * 3 + c];
    out[e] = s / (float)spp;
  }
}

__global__ void k_avg_bwd(int64_t n, int spp, const float* __restrict__ g, float* __restrict__ out) {
  int64_t total = n * spp * 3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e % 3, ray = e / 3;
    out[e] = g[(ray / spp) * 3 + c] / (float)spp;
  }
}

__global__ void k_exp(int64_t n, const float* x, float* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = expf(x[e]);
}

__global__ void k_mul(int64_t n, const float* a, const float* b, float* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a[e] * b[e];
}

bool camera_ok(const vt_camera& c) {
  if (c.w <= 0 || c.h <= 0 || c.kind < 0 || c.kind > 4) return false;
  if (c.kind == VT_CAM_MOTION_BLUR && c.lens_samples < 1) return false;
  float fl = sqrtf(c.fwd[0] * c.fwd[0] + c.fwd[1] * c.fwd[1] + c.fwd[2] * c.fwd[2]);
  if (!(fl > 0.f)) return false;
  if (c.kind == VT_CAM_THIN_LENS) {
    int m = (int)floorf(sqrtf((float)c.lens_samples) + 0.5f);
    if (c.lens_samples < 1 || m * m != c.lens_samples) return false;
  }
  if (c.kind == VT_CAM_FISHEYE_EQUIDIST && !(c.fisheye_fov > 0.f)) return false;
  return true;
}

}  // namespace

extern "C" {

int64_t vt_camera_n_rays(const vt_camera* c) {
  if (!c) return 0;
  const bool multi = c->kind == VT_CAM_THIN_LENS || c->kind == VT_CAM_MOTION_BLUR;
  return (int64_t)c->w * c->h * (multi ? c->lens_samples : 1);
}

vt_status vt_generate_rays(const vt_camera* cams, int32_t n_cams, float* o, float* d, float* time, void* stream) {
  if (!cams || n_cams < 0 || !o || !d) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t base = 0;
  for (int32_t c0 = 0; c0 < n_cams; c0 += kCamsPerLaunch) {
    CamBatch B;
    B.n = n_cams - c0 < kCamsPerLaunch ? n_cams - c0 : kCamsPerLaunch;
    int64_t acc = 0;
    for (int k = 0; k < B.n; ++k) {
      if (!camera_ok(cams[c0 + k])) return VT_ERR_INVALID_ARG;
      B.cam[k] = cams[c0 + k];
      B.first[k] = acc;
      acc += vt_camera_n_rays(&cams[c0 + k]);
    }
    B.first[B.n] = acc;
    if (acc > 0) {
      vt_note_launch();
      k_raygen<<<vt_grid(acc, 256, 152 * 64), 256, 0, st>>>(B, acc, o + 3 * base, d + 3 * base,
                                                            time ? time + base : nullptr);
    }
    VT_CUDA_TRY(cudaGetLastError());
    base += acc;
  }
  return VT_OK;
}

vt_status vt_l2_loss(int64_t n, const float* rgb, const float* target, float* grad_out, float* loss_out,
                     void* stream) {
  if (n < 0 || (n > 0 && (!rgb || !target)) || !loss_out) return VT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  VT_CUDA_TRY(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
  if (n == 0) return VT_OK;
  vt_note_launch();
  k_l2<<<vt_grid(3 * n, 256, 152 * 8), 256, 0, st>>>(3 * n, 1.0f / (float)(3 * n), rgb, target, grad_out, loss_out);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_average_samples(int64_t n_pixels, int32_t spp, const float* rgb_rays, float* rgb_px, void* stream) {
  if (n_pixels < 0 || spp < 1 || (n_pixels > 0 && (!rgb_rays || !rgb_px))) return VT_ERR_INVALID_ARG;
  if (n_pixels == 0) return VT_OK;
  vt_note_launch();
  k_avg<<<vt_grid(3 * n_pixels, 256, 152 * 64), 256, 0, (cudaStream_t)stream>>>(n_pixels, spp, rgb_rays, rgb_px);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_average_samples_bwd(int64_t n_pixels, int32_t spp, const float* grad_px, float* grad_rays,
                                 void* stream) {
  if (n_pixels < 0 || spp < 1 || (n_pixels > 0 && (!grad_px || !grad_rays))) return VT_ERR_INVALID_ARG;
  if (n_pixels == 0) return VT_OK;
  vt_note_launch();
  k_avg_bwd<<<vt_grid(3 * n_pixels * spp, 256, 152 * 64), 256, 0, (cudaStream_t)stream>>>(n_pixels, spp, grad_px,
                                                                                           grad_rays);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_sigma_from_rho(int64_t n, const float* rho, float* sigma, void* stream) {
  if (n < 0 || (n > 0 && (!rho || !sigma))) return VT_ERR_INVALID_ARG;
  if (n == 0) return VT_OK;
  vt_note_launch();
  k_exp<<<vt_grid(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(n, rho, sigma);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

vt_status vt_sigma_from_rho_bwd(int64_t n, const float* sigma, const float* grad_sigma, float* grad_rho,
                                void* stream) {
  if (n < 0 || (n > 0 && (!sigma || !grad_sigma || !grad_rho))) return VT_ERR_INVALID_ARG;
  if (n == 0) return VT_OK;
  vt_note_launch();
  k_mul<<<vt_grid(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(n, grad_sigma, sigma, grad_rho);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

}  // extern "C"
