// vt_probe.cu -- launch counter and a streaming-read bandwidth probe.
//
// The probe reads a device buffer `reps` times through the L2 (loads marked
// cache-global, so they bypass L1): when the buffer fits in the 129 MB L2 and
// `reps` is large, the time measures the L2 read bandwidth that the walk
// kernels' demand bytes are served from; for buffers larger than L2 it
// measures HBM read bandwidth.
#include "vt_internal.cuh"

std::atomic<unsigned long long> g_vt_launches{0};

namespace {

// Each thread keeps four independent 16-byte loads in flight per iteration.
__global__ void __launch_bounds__(512) k_stream_read(const float4* __restrict__ a, int64_t n, int reps,
                                                     float* sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float acc = 0.f;
  for (int r = 0; r < reps; ++r) {
    int64_t i = i0;
    for (; i + 3 * stride < n; i += 4 * stride) {
      const float4 v0 = __ldcg(a + i), v1 = __ldcg(a + i + stride), v2 = __ldcg(a + i + 2 * stride),
                   v3 = __ldcg(a + i + 3 * stride);
      acc += (v0.x + v1.y) + (v2.z + v3.w);
    }
    for (; i < n; i += stride) acc += __ldcg(a + i).x;
  }
  if (acc == 1234.5f) *sink = acc;  // data-dependent store: the loads cannot be dropped
}

}  // namespace

extern "C" {

uint64_t vt_kernel_launches(void) { return g_vt_launches.load(std::memory_order_relaxed); }

vt_status vt_stream_read(const void* buf, int64_t bytes, int32_t reps, float* sink, void* stream) {
  if (!buf || !sink || bytes <= 0 || (bytes & 15) || ((uintptr_t)buf & 15) || reps < 1) return VT_ERR_INVALID_ARG;
  const int64_t n = bytes / 16;
  int dev = 0, sms = 0;
  VT_CUDA_TRY(cudaGetDevice(&dev));
  VT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // four 512-thread blocks per SM, fewer if the buffer is small
  const int64_t want = (n + 4 * 512 - 1) / (4 * 512);
  const int g = (int)(want < 4LL * sms ? (want < 1 ? 1 : want) : 4LL * sms);
  vt_note_launch();
  k_stream_read<<<g, 512, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4*>(buf), n, reps, sink);
  VT_CUDA_TRY(cudaGetLastError());
  return VT_OK;
}

}  // extern "C"
