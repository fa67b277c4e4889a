// Measurement probes for the rooflines of the kernels (no counterpart in the
// paper): the shared-memory load bandwidth and the FP32 and FP64 FMA rates of
// this GPU, each from a kernel that does nothing else.  The caller times the
// launch (CUDA events) and divides the work reported here by the time and the
// sampled SM clock.  Built into libfofse_probes.so, not into the product
// library (include/fofse_probes.h).
#include <cuda_runtime.h>

#include "../../include/fofse_probes.h"

namespace fofse {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeSmemFloats = 8192;  // 32 KB
constexpr int kProbeUnroll = 8;

__device__ __forceinline__ float4 lds128(unsigned addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

// Every thread reads 16 B per load, consecutive lanes consecutive 16 B (no
// bank conflicts), kProbeUnroll loads per round, `rounds` rounds; the sum goes
// to sink[] so that nothing is removed.
__global__ void __launch_bounds__(kProbeThreads) fofse_smem_probe_kernel(float* sink, int rounds) {
  __shared__ __align__(16) float s[kProbeSmemFloats];
  for (int i = threadIdx.x; i < kProbeSmemFloats; i += kProbeThreads) s[i] = (float)(i & 15);
  __syncthreads();
  const unsigned base = (unsigned)__cvta_generic_to_shared(s);
  const unsigned mask = kProbeSmemFloats * 4 - 1;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  unsigned off = threadIdx.x * 16u;
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) {
      const float4 v = lds128(base + ((off + k * 4096u) & mask));
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    off += 512u;
  }
  if (acc.x + acc.y + acc.z + acc.w == -1.f) sink[blockIdx.x * kProbeThreads + threadIdx.x] = acc.x;
}

// Eight independent FMA chains per thread, `rounds` rounds of eight FMAs each.
__global__ void __launch_bounds__(kProbeThreads) fofse_fma_probe_kernel(float* sink, int rounds, float a, float b) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k);
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __fmaf_rn(x[k], a, b);
  }
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += x[k];
  if (t == -1.f) sink[blockIdx.x * kProbeThreads + threadIdx.x] = t;
}

// The same with FP64 FMAs (the pipe of the video-volume kernel).
__global__ void __launch_bounds__(kProbeThreads) fofse_dfma_probe_kernel(double* sink, int rounds, double a,
                                                                         double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k);
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += x[k];
  if (t == -1.0) sink[blockIdx.x * kProbeThreads + threadIdx.x] = t;
}

}  // namespace
}  // namespace fofse

using namespace fofse;

extern "C" {

fofse_status fofse_probe_smem(int ctas, int rounds, float* d_sink, double* bytes, void* stream) {
  if (ctas < 1 || rounds < 1 || !d_sink || !bytes) return FOFSE_E_ARG;
  fofse_smem_probe_kernel<<<ctas, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(d_sink, rounds);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return FOFSE_E_CUDA;
  *bytes = (double)ctas * kProbeThreads * rounds * kProbeUnroll * 16.0;
  return FOFSE_OK;
}

fofse_status fofse_probe_fma(int ctas, int rounds, float* d_sink, double* fmas, void* stream) {
  if (ctas < 1 || rounds < 1 || !d_sink || !fmas) return FOFSE_E_ARG;
  fofse_fma_probe_kernel<<<ctas, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      d_sink, rounds, 0.999f, 1e-3f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return FOFSE_E_CUDA;
  *fmas = (double)ctas * kProbeThreads * rounds * 8.0;
  return FOFSE_OK;
}

fofse_status fofse_probe_dfma(int ctas, int rounds, double* d_sink, double* fmas, void* stream) {
  if (ctas < 1 || rounds < 1 || !d_sink || !fmas) return FOFSE_E_ARG;
  fofse_dfma_probe_kernel<<<ctas, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      d_sink, rounds, 0.999, 1e-3);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return FOFSE_E_CUDA;
  *fmas = (double)ctas * kProbeThreads * rounds * 8.0;
  return FOFSE_OK;
}

}  // extern "C"
