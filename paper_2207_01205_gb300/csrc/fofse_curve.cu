// Error of the extrapolation over the iterations: for every block and every
// iteration count nu, the squared error over B of the model of Eq. 1 built
// from the first nu entries of the selection trace (DFT pairs, or the DCT-II
// basis for plans that use it) (the quantity behind the
// quality-over-iterations curves of Fig. 4 and Fig. 5).  The model's values
// at B are accumulated iteration by iteration, one pixel per thread (up to
// four for 32 x 32 blocks), from the trace's FP32 coefficients; each
// iteration's squared error is reduced per warp (shuffles) and then per block
// through shared memory.  The trace is staged through shared memory in chunks.
#include "fofse_internal.h"

namespace fofse {
namespace {

constexpr int kCurveThreads = 256;
constexpr int kCurveWarps = kCurveThreads / 32;
constexpr int kCurveChunk = 256;  // trace entries staged per pass
constexpr int kCurvePix = 4;      // pixels per thread (block side <= 32)

__global__ void __launch_bounds__(kCurveThreads) fofse_error_curve_kernel(const __grid_constant__ CurveArgs a) {
  __shared__ float4 s_c[kCurveChunk];  // (c_re, c_im, multiplicity, packed u1 | u2 << 16)
  __shared__ float s_part[kCurveWarps][kCurveChunk];
  const PlanDev& P = a.plan;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = P.block, br = P.border, T = P.T, iters = P.iters;
  const float2* syn = P.tab.syn_f32;
  const float2* dcs = P.tab.dct_cos_ff;  // DCT basis: cos(2 pi p / (4T)), p = u (2m+1) mod 4T
  const bool dct = P.basis == FOFSE_BASIS_DCT;
  for (int blk = blockIdx.x; blk < a.n_blocks; blk += gridDim.x) {
    const fofse_block bd = a.blocks[blk];
    if (bd.plan != a.plan_index) continue;
    float acc[kCurvePix], tru[kCurvePix];
    int mm[kCurvePix], nn[kCurvePix];
    bool val[kCurvePix];
#pragma unroll
    for (int k = 0; k < kCurvePix; ++k) {
      const int pix = tid + k * kCurveThreads;
      const int bm = pix / b, bn = pix - bm * b;
      const int fy = bd.y + bm, fx = bd.x + bn;
      // samples of B outside the frame (a broken contract) are left out
      val[k] = pix < b * b && fy >= 0 && fy < a.height && fx >= 0 && fx < a.width;
      mm[k] = br + bm;
      nn[k] = br + bn;
      acc[k] = 0.f;
      tru[k] = val[k] ? a.truth[(size_t)fy * a.pitch + fx] : 0.f;
    }
    const fofse_trace_entry* tr = a.trace + (size_t)blk * a.trace_stride;
    float* out = a.sse + (size_t)blk * a.trace_stride;
    for (int i0 = 0; i0 < iters; i0 += kCurveChunk) {
      const int nc = min(kCurveChunk, iters - i0);
      __syncthreads();  // the previous chunk's s_c and s_part are consumed
      for (int j = tid; j < nc; j += kCurveThreads) {
        const fofse_trace_entry e = tr[i0 + j];
        const int u1 = e.u1 & (T - 1), u2 = e.u2 & (T - 1);
        const bool sc = dct || (((u1 & (T / 2 - 1)) == 0) && ((u2 & (T / 2 - 1)) == 0));
        s_c[j] = make_float4(e.dc_re, e.dc_im, sc ? 1.f : 2.f, __int_as_float(u1 | (u2 << 16)));
      }
      __syncthreads();
      for (int j = 0; j < nc; ++j) {
        const float4 c = s_c[j];
        const int pk = __float_as_int(c.w);
        const int u1 = pk & 0xffff, u2 = pk >> 16;
        float err = 0.f;
#pragma unroll
        for (int k = 0; k < kCurvePix; ++k) {
          if (val[k]) {
            if (dct) {
              const float c1 = __ldg(&dcs[(u1 * (2 * mm[k] + 1)) & (4 * T - 1)]).x;
              const float c2 = __ldg(&dcs[(u2 * (2 * nn[k] + 1)) & (4 * T - 1)]).x;
              acc[k] += c.x * (c1 * c2);
            } else {
              const float2 cs = __ldg(&syn[(u1 * mm[k] + u2 * nn[k]) & (T - 1)]);
              acc[k] += c.z * (c.x * cs.x - c.y * cs.y);
            }
            const float d = fminf(fmaxf(acc[k], 0.f), 255.f) - tru[k];
            err = __fmaf_rn(d, d, err);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) err += __shfl_xor_sync(0xffffffffu, err, o);
        if (lane == 0) s_part[warp][j] = err;
      }
      __syncthreads();
      for (int j = tid; j < nc; j += kCurveThreads) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kCurveWarps; ++w) s += s_part[w][j];
        out[i0 + j] = s;
      }
    }
    for (int j = iters + tid; j < a.trace_stride; j += kCurveThreads) out[j] = 0.f;
  }
}

}  // namespace

cudaError_t launch_error_curve(const CurveArgs& a, cudaStream_t s) {
  if (a.plan.block * a.plan.block > kCurveThreads * kCurvePix) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int grid = sms * 8;
  if (grid > a.n_blocks) grid = a.n_blocks;
  if (grid < 1) return cudaSuccess;
  fofse_error_curve_kernel<<<grid, kCurveThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fofse
