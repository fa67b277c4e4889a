// Backward (adjoint) FOFSE kernel: gradients of a loss l(B_hat) with respect
// to the support samples, rho and gamma, with the selection path frozen.
//
// With the path u_1..u_I fixed, the transform-domain recursion of the
// forward pass (paper Sec. 2, Eq. 2-3 and Eq. 14 in the DFT domain) reads
//   a_i  = R0[u_i] - sum_{j<i} ( c_j W[u_i - u_j] + s_j conj(c_j) W[u_i + u_j] )
//   c_i  = gamma a_i / W[0]          (real part only for self-conjugate u_i)
//   B_hat = sum_i (1 + s_i) Re(c_i phi_{u_i})  on B   (Eq. 1)
// with R0 = DFT(w f), W = DFT(w).  Its reverse sweep, per CTA (one block):
//   1. one packed FFT of w + j e (e = dl/dB_hat on B) gives W (kept in shared
//      memory) and E = DFT(e); cbar_i = (1 + s_i) E[u_i];
//   2. for i = I..1: abar_i = gamma/W0 cbar_i and, for j < i,
//      cbar_j -= abar_i conj(W[u_i-u_j]) + s_j conj(abar_i) W[u_i+u_j]
//      (a triangular solve, in tiles of 32 iterations);
//      gammabar = sum_i Re(conj(cbar_i) c_i)/gamma, W0bar = -sum_i Re(conj(cbar_i) c_i)/W0;
//   3. back to the samples without a W-adjoint grid: summing the pair terms
//      over j < i gives the model before iteration i (g_{i-1} = sum_{j<i}
//      (1 + s_j) Re(c_j phi_{u_j})), so on every sample of A
//        xbar[m,n] = sum_i Re(abar_i phi_{u_i}[m,n])            (dl/dx, x = w f)
//        wbar[m,n] = sum_i (f - g_{i-1})[m,n] Re(abar_i phi_{u_i}[m,n]) + W0bar,
//      accumulated in one pass over the trace while the residual f - g is
//      rebuilt sample by sample (no atomics, deterministic; wbar comes from
//      the residual, not from the difference of two large terms);
//   4. fbar = w xbar on A (atomically added into the frame gradient, blocks
//      overlap), rhobar = sum_A wbar w dist / rho (Eq. 15).
// FP32 arithmetic throughout (the gradients' tolerance is relative 1e-3).
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <set>
#include <utility>

#include "fofse_arith.cuh"
#include "fofse_fft.cuh"
#include "fofse_internal.h"

namespace fofse {
namespace {

using A = ArF32;
using Cx = ArF32::C;

template <int T> __device__ __forceinline__ bool self_conj(int u1, int u2) {
  return ((u1 & (T / 2 - 1)) == 0) && ((u2 & (T / 2 - 1)) == 0);
}

template <int T, int NT>
__global__ void __launch_bounds__(NT) fofse_backward_kernel(const __grid_constant__ BwdArgs args) {
  constexpr int LOGT = ilog2c(T), T2 = 2 * T, NW = NT / 32;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const PlanDev& P = args.plan;
  const int iters = P.iters;
  float* Z = reinterpret_cast<float*>(smem);  // FFT buffer, then W
  float2* syn = reinterpret_cast<float2*>(Z + T * T2);  // (cos, sin)(2 pi p / T)
  Cx* tw = reinterpret_cast<Cx*>(syn + T);
  int* tu = reinterpret_cast<int*>(tw + T / 2);         // u1 << 16 | u2
  float2* tc = reinterpret_cast<float2*>(tu + ((iters + 1) & ~1));  // c_i
  float2* tg = tc + iters;                              // cbar_i
  float2* ta = tg + iters;                              // abar_i
  double* red = reinterpret_cast<double*>(ta + iters);  // 4 NW

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int blk = blockIdx.x;
  const fofse_block bd = args.blocks[blk];
  if (bd.plan != args.plan_index) return;
  const float w0 = args.w0[blk];
  if (!(w0 > 0.f)) return;  // block without support (or not finite): zero gradient
  const int b = P.block, br = P.border, Ls = P.Ls;
  const int ly0 = bd.y - br, lx0 = bd.x - br;
  const float gamma = (float)P.gamma;

  // ---- trace, cleared gradient grids, packed input z = w + j e ---------------
  for (int i = tid; i < iters; i += NT) {
    const fofse_trace_entry e = args.trace[(size_t)blk * args.trace_stride + i];
    tu[i] = ((int)(uint16_t)e.u1 << 16) | (int)(uint16_t)e.u2;
    tc[i] = make_float2(e.dc_re, e.dc_im);
  }
  for (int e = tid; e < T; e += NT) syn[e] = P.tab.syn_f32[e];
  for (int e = tid; e < T / 2; e += NT) tw[e] = {P.tab.tw_f32[e].x, P.tab.tw_f32[e].y};
  for (int e = tid; e < T * T; e += NT) {
    const int r = e >> LOGT, c = e & (T - 1);
    const int m = __brev(r) >> (32 - LOGT), n = __brev(c) >> (32 - LOGT);
    float wv = 0.f, ev = 0.f;
    if (m < Ls && n < Ls) {
      const bool inB = m >= br && m < br + b && n >= br && n < br + b;
      bool inS = true;
      if (P.support == FOFSE_SUPPORT_CAUSAL_L)
        inS = (m < br) ? (n < br + b) : (m < br + b ? n < br : false);
      const int fy = ly0 + m, fx = lx0 + n;
      const bool in = fy >= 0 && fy < args.height && fx >= 0 && fx < args.width;
      if (in && !inB && inS && args.avail[(size_t)fy * args.pitch + fx]) wv = P.tab.w_f32[m * Ls + n];
      if (inB) ev = args.grad_blocks[(size_t)blk * args.grad_stride + (m - br) * args.grad_ld + (n - br)];
    }
    Z[r * T2 + c] = wv;
    Z[r * T2 + T + c] = ev;
  }
  __syncthreads();
  fft2d_dit<A, T, NT, false>(Z, tw, Ls, T);

  // ---- cbar_i = (1 + s_i) E[u_i], E = (Z[u] - conj Z[-u]) / (2j) ---------------
  for (int i = tid; i < iters; i += NT) {
    const int u1 = tu[i] >> 16, u2 = tu[i] & 0xffff;
    const int m1 = (T - u1) & (T - 1), m2 = (T - u2) & (T - 1);
    const Cx a = A::load(Z, u1 * T2 + u2, T), mm = A::load(Z, m1 * T2 + m2, T);
    const float dre = a.re - mm.re, dim = a.im + mm.im;  // d = a - conj(mm)
    const float mult = self_conj<T>(u1, u2) ? 0.5f : 1.f;   // (1 + s) / 2
    tg[i] = make_float2(mult * dim, -mult * dre);
  }
  __syncthreads();
  // ---- W[k] = (Z[k] + conj Z[-k]) / 2 in place --------------------------------
  for (int e = tid; e < T * T; e += NT) {
    const int k1 = e >> LOGT, k2 = e & (T - 1);
    const int m1 = (T - k1) & (T - 1), m2 = (T - k2) & (T - 1);
    const int me = m1 * T + m2;
    if (e <= me) {
      const Cx a = A::load(Z, k1 * T2 + k2, T), mm = A::load(Z, m1 * T2 + m2, T);
      const Cx wv = A::half(A::add(a, A::conj(mm)));
      A::store(Z, k1 * T2 + k2, T, wv);
      if (me != e) A::store(Z, m1 * T2 + m2, T, A::conj(wv));
    }
  }
  __syncthreads();

  // ---- reverse sweep of the triangular recurrence -----------------------------
  // (a) cbar / abar: a lower-triangular solve, sequential in i (descending).
  //     It runs in tiles of 32 iterations: warp 0 resolves a tile's diagonal
  //     part warp-synchronously (lane = iteration within the tile), then every
  //     thread applies the tile's abar to the earlier iterations.  Two barriers
  //     per tile instead of one per iteration.
  const float g_w0 = gamma / w0;
  for (int hi = iters; hi > 0; hi -= 32) {
    const int lo = hi > 32 ? hi - 32 : 0;
    if (warp == 0) {
      const int j = lo + lane;
      const bool act = j < hi;
      const int uj = act ? tu[j] : 0;
      const int uj1 = uj >> 16, uj2 = uj & 0xffff;
      const bool sj = !self_conj<T>(uj1, uj2);
      float2 g = act ? tg[j] : make_float2(0.f, 0.f);
      float2 ab = make_float2(0.f, 0.f);
      for (int i = hi - 1; i >= lo; --i) {
        const int li = i - lo;
        const int ui = __shfl_sync(0xffffffffu, uj, li);
        const float gr_i = __shfl_sync(0xffffffffu, g.x, li);
        const float gi_i = __shfl_sync(0xffffffffu, g.y, li);
        const int ui1 = ui >> 16, ui2 = ui & 0xffff;
        const bool si = !self_conj<T>(ui1, ui2);
        const float abr = g_w0 * gr_i, abi = si ? g_w0 * gi_i : 0.f;
        if (lane == li) ab = make_float2(abr, abi);
        if (act && lane < li) {
          const int dm = ((ui1 - uj1) & (T - 1)) * T2 + ((ui2 - uj2) & (T - 1));
          const Cx Wm = A::load(Z, dm, T);
          float gr = abr * Wm.re + abi * Wm.im;
          float gi = abi * Wm.re - abr * Wm.im;
          if (sj) {
            const int dp = ((ui1 + uj1) & (T - 1)) * T2 + ((ui2 + uj2) & (T - 1));
            const Cx Wp = A::load(Z, dp, T);
            gr += abr * Wp.re + abi * Wp.im;
            gi += abr * Wp.im - abi * Wp.re;
          }
          g.x -= gr;
          g.y -= gi;
        }
      }
      if (act) {
        tg[j] = g;
        ta[j] = ab;
      }
    }
    __syncthreads();
    for (int j = tid; j < lo; j += NT) {
      const int uj = tu[j];
      const int uj1 = uj >> 16, uj2 = uj & 0xffff;
      const bool sj = !self_conj<T>(uj1, uj2);
      float gr = 0.f, gi = 0.f;
      for (int i = lo; i < hi; ++i) {
        const int ui = tu[i];
        const int ui1 = ui >> 16, ui2 = ui & 0xffff;
        const float2 ab = ta[i];
        const int dm = ((ui1 - uj1) & (T - 1)) * T2 + ((ui2 - uj2) & (T - 1));
        const Cx Wm = A::load(Z, dm, T);
        gr += ab.x * Wm.re + ab.y * Wm.im;
        gi += ab.y * Wm.re - ab.x * Wm.im;
        if (sj) {
          const int dp = ((ui1 + uj1) & (T - 1)) * T2 + ((ui2 + uj2) & (T - 1));
          const Cx Wp = A::load(Z, dp, T);
          gr += ab.x * Wp.re + ab.y * Wp.im;
          gi += ab.x * Wp.im - ab.y * Wp.re;
        }
      }
      float2 g = tg[j];
      g.x -= gr;
      g.y -= gi;
      tg[j] = g;
    }
    __syncthreads();
  }
  // (b) gammabar and W0bar from the final cbar; (1 + s_i) c_i for the model rebuild
  float dot_acc = 0.f;
  for (int i = tid; i < iters; i += NT) {
    const int ui = tu[i];
    const bool si = !self_conj<T>(ui >> 16, ui & 0xffff);
    const float2 cb = tg[i], ci = tc[i];
    dot_acc += cb.x * ci.x + (si ? cb.y * ci.y : 0.f);
    tg[i] = si ? make_float2(2.f * ci.x, 2.f * ci.y) : ci;  // cbar no longer needed
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
  if (lane == 0) red[warp] = dot_acc;
  __syncthreads();
  double dot = 0.0;
  for (int w = 0; w < NW; ++w) dot += red[w];
  const float w0bar = (float)(-dot / w0);  // W0 = W[0] = sum of w
  if (tid == 0 && args.grad_rho_gamma) atomicAdd(&args.grad_rho_gamma[1], (float)(dot / gamma));
  __syncthreads();  // red is reused below

  // ---- chain to the samples, rho and gamma ------------------------------------
  // B_hat is homogeneous of degree 0 in w (scaling w scales R0, W and W[0]
  // alike), so sum_A wbar w = 0 and rhobar = sum_A wbar w (dist - dbar) / rho
  // for any dbar.  With dbar = sum w dist / sum w the FP32 error components of
  // wbar that are uniform over A cancel; the four sums are accumulated in FP64.
  const float c0 = br + (b - 1) * 0.5f;
  double s_wwd = 0.0, s_ww = 0.0, s_wd = 0.0, s_w = 0.0;
  for (int e = tid; e < Ls * Ls; e += NT) {
    const int m = e / Ls, n = e - m * Ls;
    const bool inB = m >= br && m < br + b && n >= br && n < br + b;
    bool inS = true;
    if (P.support == FOFSE_SUPPORT_CAUSAL_L)
      inS = (m < br) ? (n < br + b) : (m < br + b ? n < br : false);
    const int fy = ly0 + m, fx = lx0 + n;
    const bool in = fy >= 0 && fy < args.height && fx >= 0 && fx < args.width;
    if (!in || inB || !inS) continue;
    const size_t fi = (size_t)fy * args.pitch + fx;
    if (!args.avail[fi]) continue;
    // rebuild the residual f - g_{i-1} and accumulate xbar, wbar along the trace
    const float f = args.frame[fi];
    float r = f, xbar = 0.f, wb = 0.f;
    for (int i = 0; i < iters; ++i) {
      const int ui = tu[i];
      const int ph = ((ui >> 16) * m + (ui & 0xffff) * n) & (T - 1);
      const float2 cs = syn[ph];
      const float2 ab = ta[i], cm = tg[i];
      const float q = ab.x * cs.x - ab.y * cs.y;  // Re(abar_i phi_{u_i})
      xbar += q;
      wb = fmaf(r, q, wb);
      r -= cm.x * cs.x - cm.y * cs.y;             // (1 + s_i) Re(c_i phi_{u_i})
    }
    const float w = P.tab.w_f32[m * Ls + n];
    if (args.grad_frame) atomicAdd(&args.grad_frame[fi], w * xbar);
    const float wbar = wb + w0bar;
    const float dm = m - c0, dn = n - c0;
    const double d = (double)sqrtf(dm * dm + dn * dn);
    const double ww = (double)wbar * (double)w;
    s_wwd += ww * d;
    s_ww += ww;
    s_wd += (double)w * d;
    s_w += (double)w;
  }
  if (args.grad_rho_gamma) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s_wwd += __shfl_xor_sync(0xffffffffu, s_wwd, o);
      s_ww += __shfl_xor_sync(0xffffffffu, s_ww, o);
      s_wd += __shfl_xor_sync(0xffffffffu, s_wd, o);
      s_w += __shfl_xor_sync(0xffffffffu, s_w, o);
    }
    if (lane == 0) {
      red[4 * warp + 0] = s_wwd;
      red[4 * warp + 1] = s_ww;
      red[4 * warp + 2] = s_wd;
      red[4 * warp + 3] = s_w;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0, bb = 0, c = 0, d = 0;
      for (int w = 0; w < NW; ++w) {
        a += red[4 * w];
        bb += red[4 * w + 1];
        c += red[4 * w + 2];
        d += red[4 * w + 3];
      }
      const double dbar = d > 0 ? c / d : 0.0;
      atomicAdd(&args.grad_rho_gamma[0], (float)((a - dbar * bb) / (double)P.rho));
    }
  }
}

template <int T, int NT> size_t bwd_smem(int iters) {
  size_t off = 128 + sizeof(float) * T * 2 * T + sizeof(float2) * T + sizeof(Cx) * (T / 2);
  off += sizeof(int) * ((iters + 1) & ~1) + 3 * sizeof(float2) * iters + 4 * sizeof(double) * (NT / 32);
  return off;
}

template <int T, int NT> cudaError_t launch_bwd(const BwdArgs& a, cudaStream_t s) {
  const size_t sm = bwd_smem<T, NT>(a.plan.iters);
  auto kern = fofse_backward_kernel<T, NT>;
  {  // the kernel's shared-memory limit (one per device) only grows: a smaller
     // request never lowers it below a size launched before
    static std::mutex mu;
    static std::map<int, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto lim = limit.find(dev);
    if (lim == limit.end() || lim->second < sm) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      limit[dev] = sm;
    }
  }
  kern<<<a.n_blocks, NT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward(const BwdArgs& a, cudaStream_t s) {
  if (a.plan.precision == FOFSE_FP64_VALIDATE) return cudaErrorNotSupported;
  if (a.plan.T == 128) return launch_bwd<128, 512>(a, s);
  if (a.plan.T == 64) return launch_bwd<64, 256>(a, s);
  if (a.plan.T == 32) return launch_bwd<32, 128>(a, s);
  return cudaErrorNotSupported;
}

}  // namespace fofse
