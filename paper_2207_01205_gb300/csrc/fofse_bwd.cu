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

template <int T, int NT, bool SPLIT>
__global__ void __launch_bounds__(NT) fofse_backward_kernel(const __grid_constant__ BwdArgs args) {
  constexpr int LOGT = ilog2c(T), T2 = 2 * T, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];  // 16-byte slots, no TMA
  unsigned char* smem = smem_raw;
  const PlanDev& P = args.plan;
  const int iters = P.iters;
  // split form: no synthesis table and no copy of c_i (the sample kernel
  // has them), so that six blocks fit on an SM
  float* Z = reinterpret_cast<float*>(smem);  // FFT buffer, then W
  float2* syn = reinterpret_cast<float2*>(Z + T * T2);  // (cos, sin)(2 pi p / T)
  int* tu = reinterpret_cast<int*>(syn + (SPLIT ? 0 : T));  // u1 << 16 | u2
  float2* tc = reinterpret_cast<float2*>(tu + ((iters + 1) & ~1));  // c_i
  float2* tg = tc + (SPLIT ? 0 : iters);                // cbar_i
  float2* ta = tg + iters;                              // abar_i
  double* red = reinterpret_cast<double*>(ta + iters);  // 4 NW (NW when split)
  const Cx* tw = reinterpret_cast<const Cx*>(P.tab.tw_f32);  // read through L1

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int blk = blockIdx.x;
  const fofse_block bd = args.blocks[blk];
  if (bd.plan != args.plan_index) return;
  const float w0 = args.w0[blk];
  if (!(w0 > 0.f)) return;  // block without support (or not finite): zero gradient
  const int b = P.block, br = P.border, Ls = P.Ls;
  const int ly0 = bd.y - br, lx0 = bd.x - br;
  const float gamma = P.rho_gamma_dev ? P.rho_gamma_dev[1] : (float)P.gamma;

  // ---- trace, cleared gradient grids, packed input z = w + j e ---------------
  for (int i = tid; i < iters; i += NT) {
    const fofse_trace_entry e = args.trace[(size_t)blk * args.trace_stride + i];
    tu[i] = ((int)(uint16_t)e.u1 << 16) | (int)(uint16_t)e.u2;
    if (!SPLIT) tc[i] = make_float2(e.dc_re, e.dc_im);
  }
  if (!SPLIT)
    for (int e = tid; e < T; e += NT) syn[e] = P.tab.syn_f32[e];
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
    float2 ci;
    if (SPLIT) {
      const fofse_trace_entry e = args.trace[(size_t)blk * args.trace_stride + i];
      ci = make_float2(e.dc_re, e.dc_im);
    } else {
      ci = tc[i];
    }
    const float2 cb = tg[i];
    dot_acc += cb.x * ci.x + (si ? cb.y * ci.y : 0.f);
    if (!SPLIT) tg[i] = si ? make_float2(2.f * ci.x, 2.f * ci.y) : ci;  // cbar no longer needed
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
  if (lane == 0) red[warp] = dot_acc;
  __syncthreads();
  double dot = 0.0;
  for (int w = 0; w < NW; ++w) dot += red[w];
  const float w0bar = (float)(-dot / w0);  // W0 = W[0] = sum of w
  if (tid == 0 && args.grad_rho_gamma) atomicAdd(&args.grad_rho_gamma[1], (float)(dot / gamma));
  if constexpr (SPLIT) {  // the sample kernel takes it from here
    for (int i = tid; i < iters; i += NT) args.abar[(size_t)blk * args.trace_stride + i] = ta[i];
    if (tid == 0) args.w0bar[blk] = w0bar;
    return;
  }
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
      atomicAdd(&args.grad_rho_gamma[0], (float)((a - dbar * bb) / (double)(P.rho_gamma_dev ? P.rho_gamma_dev[0] : P.rho)));
    }
  }
}

// Number of support positions of a block (A's shape inside L, B excluded) and
// the position of rank k in L coordinates.  Full support: the rows above B,
// the rows of B without B, the rows below B.  Causal L shape: the rows above B
// up to its right edge, then the samples left of B in B's rows.
__device__ __forceinline__ int support_positions(int support, int Ls, int b, int br) {
  return support == FOFSE_SUPPORT_CAUSAL_L ? br * (br + b) + b * br : Ls * Ls - b * b;
}
__device__ __forceinline__ void support_rank_to_mn(int k, int support, int Ls, int b, int br, int& m,
                                                   int& n) {
  if (support == FOFSE_SUPPORT_CAUSAL_L) {
    const int top = br * (br + b);
    if (k < top) {
      m = k / (br + b);
      n = k - m * (br + b);
    } else {
      const int k2 = k - top;
      m = br + k2 / br;
      n = k2 - (m - br) * br;
    }
    return;
  }
  const int top = br * Ls, mid = b * (Ls - b);
  if (k < top) {
    m = k / Ls;
    n = k - m * Ls;
  } else if (k < top + mid) {
    const int k2 = k - top, w = Ls - b;
    const int r = k2 / w, c = k2 - r * w;
    m = br + r;
    n = c < br ? c : c + b;
  } else {
    const int k2 = k - top - mid;
    const int r = k2 / Ls;
    m = br + b + r;
    n = k2 - r * Ls;
  }
}

// Sample pass of the split backward: CTA (block, chunk) rebuilds the residual
// f - g_{i-1} along the trace and accumulates xbar and wbar (see the header
// comment) for S support samples per thread at a time.  Per sample and
// iteration: the phase (u1 m + u2 n) mod T from one 32-bit multiply of packed
// operands (mn = m 2^(32-L) + n 2^(16-L), U = u1 + u2 2^16, L = log2 T: the
// product's top L bits are the phase, the cross term n u1 2^(16-L) stays
// below them), one table load and six FP32 operations.  The chunk CTAs of a
// block add their FP64 d/drho sums into the block's accumulators; the last to
// finish turns them into the block's d/drho.
template <int T, int NT, int S>
__global__ void __launch_bounds__(NT) fofse_backward_samples_kernel(const __grid_constant__ BwdArgs args,
                                                                    int chunks) {
  constexpr int LOGT = ilog2c(T), NW = NT / 32;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 15) & ~uintptr_t(15));
  const PlanDev& P = args.plan;
  const int iters = P.iters;
  // phase packing: mn = m 2^(32-L) + n 2^SN, U = u1 + u2 2^TU with SN + TU =
  // 32 - L puts (m u1 + n u2) mod T in the product's top L bits; the cross
  // term n u1 2^SN < 2^(29-L) stays below them, so the product shifted right
  // by 29 - L is the byte offset (phase x 8) of the table entry
  constexpr int SN = 29 - 3 * LOGT, TU = 3 + 2 * LOGT;
  static_assert(SN >= 0 && TU >= LOGT, "phase packing");
  __shared__ __align__(16) float2 syn[T];  // (cos, sin)(2 pi p / T)
  float2* tab = reinterpret_cast<float2*>(smem);   // abar_i
  float2* tcm = tab + iters;                       // (1 + s_i) c_i
  unsigned* tU = reinterpret_cast<unsigned*>(tcm + iters);  // u1 + u2 2^TU
  double* red = reinterpret_cast<double*>(smem + ((sizeof(float2) * 2 * iters +
                                                    sizeof(unsigned) * iters + 15) & ~size_t(15)));
  __shared__ bool s_last;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int blk = blockIdx.x / chunks, chunk = blockIdx.x - blk * chunks;
  const fofse_block bd = args.blocks[blk];
  if (bd.plan != args.plan_index) return;
  const float w0 = args.w0[blk];
  if (!(w0 > 0.f)) return;  // no support: zero gradient (the solve kernel skipped it too)
  const int b = P.block, br = P.border, Ls = P.Ls;
  const int ly0 = bd.y - br, lx0 = bd.x - br;

  for (int e = tid; e < T; e += NT) syn[e] = P.tab.syn_f32[e];
  for (int i = tid; i < iters; i += NT) {
    const fofse_trace_entry e = args.trace[(size_t)blk * args.trace_stride + i];
    const int u1 = (uint16_t)e.u1, u2 = (uint16_t)e.u2;
    const float mult = self_conj<T>(u1, u2) ? 1.f : 2.f;
    tcm[i] = make_float2(mult * e.dc_re, mult * e.dc_im);
    tU[i] = (unsigned)u1 | ((unsigned)u2 << TU);
    tab[i] = args.abar[(size_t)blk * args.trace_stride + i];
  }
  __syncthreads();

  const int npos = support_positions(P.support, Ls, b, br);
  const float c0 = br + (b - 1) * 0.5f;
  const float w0bar = args.w0bar[blk];
  float p_wwd = 0.f, p_ww = 0.f, p_wd = 0.f, p_w = 0.f;  // this thread's samples
  for (int base = chunk * NT * S; base < npos; base += chunks * NT * S) {
    float r[S], xb[S], wb[S];
    unsigned mn[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const int k = base + tid + j * NT;
      r[j] = 0.f;
      xb[j] = 0.f;
      wb[j] = 0.f;
      mn[j] = 0u;
      if (k < npos) {
        int m, n;
        support_rank_to_mn(k, P.support, Ls, b, br, m, n);
        const int fy = ly0 + m, fx = lx0 + n;
        if (fy >= 0 && fy < args.height && fx >= 0 && fx < args.width) {
          const size_t fi = (size_t)fy * args.pitch + fx;
          if (args.avail[fi]) r[j] = args.frame[fi];
        }
        mn[j] = ((unsigned)m << (32 - LOGT)) | ((unsigned)n << SN);
      }
    }
    for (int i = 0; i < iters; ++i) {
      const unsigned U = tU[i];
      const float2 ab = tab[i], cm = tcm[i];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const float2 cs = *reinterpret_cast<const float2*>(
            reinterpret_cast<const char*>(syn) + ((mn[j] * U) >> (29 - LOGT)));
        const float q = __fmaf_rn(ab.x, cs.x, -ab.y * cs.y);  // Re(abar_i phi_{u_i})
        xb[j] += q;
        wb[j] = __fmaf_rn(r[j], q, wb[j]);
        r[j] = __fmaf_rn(-cm.x, cs.x, __fmaf_rn(cm.y, cs.y, r[j]));  // - (1 + s) Re(c phi)
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const int k = base + tid + j * NT;
      if (k >= npos) continue;
      int m, n;
      support_rank_to_mn(k, P.support, Ls, b, br, m, n);
      const int fy = ly0 + m, fx = lx0 + n;
      if (fy < 0 || fy >= args.height || fx < 0 || fx >= args.width) continue;
      const size_t fi = (size_t)fy * args.pitch + fx;
      if (!args.avail[fi]) continue;
      const float w = P.tab.w_f32[m * Ls + n];
      if (args.grad_frame) atomicAdd(&args.grad_frame[fi], w * xb[j]);
      const float wbar = wb[j] + w0bar;
      const float dm = m - c0, dn = n - c0;
      const float d = sqrtf(dm * dm + dn * dn);
      const float ww = wbar * w;
      p_wwd = __fmaf_rn(ww, d, p_wwd);
      p_ww += ww;
      p_wd = __fmaf_rn(w, d, p_wd);
      p_w += w;
    }
  }
  if (!args.grad_rho_gamma) return;
  // a few samples per thread in FP32, the sums over threads and CTAs in FP64
  double s_wwd = p_wwd, s_ww = p_ww, s_wd = p_wd, s_w = p_w;
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
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < NW; ++w)
      for (int q = 0; q < 4; ++q) v[q] += red[4 * w + q];
    double* acc = args.acc + 4 * (size_t)blk;
    for (int q = 0; q < 4; ++q) atomicAdd(&acc[q], v[q]);
    __threadfence();
    s_last = atomicAdd(&args.cnt[blk], 1u) == (unsigned)(chunks - 1);
  }
  __syncthreads();
  if (s_last && tid == 0) {  // every chunk's sums are in: d/drho of this block
    __threadfence();
    const volatile double* acc = args.acc + 4 * (size_t)blk;
    const double a = acc[0], bb = acc[1], c = acc[2], d = acc[3];
    const double dbar = d > 0 ? c / d : 0.0;
    atomicAdd(&args.grad_rho_gamma[0], (float)((a - dbar * bb) / (double)(P.rho_gamma_dev ? P.rho_gamma_dev[0] : P.rho)));
  }
}

template <int T, int NT> size_t bwd_smem(int iters, bool split) {
  size_t off = 128 + sizeof(float) * T * 2 * T + (split ? 0 : sizeof(float2) * T);
  off += sizeof(int) * ((iters + 1) & ~1) + (split ? 2 : 3) * sizeof(float2) * iters;
  return off + (split ? 1 : 4) * sizeof(double) * (NT / 32);
}

// The shared-memory limit of a kernel is one attribute per device; it only
// grows, so a smaller request never lowers it below a size launched before.
template <class K> cudaError_t raise_smem_limit(K kern, size_t sm) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* kp = reinterpret_cast<const void*>(kern);
  std::lock_guard<std::mutex> lk(mu);
  auto lim = limit.find({kp, dev});
  if (lim == limit.end() || lim->second < sm) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    limit[{kp, dev}] = sm;
  }
  return cudaSuccess;
}

template <int T, int NT, int NTS, int S> cudaError_t launch_bwd(const BwdArgs& a, cudaStream_t s) {
  const size_t sm = bwd_smem<T, NT>(a.plan.iters, a.abar != nullptr);
  cudaError_t e;
  if (!a.abar) {  // one kernel per block
    auto kern = fofse_backward_kernel<T, NT, false>;
    if ((e = raise_smem_limit(kern, sm)) != cudaSuccess) return e;
    kern<<<a.n_blocks, NT, sm, s>>>(a);
    return cudaGetLastError();
  }
  auto solve = fofse_backward_kernel<T, NT, true>;
  if ((e = raise_smem_limit(solve, sm)) != cudaSuccess) return e;
  solve<<<a.n_blocks, NT, sm, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int iters = a.plan.iters;
  const size_t sms = ((sizeof(float2) * 2 * iters + sizeof(unsigned) * iters + 15) & ~size_t(15)) +
                     sizeof(double) * 4 * (NTS / 32) + 16;
  const int Ls = a.plan.Ls, b = a.plan.block, br = a.plan.border;
  const int npos = a.plan.support == FOFSE_SUPPORT_CAUSAL_L ? br * (br + b) + b * br : Ls * Ls - b * b;
  const int chunks = (npos + NTS * S - 1) / (NTS * S);
  if ((size_t)a.n_blocks * chunks > 0x7fffffffu) return cudaErrorInvalidValue;
  auto samples = fofse_backward_samples_kernel<T, NTS, S>;
  if ((e = raise_smem_limit(samples, sms)) != cudaSuccess) return e;
  samples<<<(unsigned)(a.n_blocks * chunks), NTS, sms, s>>>(a, chunks);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward(const BwdArgs& a, cudaStream_t s) {
  if (a.plan.precision == FOFSE_FP64_VALIDATE) return cudaErrorNotSupported;
  if (a.plan.basis == FOFSE_BASIS_DCT) return launch_backward_dct(a, s);
  if (a.plan.T == 128) return launch_bwd<128, 512, 128, 4>(a, s);
  if (a.plan.T == 64) return launch_bwd<64, 256, 128, 4>(a, s);
  if (a.plan.T == 32) return launch_bwd<32, 128, 64, 4>(a, s);
  return cudaErrorNotSupported;
}

}  // namespace fofse
