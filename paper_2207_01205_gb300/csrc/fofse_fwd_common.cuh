// Pieces shared by the forward kernels (all-bins and filtered-exact variants):
// plan table access per arithmetic back-end, TMA / mbarrier helpers, the
// spectrum-table accessors, the W build from the packed FFT, the exact
// triangular recurrence of the working spectrum, and the cached kernel
// attribute setup.  Included by one translation unit per kernel family
// (internal linkage).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <utility>

#include "fofse_arith.cuh"
#include "fofse_fft.cuh"
#include "fofse_internal.h"

namespace fofse {
namespace {

constexpr unsigned kWaitLimit = 1u << 24;  // bounded mbarrier polls

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// ---------------------------------------------------------------------------
// per-back-end plan scalars and tables
// ---------------------------------------------------------------------------
template <class A> struct PlanIO;
template <> struct PlanIO<ArFF> {
  using Syn = float2;
  using SynAcc = float;
  __device__ static ArFF::C twiddle(const PlanTables& t, int e) {
    float4 v = t.tw_ff[e];
    return {{v.x, v.z}, {v.y, v.w}};
  }
  __device__ static ArFF::C weighted(const PlanTables& t, int i, float f, ArFF::C& wout) {
    float2 w = t.w_ff[i];  // (hi, lo)
    ff x = ff_two_prod(w.x, f);
    x.l = __fmaf_rn(w.y, f, x.l);
    x = ff_fast_two_sum(x.h, x.l);
    wout = {{w.x, w.y}, {0.f, 0.f}};
    return {x, {w.x, w.y}};  // z = x + j w
  }
  __device__ static ff gamma(const PlanDev& p) {
    return p.rho_gamma_dev ? ff{p.rho_gamma_dev[1], 0.f} : ff{p.gamma_h, p.gamma_l};
  }
  __device__ static ff inv_w0(ff g, ff w0) { return ff_div(g, w0); }
  __device__ static bool w0_zero(const ArFF::C& w) { return w.re.h == 0.f; }
  __device__ static bool w0_finite(const ArFF::C& w) { return isfinite(w.re.h); }
  __device__ static float w0_out(const ArFF::C& w) { return w.re.h + w.re.l; }
  __device__ static Syn syn(const PlanTables& t, int p) { return t.syn_f32[p]; }
  __device__ static float round_re(const ArFF::C& c) { return c.re.h; }
  __device__ static float round_im(const ArFF::C& c) { return c.im.h; }
  __device__ static float synacc(const ArFF::C& c, bool re) { return re ? c.re.h : c.im.h; }
};
template <> struct PlanIO<ArF64> {
  using Syn = double2;
  using SynAcc = double;
  __device__ static ArF64::C twiddle(const PlanTables& t, int e) {
    double2 v = t.tw_f64[e];
    return {v.x, v.y};
  }
  __device__ static ArF64::C weighted(const PlanTables& t, int i, float f, ArF64::C& wout) {
    double w = t.w_f64[i];
    wout = {w, 0.0};
    return {w * (double)f, w};
  }
  __device__ static double gamma(const PlanDev& p) {
    return p.rho_gamma_dev ? (double)p.rho_gamma_dev[1] : p.gamma;
  }
  __device__ static double inv_w0(double g, double w0) { return g / w0; }
  __device__ static bool w0_zero(const ArF64::C& w) { return w.re == 0.0; }
  __device__ static bool w0_finite(const ArF64::C& w) { return isfinite(w.re); }
  __device__ static float w0_out(const ArF64::C& w) { return (float)w.re; }
  __device__ static Syn syn(const PlanTables& t, int p) { return t.syn_f64[p]; }
  __device__ static float round_re(const ArF64::C& c) { return (float)c.re; }
  __device__ static float round_im(const ArF64::C& c) { return (float)c.im; }
  __device__ static double synacc(const ArF64::C& c, bool re) { return re ? c.re : c.im; }
};
template <class A> struct TraceSm {
  int u;                             // u1 << 16 | u2 (canonical index)
  typename PlanIO<A>::SynAcc re, im; // (1 + s) c
  float dre, dim;                    // c rounded to FP32 (for the trace output)
};

// ---------------------------------------------------------------------------
// TMA / mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class A, int T> struct Geo {
  static constexpr int LOGT = ilog2(T);
  static constexpr int T2 = 2 * T;
  static constexpr int M = (T - 1) * 2 * T + (T - 1);
  static constexpr int NBINS = T * T / 2 + 2;  // one index per conjugate pair
};

// Slot s of the T x T/2 slot grid (row = s / (T/2), column = s % (T/2)) ->
// packed x_k = k1*2T + k2 of a bin of the canonical set.  Columns 1..T/2-1
// are the interior bins of every row; column 0 holds bins (r, 0) for
// r <= T/2 and, in rows T/2+1..T-1, the bins (r - T/2 - 1, T/2) of the last
// half-spectrum column.  Two bins remain, (T/2 - 1, T/2) and (T/2, T/2): the
// "extra" slots.  Consecutive lanes hold consecutive columns of one row, so
// the shifted gathers W[k -+ u] of a warp hit 32 consecutive columns (mod T)
// of one shared-memory row: no bank conflicts.
template <int T> __device__ __forceinline__ int slot_xk(int s) {
  const int row = s >> (ilog2(T) - 1), col = s & (T / 2 - 1);
  int k1 = row, k2 = col;
  if (col == 0 && row > T / 2) {
    k1 = row - (T / 2 + 1);
    k2 = T / 2;
  }
  return k1 * 2 * T + k2;
}
template <int T> __device__ __forceinline__ int extra_xk(int e) {
  return (T / 2 - 1 + e) * 2 * T + T / 2;
}
template <int T> __device__ __forceinline__ int code_of(int xk) {
  int k1 = xk >> (ilog2(T) + 1), k2 = xk & (2 * T - 1);
  bool mir = (k2 > 0) && (k2 < T / 2) && (k1 > T / 2);
  int canon = mir ? (((T - k1) & (T - 1)) * T + (T - k2)) : (k1 * T + k2);
  return canon * 2 + (mir ? 1 : 0);
}

// Where W lives during the iterations.  Full: the whole T x T grid in shared
// memory in the two-plane layout above (T <= 64; the FFT runs in place).
// Half: only the Hermitian half k2 in [0, T/2] (rows of 2 (T/2 + 1)
// elements: part 0 at r*HS + c, part 1 at r*HS + HO + c); a gather at
// a2 > T/2 reads the mirror and conjugates.  Used at T = 128, where the full
// float-float grid (256 KB) does not fit; the FFT then runs in a per-CTA slot
// of global scratch (L2-resident).
template <class A, int T, bool HALF> struct WTab;
template <class A, int T> struct WTab<A, T, false> {
  using C = typename A::C;
  using E = typename A::E;
  static constexpr int M = (T - 1) * 2 * T + (T - 1);
  static constexpr size_t elems = (size_t)T * 2 * T;
  __device__ __forceinline__ static C minus(const E* W, int x, int y) {
    return A::load(W, (x + T - y) & M, T);
  }
  __device__ __forceinline__ static C plus(const E* W, int x, int y) {
    return A::load(W, (x + y) & M, T);
  }
  __device__ __forceinline__ static C at0(const E* W) { return A::load(W, 0, T); }
};
template <class A, int T> struct WTab<A, T, true> {
  using C = typename A::C;
  using E = typename A::E;
  static constexpr int LOGT = ilog2(T);
  static constexpr int M = (T - 1) * 2 * T + (T - 1);
  static constexpr int HO = T / 2 + 1, HS = 2 * HO;
  static constexpr size_t elems = (size_t)T * HS;
  __device__ __forceinline__ static C get(const E* W, int a) {  // a = a1*2T + a2, a2 < T
    const int a1 = a >> (LOGT + 1), a2 = a & (T - 1);
    const bool mir = a2 > T / 2;
    const int r = mir ? ((T - a1) & (T - 1)) : a1;
    const int c = mir ? (T - a2) : a2;
    const C v = A::load(W + r * HS, c, HO);
    return mir ? A::conj(v) : v;
  }
  __device__ __forceinline__ static C minus(const E* W, int x, int y) { return get(W, (x + T - y) & M); }
  __device__ __forceinline__ static C plus(const E* W, int x, int y) { return get(W, (x + y) & M); }
  __device__ __forceinline__ static C at0(const E* W) { return A::load(W, 0, HO); }
};

// Build W[k] = (Z[k] - conj Z[-k]) / (2j) from the packed FFT: in place over the
// full grid (W[-k] = conj W[k]), or its Hermitian half into shared memory.
template <class A, int T, int NT, bool HALF>
__device__ __forceinline__ void build_wtab(typename A::E* Z, typename A::E* Wsm) {
  using C = typename A::C;
  constexpr int T2 = 2 * T, LOGT = ilog2(T);
  const int tid = threadIdx.x;
  if constexpr (!HALF) {
    for (int e = tid; e < T * T; e += NT) {
      const int k1 = e >> LOGT, k2 = e & (T - 1);
      const int m1 = (T - k1) & (T - 1), m2 = (T - k2) & (T - 1);
      const int me = m1 * T + m2;
      if (e <= me) {
        C a = A::load(Z, k1 * T2 + k2, T), m = A::load(Z, m1 * T2 + m2, T);
        C d = A::sub(a, A::conj(m));  // W = -j d / 2
        C wv;
        wv.re = d.im;
        wv.im = d.re;
        wv = A::conj(A::half(wv));
        A::store(Z, k1 * T2 + k2, T, wv);
        if (me != e) A::store(Z, m1 * T2 + m2, T, A::conj(wv));
      }
    }
  } else {
    constexpr int HO = WTab<A, T, true>::HO, HS = WTab<A, T, true>::HS;
    for (int e = tid; e < T * HO; e += NT) {
      const int k1 = e / HO, k2 = e - k1 * HO;
      const int m1 = (T - k1) & (T - 1), m2 = (T - k2) & (T - 1);
      C a = A::load(Z, k1 * T2 + k2, T), m = A::load(Z, m1 * T2 + m2, T);
      C d = A::sub(a, A::conj(m));
      C wv;
      wv.re = d.im;
      wv.im = d.re;
      wv = A::conj(A::half(wv));
      A::store(Wsm + k1 * HS, k2, HO, wv);
    }
  }
}

__device__ __forceinline__ float m32(float2 r) { return __fmaf_rn(r.x, r.x, __fmul_rn(r.y, r.y)); }

struct ffc { ff re, im; };
__device__ __forceinline__ ffc ffc_add(ffc a, ffc b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ ffc ffc_shfl(ffc v, int o) {
  return {{__shfl_xor_sync(0xffffffffu, v.re.h, o), __shfl_xor_sync(0xffffffffu, v.re.l, o)},
          {__shfl_xor_sync(0xffffffffu, v.im.h, o), __shfl_xor_sync(0xffffffffu, v.im.l, o)}};
}
__device__ __forceinline__ ffc ffc_warp_sum(ffc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ffc_add(v, ffc_shfl(v, o));
  return v;
}
// sum over j in {j0, j0 + stride, ...} < j1 of  c_j W[k - u_j] + s_j conj(c_j) W[k + u_j]
// (exact float-float; canonical u_j packed as y_j = u1 * 2T + u2, c_j as (re.h, re.l, im.h, im.l))
template <class WT, int T>
__device__ __forceinline__ ffc recur_partial(const ArFF::E* Wsm, const int* ty, const float4* tc,
                                             int x, int j0, int j1, int stride) {
  ffc acc = {{0.f, 0.f}, {0.f, 0.f}};
  for (int j = j0; j < j1; j += stride) {
    const int y = ty[j];
    const float4 c4 = tc[j];
    const ArFF::C c = {{c4.x, c4.y}, {c4.z, c4.w}};
    const int u1 = y >> (ilog2(T) + 1), u2 = y & (2 * T - 1);
    const bool sc = ((u1 & (T / 2 - 1)) == 0) && ((u2 & (T / 2 - 1)) == 0);
    const ArFF::C Wm = WT::minus(Wsm, x, y);
    ArFF::C t;
    if (!sc) {
      const ArFF::C Wp = WT::plus(Wsm, x, y);
      ff s1 = ff_add_raw(Wm.re, Wp.re), s2 = ff_sub_raw(Wm.im, Wp.im);
      ff s3 = ff_sub_raw(Wm.re, Wp.re), s4 = ff_add_raw(Wm.im, Wp.im);
      t.re = ff_dot2(c.re, s1, ff_neg(c.im), s2);
      t.im = ff_dot2(c.re, s4, c.im, s3);
    } else {
      t.re = ff_dot2(c.re, Wm.re, ff{0.f, 0.f}, ff{0.f, 0.f});
      t.im = ff_dot2(c.re, Wm.im, ff{0.f, 0.f}, ff{0.f, 0.f});
    }
    acc.re = ff_add(acc.re, t.re);
    acc.im = ff_add(acc.im, t.im);
  }
  return acc;
}
// exact order on (value, code): larger |R|^2 first, then the smaller code
__device__ __forceinline__ bool exact_better(const ffc& a, int ca, const ffc& b, int cb) {
  const ff ma = ff_norm2(a.re, a.im), mb = ff_norm2(b.re, b.im);
  if (ma.h != mb.h) return ma.h > mb.h;
  if (ma.l != mb.l) return ma.l > mb.l;
  return ca < cb;
}

// Kernel attribute setting and occupancy query, done once per (kernel, device,
// shared-memory size) and cached: launches then issue no query, which keeps
// the batch call cheap and safe to record in a CUDA graph.
// Entries are keyed by the kernel itself (kernels of one signature share this
// template instance).  The dynamic shared-memory limit of a kernel is one
// attribute per device, so it only ever grows (to the largest size requested
// so far): a later, smaller request must not lower it below a size whose
// launch is already cached.
template <class K> cudaError_t prepare_kernel(K kern, int nt, size_t smem, int* max_ctas) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  static std::map<std::pair<const void*, int>, size_t> limit;
  const void* kp = reinterpret_cast<const void*>(kern);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({kp, dev, smem});
  if (it != cache.end()) {
    *max_ctas = it->second;
    return cudaSuccess;
  }
  auto lim = limit.find({kp, dev});
  if (lim == limit.end() || lim->second < smem) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    limit[{kp, dev}] = smem;
  }
  int sms = 0, per = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, nt, smem)) != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  cache[{kp, dev, smem}] = sms * per;
  *max_ctas = sms * per;
  return cudaSuccess;
}

}  // namespace
}  // namespace fofse
