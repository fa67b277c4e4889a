// Forward FOFSE kernel (paper Sec. 2 in its transform-domain form, Sec. 4 setup).
//
// One CTA extrapolates one lost block:
//   1. stage   the support tile (frame + availability) of the area L into
//              shared memory with two TMA tile loads (plain loads when the
//              frame's alignment does not allow TMA);
//   2. weight  w = rho^dist on A (Eq. 4, Eq. 15), x = w f, packed as z = x + j w
//              at bit-reversed positions of a T x T grid (L at the origin);
//   3. FFT     one in-place radix-2 DIT 2-D FFT of z in shared memory, then the
//              Hermitian split Z -> R_w = DFT(x) (kept in registers, one index
//              per conjugate pair) and W = DFT(w) (kept in shared memory, full
//              grid, for the shifted gathers);
//   4. loop    `iters` times: block argmax of |R_w|^2 over the canonical set
//              (Eq. 9; warp shuffles + one barrier), c = gamma R_w[u] / W[0]
//              (Eq. 5, Eq. 14), R_w[k] -= c W[k-u] + s conj(c) W[k+u] for every
//              register-resident bin (the spectrum of the added pair, Eq. 2-3);
//   5. synth   B_hat = sum_i (1 + s_i) Re(c_i phi_{u_i}) over B (Eq. 1), written
//              to the packed output and/or scattered into the output frame.
//
// Shared-memory spectrum layout: T rows of 2T elements of type A::E; element
// (k1, k2) has part 0 at k1*2T + k2 and part 1 at k1*2T + T + k2 (float-float:
// hi plane / lo plane; FP64 and plain FP32: real / imaginary plane).  With
// that stride the cyclic shifts k -+ u of a bin stored as x_k = k1*2T + k2
// are one add and one AND: ((x_k + T - y_u) & M) and ((x_k + y_u) & M),
// M = (T-1)*2T + (T-1).
#include <cuda.h>
#include <cuda_runtime.h>

#include "fofse_arith.cuh"
#include "fofse_fft.cuh"
#include "fofse_internal.h"

namespace fofse {
namespace {

constexpr unsigned kWaitLimit = 1u << 24;  // bounded mbarrier polls

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// ---------------------------------------------------------------------------
// argmax candidates
// ---------------------------------------------------------------------------
template <class A> struct Cand;

template <> struct Cand<ArFF> {
  float m;  // FP32 estimate of |R|^2 (hi parts only)
  int code; // 2 * canonical index + (stored bin is the mirror)
  ff re, im;
};
template <> struct Cand<ArF64> {
  double m;
  int code;
  double re, im;
};
template <> struct Cand<ArF32> {
  float m;
  int code;
  float re, im;
};

__device__ __forceinline__ Cand<ArFF> make_cand(const ArFF::C& r, int code) {
  return {__fmaf_rn(r.re.h, r.re.h, __fmul_rn(r.im.h, r.im.h)), code, r.re, r.im};
}
__device__ __forceinline__ Cand<ArF64> make_cand(const ArF64::C& r, int code) {
  return {__dadd_rn(__dmul_rn(r.re, r.re), __dmul_rn(r.im, r.im)), code, r.re, r.im};
}
__device__ __forceinline__ Cand<ArF32> make_cand(const ArF32::C& r, int code) {
  return {__fadd_rn(__fmul_rn(r.re, r.re), __fmul_rn(r.im, r.im)), code, r.re, r.im};
}
template <class A> __device__ __forceinline__ Cand<A> empty_cand() {
  Cand<A> c;
  c.m = -1;
  c.code = 0x7fffffff;
  c.re = {};
  c.im = {};
  return c;
}

// Relative margin above which the FP32 estimates decide; below it the
// float-float magnitudes decide.  The estimates are within 2^-22 of |R|^2.
constexpr float kNearRel = 9.5367431640625e-07f;  // 2^-20

__device__ __forceinline__ bool better(const Cand<ArFF>& a, const Cand<ArFF>& b) {
  if (a.m > b.m + fabsf(b.m) * kNearRel) return true;
  if (b.m > a.m + fabsf(a.m) * kNearRel) return false;
  ff ma = ff_norm2(a.re, a.im), mb = ff_norm2(b.re, b.im);
  if (a.m < 0.f) ma = {-1.f, 0.f};
  if (b.m < 0.f) mb = {-1.f, 0.f};
  if (ma.h != mb.h) return ma.h > mb.h;
  if (ma.l != mb.l) return ma.l > mb.l;
  return a.code < b.code;
}
__device__ __forceinline__ bool better(const Cand<ArF64>& a, const Cand<ArF64>& b) {
  return a.m > b.m || (a.m == b.m && a.code < b.code);
}
__device__ __forceinline__ bool better(const Cand<ArF32>& a, const Cand<ArF32>& b) {
  return a.m > b.m || (a.m == b.m && a.code < b.code);
}

__device__ __forceinline__ Cand<ArFF> shfl(const Cand<ArFF>& c, int off) {
  Cand<ArFF> o;
  o.m = __shfl_xor_sync(0xffffffffu, c.m, off);
  o.code = __shfl_xor_sync(0xffffffffu, c.code, off);
  o.re.h = __shfl_xor_sync(0xffffffffu, c.re.h, off);
  o.re.l = __shfl_xor_sync(0xffffffffu, c.re.l, off);
  o.im.h = __shfl_xor_sync(0xffffffffu, c.im.h, off);
  o.im.l = __shfl_xor_sync(0xffffffffu, c.im.l, off);
  return o;
}
__device__ __forceinline__ Cand<ArF64> shfl(const Cand<ArF64>& c, int off) {
  Cand<ArF64> o;
  o.m = __shfl_xor_sync(0xffffffffu, c.m, off);
  o.code = __shfl_xor_sync(0xffffffffu, c.code, off);
  o.re = __shfl_xor_sync(0xffffffffu, c.re, off);
  o.im = __shfl_xor_sync(0xffffffffu, c.im, off);
  return o;
}
__device__ __forceinline__ Cand<ArF32> shfl(const Cand<ArF32>& c, int off) {
  Cand<ArF32> o;
  o.m = __shfl_xor_sync(0xffffffffu, c.m, off);
  o.code = __shfl_xor_sync(0xffffffffu, c.code, off);
  o.re = __shfl_xor_sync(0xffffffffu, c.re, off);
  o.im = __shfl_xor_sync(0xffffffffu, c.im, off);
  return o;
}

// Warp-wide argmax; every lane returns the winner.  Exact compare for the
// FP64 / plain FP32 back-ends.  For float-float, the FP32 estimates are
// reduced first; only if another lane's estimate lies within the near margin
// of the maximum are the float-float magnitudes compared (rare).
template <class A> __device__ __forceinline__ Cand<A> warp_argmax(Cand<A> c, int) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const Cand<A> other = shfl(c, o);
    if (better(other, c)) c = other;
  }
  return c;
}
__device__ __forceinline__ Cand<ArFF> warp_argmax(Cand<ArFF> c, int lane) {
  float M = c.m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
  const unsigned near = __ballot_sync(0xffffffffu, c.m >= M - fabsf(M) * kNearRel);
  if (__popc(near) != 1) {  // a near-tie: decide with the float-float magnitudes
    if (!((near >> lane) & 1u)) c = empty_cand<ArFF>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Cand<ArFF> other = shfl(c, o);
      if (better(other, c)) c = other;
    }
    return c;
  }
  const int src = __ffs(near) - 1;
  Cand<ArFF> w;
  w.m = M;
  w.code = __shfl_sync(0xffffffffu, c.code, src);
  w.re.h = __shfl_sync(0xffffffffu, c.re.h, src);
  w.re.l = __shfl_sync(0xffffffffu, c.re.l, src);
  w.im.h = __shfl_sync(0xffffffffu, c.im.h, src);
  w.im.l = __shfl_sync(0xffffffffu, c.im.l, src);
  return w;
}
template <int NW, class A> __device__ __forceinline__ Cand<A> block_argmax_generic(const Cand<A>* sl) {
  Cand<A> win = sl[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) {
    const Cand<A> c = sl[w];
    if (better(c, win)) win = c;
  }
  return win;
}
template <int NW> __device__ __forceinline__ Cand<ArF64> block_argmax(const Cand<ArF64>* sl) {
  return block_argmax_generic<NW>(sl);
}
template <int NW> __device__ __forceinline__ Cand<ArF32> block_argmax(const Cand<ArF32>* sl) {
  return block_argmax_generic<NW>(sl);
}
template <int NW> __device__ __forceinline__ Cand<ArFF> block_argmax(const Cand<ArFF>* sl) {
  float M = sl[0].m;
  int wi = 0;
#pragma unroll
  for (int w = 1; w < NW; ++w) {
    const float m = sl[w].m;
    if (m > M) {
      M = m;
      wi = w;
    }
  }
  const float thr = M - fabsf(M) * kNearRel;
  int cnt = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) cnt += sl[w].m >= thr ? 1 : 0;
  if (cnt == 1) return sl[wi];
  Cand<ArFF> win = empty_cand<ArFF>();  // near-tie across warps
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const Cand<ArFF> c = sl[w];
    if (c.m >= thr && better(c, win)) win = c;
  }
  return win;
}

// ---------------------------------------------------------------------------
// coefficient (Eq. 5 with |phi| = 1, Eq. 14) and the rank-1 shifted update
// ---------------------------------------------------------------------------
__device__ __forceinline__ ArFF::C coef(const Cand<ArFF>& w, ff inv, bool sc) {
  ArFF::C d;
  d.re = ff_mul(w.re, inv);
  d.im = sc ? ff{0.f, 0.f} : ff_mul(w.im, inv);
  return d;
}
__device__ __forceinline__ ArF64::C coef(const Cand<ArF64>& w, double inv, bool sc) {
  return {w.re * inv, sc ? 0.0 : w.im * inv};
}
__device__ __forceinline__ ArF32::C coef(const Cand<ArF32>& w, float inv, bool sc) {
  return {w.re * inv, sc ? 0.f : w.im * inv};
}

// R -= c Wm + conj(c) Wp, written as
//   Re: p (Wm.re + Wp.re) - q (Wm.im - Wp.im),  Im: p (Wm.im + Wp.im) + q (Wm.re - Wp.re)
__device__ __forceinline__ void update_pair(ArFF::C& R, const ArFF::C& c, const ArFF::C& Wm,
                                            const ArFF::C& Wp) {
  ff s1 = ff_add_raw(Wm.re, Wp.re), s2 = ff_sub_raw(Wm.im, Wp.im);
  ff s3 = ff_sub_raw(Wm.re, Wp.re), s4 = ff_add_raw(Wm.im, Wp.im);
  ff tre = ff_dot2(c.re, s1, ff_neg(c.im), s2);
  ff tim = ff_dot2(c.re, s4, c.im, s3);
  R.re = ff_sub(R.re, tre);
  R.im = ff_sub(R.im, tim);
}
// self-conjugate u: real c, R -= c Wm
__device__ __forceinline__ void update_single(ArFF::C& R, const ArFF::C& c, const ArFF::C& Wm) {
  ff tre = ff_dot2(c.re, Wm.re, ff{0.f, 0.f}, ff{0.f, 0.f});
  ff tim = ff_dot2(c.re, Wm.im, ff{0.f, 0.f}, ff{0.f, 0.f});
  R.re = ff_sub(R.re, tre);
  R.im = ff_sub(R.im, tim);
}
template <class A>
__device__ __forceinline__ void update_pair(typename A::C& R, const typename A::C& c,
                                            const typename A::C& Wm, const typename A::C& Wp) {
  R.re = R.re - (c.re * (Wm.re + Wp.re) - c.im * (Wm.im - Wp.im));
  R.im = R.im - (c.re * (Wm.im + Wp.im) + c.im * (Wm.re - Wp.re));
}
template <class A>
__device__ __forceinline__ void update_single(typename A::C& R, const typename A::C& c,
                                              const typename A::C& Wm) {
  R.re = R.re - c.re * Wm.re;
  R.im = R.im - c.re * Wm.im;
}
template <class A> struct Upd {
  __device__ __forceinline__ static void pair(typename A::C& R, const typename A::C& c,
                                              const typename A::C& Wm, const typename A::C& Wp) {
    update_pair<A>(R, c, Wm, Wp);
  }
  __device__ __forceinline__ static void single(typename A::C& R, const typename A::C& c,
                                                const typename A::C& Wm) {
    update_single<A>(R, c, Wm);
  }
};
template <> struct Upd<ArFF> {
  __device__ __forceinline__ static void pair(ArFF::C& R, const ArFF::C& c, const ArFF::C& Wm,
                                              const ArFF::C& Wp) {
    update_pair(R, c, Wm, Wp);
  }
  __device__ __forceinline__ static void single(ArFF::C& R, const ArFF::C& c, const ArFF::C& Wm) {
    update_single(R, c, Wm);
  }
};

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
  __device__ static ff gamma(const PlanDev& p) { return {p.gamma_h, p.gamma_l}; }
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
  __device__ static double gamma(const PlanDev& p) { return p.gamma; }
  __device__ static double inv_w0(double g, double w0) { return g / w0; }
  __device__ static bool w0_zero(const ArF64::C& w) { return w.re == 0.0; }
  __device__ static bool w0_finite(const ArF64::C& w) { return isfinite(w.re); }
  __device__ static float w0_out(const ArF64::C& w) { return (float)w.re; }
  __device__ static Syn syn(const PlanTables& t, int p) { return t.syn_f64[p]; }
  __device__ static float round_re(const ArF64::C& c) { return (float)c.re; }
  __device__ static float round_im(const ArF64::C& c) { return (float)c.im; }
  __device__ static double synacc(const ArF64::C& c, bool re) { return re ? c.re : c.im; }
};
template <> struct PlanIO<ArF32> {
  using Syn = float2;
  using SynAcc = float;
  __device__ static ArF32::C twiddle(const PlanTables& t, int e) {
    float2 v = t.tw_f32[e];
    return {v.x, v.y};
  }
  __device__ static ArF32::C weighted(const PlanTables& t, int i, float f, ArF32::C& wout) {
    float w = t.w_f32[i];
    wout = {w, 0.f};
    return {w * f, w};
  }
  __device__ static float gamma(const PlanDev& p) { return (float)p.gamma; }
  __device__ static float inv_w0(float g, float w0) { return g / w0; }
  __device__ static bool w0_zero(const ArF32::C& w) { return w.re == 0.f; }
  __device__ static bool w0_finite(const ArF32::C& w) { return isfinite(w.re); }
  __device__ static float w0_out(const ArF32::C& w) { return w.re; }
  __device__ static Syn syn(const PlanTables& t, int p) { return t.syn_f32[p]; }
  __device__ static float round_re(const ArF32::C& c) { return c.re; }
  __device__ static float round_im(const ArF32::C& c) { return c.im; }
  __device__ static float synacc(const ArF32::C& c, bool re) { return re ? c.re : c.im; }
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

template <class A, int T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fofse_forward_kernel(const __grid_constant__ FwdArgs args,
                                                           const __grid_constant__ CUtensorMap tmF,
                                                           const __grid_constant__ CUtensorMap tmA) {
  using C = typename A::C;
  using E = typename A::E;
  using IO = PlanIO<A>;
  using G = Geo<A, T>;
  constexpr int T2 = G::T2, LOGT = G::LOGT, NBINS = G::NBINS;
  constexpr int NSLOT = T * T / 2;
  constexpr int NBF = NSLOT / NT;  // full steps; the 2 extra bins go to threads 0 and 1
  constexpr int NB = NBF + 1;
  constexpr int NW = NT / 32;
  static_assert(NSLOT % NT == 0 && NT >= 64, "slot grid");
  static_assert(NBINS == NSLOT + 2, "bins");

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  E* Z = reinterpret_cast<E*>(smem);
  size_t off = sizeof(E) * T * T2;
  C* tw = reinterpret_cast<C*>(smem + off);
  off += sizeof(C) * (T / 2);
  using Syn = typename IO::Syn;
  Syn* syn = reinterpret_cast<Syn*>(smem + off);
  off += sizeof(Syn) * T;
  Cand<A>* slots = reinterpret_cast<Cand<A>*>(smem + off);
  off += sizeof(Cand<A>) * 2 * NW;
  off = (off + 15) & ~size_t(15);
  TraceSm<A>* tr = reinterpret_cast<TraceSm<A>*>(smem + off);
  __shared__ uint64_t mbar;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int blk = blockIdx.x;
  const PlanDev& P = args.plan;
  const fofse_block bd = args.blocks[blk];
  if (bd.plan != args.plan_index) return;
  const int b = P.block, br = P.border, Ls = P.Ls, iters = P.iters;
  const int ly0 = bd.y - br, lx0 = bd.x - br;  // L's top-left in the frame

  // ---- 1. stage the support tile --------------------------------------------
  float* stF = reinterpret_cast<float*>(smem);
  const int bytesF = args.box_f * Ls * 4;
  uint8_t* stA = smem + ((bytesF + 127) & ~127);
  const int fx0 = lx0 & ~3, fo = lx0 - fx0;    // 16-byte aligned starts
  const int ax0 = lx0 & ~15, ao = lx0 - ax0;
  if (args.use_tma) {
    if (tid == 0) {
      mbar_init(&mbar, 1);
      fence_proxy_async();
    }
    __syncthreads();
    if (tid == 0) {
      mbar_expect_tx(&mbar, (unsigned)(bytesF + args.box_a * Ls));
      tma_load_2d(stF, &tmF, fx0, ly0, &mbar);
      tma_load_2d(stA, &tmA, ax0, ly0, &mbar);
    }
    bool done = false;
    for (unsigned it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(&mbar, 0);
    if (!done) {
      atomicOr(args.err, kErrTimeout);
      if (args.status && tid == 0) args.status[blk] = kBlkTimeout;
      // wait (bounded again) for the copy in flight before the CTA retires
      for (unsigned it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(&mbar, 0);
      return;
    }
  }

  // ---- 2. weighting and the packed input z = w f + j w (bit-reversed) -------
  constexpr int PER = (T * T + NT - 1) / NT;
  float fv[PER];
  unsigned use = 0;
  bool bad = false;
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int e = tid + s * NT;
    fv[s] = 0.f;
    if (e < T * T) {
      const int m = __brev(e >> LOGT) >> (32 - LOGT);
      const int n = __brev(e & (T - 1)) >> (32 - LOGT);
      if (m < Ls && n < Ls) {
        bool inB = m >= br && m < br + b && n >= br && n < br + b;
        bool inS = true;
        if (P.support == FOFSE_SUPPORT_CAUSAL_L)
          inS = (m < br) ? (n < br + b) : (m < br + b ? n < br : false);
        int av;
        float f;
        if (args.use_tma) {
          av = stA[m * args.box_a + ao + n];
          f = stF[m * args.box_f + fo + n];
        } else {
          const int fy = ly0 + m, fx = lx0 + n;
          const bool in = fy >= 0 && fy < args.height && fx >= 0 && fx < args.width;
          av = in ? args.avail[(size_t)fy * args.pitch + fx] : 0;
          f = in ? args.frame[(size_t)fy * args.pitch + fx] : 0.f;
        }
        if (av && !inB && inS) {
          use |= 1u << s;
          fv[s] = f;
          bad |= !isfinite(f);
        }
      }
    }
  }
  int any_bad = __syncthreads_or(bad);  // the staging area is overwritten below
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int e = tid + s * NT;
    if (e < T * T) {
      const int r = e >> LOGT, c = e & (T - 1);
      C z = A::zero();
      if (use & (1u << s)) {
        const int m = __brev(r) >> (32 - LOGT), n = __brev(c) >> (32 - LOGT);
        C wdummy;
        z = IO::weighted(P.tab, m * Ls + n, fv[s], wdummy);
      }
      A::store(Z, r * T2 + c, T, z);
    }
  }
  for (int e = tid; e < T / 2; e += NT) tw[e] = IO::twiddle(P.tab, e);
  for (int e = tid; e < T; e += NT) syn[e] = IO::syn(P.tab, e);
  __syncthreads();

  // ---- 3. FFT: rows that hold data, then all columns (radix-2 DIT) ----------
  fft2d_dit<A, T, NT, false>(Z, tw, Ls, T);

  // ---- split: R_w[k] = (Z[k] + conj Z[-k]) / 2 into registers ---------------
  C R[NB];
  int kc[NB];  // x_k | code << 16
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    kc[i] = 0;
    R[i] = A::zero();
    if (i < NBF || tid < 2) {
      const int x = i < NBF ? slot_xk<T>(tid + i * NT) : extra_xk<T>(tid);
      kc[i] = x | (code_of<T>(x) << 16);
      const int k1 = x >> (LOGT + 1), k2 = x & (T2 - 1);
      const int mx = ((T - k1) & (T - 1)) * T2 + ((T - k2) & (T - 1));
      C a = A::load(Z, x, T), m = A::load(Z, mx, T);
      R[i] = A::half(A::add(a, A::conj(m)));
      if (!A::finite(R[i])) bad = true;
    }
  }
  any_bad |= __syncthreads_or(bad);
  // ---- W[k] = (Z[k] - conj Z[-k]) / (2j) in place, W[-k] = conj W[k] ---------
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
  __syncthreads();

  const C W0c = A::load(Z, 0, T);
  int st = FOFSE_BLK_OK;
  if (IO::w0_zero(W0c)) st = FOFSE_BLK_NO_SUPPORT;
  else if (any_bad || !IO::w0_finite(W0c)) st = FOFSE_BLK_NONFINITE;

  if (st == FOFSE_BLK_OK) {
    const auto inv = IO::inv_w0(IO::gamma(P), W0c.re);
    // initial candidates
    Cand<A> best = empty_cand<A>();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i < NBF || tid < 2) {
        const Cand<A> c = make_cand(R[i], kc[i] >> 16);
        if (better(c, best)) best = c;
      }
    }
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
      // ---- 4a. block argmax (Eq. 9) ----
      best = warp_argmax(best, lane);
      Cand<A>* sl = slots + (it & 1) * NW;
      if (lane == 0) sl[warp] = best;
      __syncthreads();
      const Cand<A> win = block_argmax<NW>(sl);
      // ---- 4b. coefficient (Eq. 5, Eq. 14) ----
      const int canon = win.code >> 1;
      const bool mir = win.code & 1;
      const int u1 = canon >> LOGT, u2 = canon & (T - 1);
      const int s1 = mir ? ((T - u1) & (T - 1)) : u1;
      const int s2 = mir ? ((T - u2) & (T - 1)) : u2;
      const bool sc = ((s1 & (T / 2 - 1)) == 0) && ((s2 & (T / 2 - 1)) == 0);
      const C c = coef(win, inv, sc);
      if (tid == 0) {
        TraceSm<A> t;
        t.u = (u1 << 16) | u2;
        const float mult = sc ? 1.f : 2.f;
        t.re = mult * IO::synacc(c, true);
        t.im = (mir ? -mult : mult) * IO::synacc(c, false);
        t.dre = IO::round_re(c);
        t.dim = mir ? -IO::round_im(c) : IO::round_im(c);
        tr[it] = t;
      }
      // ---- 4c. rank-1 cyclic-shift update + next local argmax ----
      const int y = s1 * T2 + s2;
      best = empty_cand<A>();
      if (!sc) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < NBF || tid < 2) {
            const int x = kc[i] & 0xffff;
            const C Wm = A::load(Z, (x + T - y) & G::M, T);
            const C Wp = A::load(Z, (x + y) & G::M, T);
            Upd<A>::pair(R[i], c, Wm, Wp);
            const Cand<A> cd = make_cand(R[i], kc[i] >> 16);
            if (better(cd, best)) best = cd;
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < NBF || tid < 2) {
            const C Wm = A::load(Z, ((kc[i] & 0xffff) + T - y) & G::M, T);
            Upd<A>::single(R[i], c, Wm);
            const Cand<A> cd = make_cand(R[i], kc[i] >> 16);
            if (better(cd, best)) best = cd;
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- 5. synthesis of B (Eq. 1) and outputs ---------------------------------
  using SA = typename IO::SynAcc;
  const int nIt = (st == FOFSE_BLK_OK) ? iters : 0;
  for (int p = tid; p < b * b; p += NT) {
    const int bm = p / b, bn = p - bm * b;
    const int m = br + bm, n = br + bn;
    SA acc = 0;
    for (int i = 0; i < nIt; ++i) {
      const TraceSm<A> t = tr[i];
      const int ph = ((t.u >> 16) * m + (t.u & 0xffff) * n) & (T - 1);
      const Syn cs = syn[ph];
      acc += t.re * cs.x - t.im * cs.y;
    }
    const float v = (float)acc;
    if (args.out_blocks) args.out_blocks[(size_t)blk * args.out_stride + p] = v;
    if (args.out_frame) {
      const int fy = bd.y + bm, fx = bd.x + bn;
      if (fy >= 0 && fy < args.height && fx >= 0 && fx < args.width)
        args.out_frame[(size_t)fy * args.pitch + fx] = v;
    }
  }
  if (args.trace) {
    for (int i = tid; i < iters; i += NT) {
      fofse_trace_entry e;
      if (i < nIt) {
        const TraceSm<A> t = tr[i];
        e.u1 = (int16_t)(t.u >> 16);
        e.u2 = (int16_t)(t.u & 0xffff);
        e.dc_re = t.dre;
        e.dc_im = t.dim;
      } else {
        e.u1 = e.u2 = 0;
        e.dc_re = e.dc_im = 0.f;
      }
      args.trace[(size_t)blk * args.trace_stride + i] = e;
    }
  }
  if (tid == 0) {
    if (args.w0) args.w0[blk] = st == FOFSE_BLK_OK ? IO::w0_out(W0c) : 0.f;
    if (args.status) args.status[blk] = st;
  }
}

template <class A, int T, int NT> size_t smem_bytes(int iters) {
  size_t off = 1024 + sizeof(typename A::E) * T * 2 * T;  // + alignment slack
  off += sizeof(typename A::C) * (T / 2);
  off += sizeof(typename PlanIO<A>::Syn) * T;
  off += sizeof(Cand<A>) * 2 * (NT / 32);
  off = (off + 15) & ~size_t(15);
  off += sizeof(TraceSm<A>) * (size_t)iters;
  return off;
}

template <class A, int T, int NT, int MINB = 1>
cudaError_t launch_one(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta,
                       cudaStream_t s) {
  const size_t sm = smem_bytes<A, T, NT>(a.plan.iters);
  auto kern = fofse_forward_kernel<A, T, NT, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<a.n_blocks, NT, sm, s>>>(a, *tf, *ta);
  return cudaGetLastError();
}

}  // namespace

size_t forward_smem_bytes(int precision, int T, int iters) {
  if (T == 64) {
    if (precision == FOFSE_FP64_VALIDATE) return smem_bytes<ArF64, 64, 256>(iters);
    if (precision == FOFSE_FP32_PLAIN) return smem_bytes<ArF32, 64, 256>(iters);
    return smem_bytes<ArFF, 64, 256>(iters);
  }
  if (T == 32) {
    if (precision == FOFSE_FP64_VALIDATE) return smem_bytes<ArF64, 32, 128>(iters);
    if (precision == FOFSE_FP32_PLAIN) return smem_bytes<ArF32, 32, 128>(iters);
    return smem_bytes<ArFF, 32, 128>(iters);
  }
  return 0;
}

cudaError_t launch_forward(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta,
                           cudaStream_t s) {
  const int T = a.plan.T, pr = a.plan.precision;
  if (T == 64) {
    if (pr == FOFSE_FP64_VALIDATE) return launch_one<ArF64, 64, 256>(a, tf, ta, s);
    if (pr == FOFSE_FP32_PLAIN) return launch_one<ArF32, 64, 256>(a, tf, ta, s);
    return launch_one<ArFF, 64, 256, 3>(a, tf, ta, s);
  }
  if (T == 32) {
    if (pr == FOFSE_FP64_VALIDATE) return launch_one<ArF64, 32, 128>(a, tf, ta, s);
    if (pr == FOFSE_FP32_PLAIN) return launch_one<ArF32, 32, 128>(a, tf, ta, s);
    return launch_one<ArFF, 32, 128>(a, tf, ta, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fofse
