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
// hi plane / lo plane; FP64: real / imaginary plane).  With
// that stride the cyclic shifts k -+ u of a bin stored as x_k = k1*2T + k2
// are one add and one AND: ((x_k + T - y_u) & M) and ((x_k + y_u) & M),
// M = (T-1)*2T + (T-1).
#include "fofse_fwd_common.cuh"

namespace fofse {
namespace {

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
__device__ __forceinline__ Cand<ArFF> make_cand(const ArFF::C& r, int code) {
  return {__fmaf_rn(r.re.h, r.re.h, __fmul_rn(r.im.h, r.im.h)), code, r.re, r.im};
}
__device__ __forceinline__ Cand<ArF64> make_cand(const ArF64::C& r, int code) {
  return {__dadd_rn(__dmul_rn(r.re, r.re), __dmul_rn(r.im, r.im)), code, r.re, r.im};
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

// Per-thread top-2 of the FP32 magnitude estimates (filtered variant).
struct Top2 {
  float m1;   // largest |R32|^2
  int c1;     // its code (2 * canonical index + mirror flag)
  int s1;     // its slot (where its exact initial value R0 is kept)
  float m2;   // largest |R32|^2 among the other bins
};

template <class A, int T, int NT, bool HALF> struct FwdLayout {
  using C = typename A::C;
  using E = typename A::E;
  using IO = PlanIO<A>;
  static constexpr int NW = NT / 32;
  // offsets (bytes) from the 1024-aligned base of dynamic shared memory
  static constexpr size_t w_bytes = sizeof(E) * WTab<A, T, HALF>::elems;
  static constexpr size_t tw_off = w_bytes;
  static constexpr size_t syn_off = tw_off + sizeof(C) * (T / 2);
  static constexpr size_t slot_off = syn_off + sizeof(typename IO::Syn) * T;
  static constexpr size_t ex_off = (slot_off + sizeof(Cand<A>) * 2 * NW + 15) & ~size_t(15);
  static constexpr size_t tr_off = (ex_off + 2 * sizeof(C) + 15) & ~size_t(15);
  __host__ __device__ static size_t bytes(int iters) {
    return 1024 + tr_off + sizeof(TraceSm<A>) * (size_t)iters;
  }
  // per-CTA global scratch: the FFT buffer of the half-W variant
  static constexpr size_t scratch_bytes = HALF ? sizeof(E) * (size_t)T * 2 * T : 0;
};

// ---------------------------------------------------------------------------
// filtered-exact helpers (float-float exact values, FP32 working spectrum)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void top2_insert(Top2& t, float m, int code, int slot) {
  if (m > t.m1) {
    t.m2 = t.m1;
    t.m1 = m;
    t.c1 = code;
    t.s1 = slot;
  } else {
    t.m2 = fmaxf(t.m2, m);
  }
}
__device__ __forceinline__ void top2_merge(Top2& a, const Top2& b) {
  if (b.m1 > a.m1 || (b.m1 == a.m1 && b.c1 < a.c1)) {
    a.m2 = fmaxf(a.m1, b.m2);
    a.m1 = b.m1;
    a.c1 = b.c1;
    a.s1 = b.s1;
  } else {
    a.m2 = fmaxf(a.m2, b.m1);
  }
}
__device__ __forceinline__ Top2 top2_shfl(const Top2& t, int o) {
  Top2 r;
  r.m1 = __shfl_xor_sync(0xffffffffu, t.m1, o);
  r.c1 = __shfl_xor_sync(0xffffffffu, t.c1, o);
  r.s1 = __shfl_xor_sync(0xffffffffu, t.s1, o);
  r.m2 = __shfl_xor_sync(0xffffffffu, t.m2, o);
  return r;
}

template <class A, int T, int NT, bool HALF>
__device__ __forceinline__ void forward_block(const FwdArgs& args, const CUtensorMap* tmF,
                                              const CUtensorMap* tmA, int blk, unsigned char* smem,
                                              uint64_t* mbar, unsigned& tma_phase,
                                              unsigned char* cta_scratch) {
  using C = typename A::C;
  using E = typename A::E;
  using IO = PlanIO<A>;
  using L = FwdLayout<A, T, NT, HALF>;
  using WT = WTab<A, T, HALF>;
  constexpr int T2 = 2 * T, LOGT = ilog2(T), NBINS = T * T / 2 + 2;
  constexpr int NSLOT = T * T / 2;
  constexpr int NB = NSLOT / NT;  // register-resident bins per thread
  constexpr int NW = NT / 32;
  static_assert(NSLOT % NT == 0 && NT >= 64, "slot grid");
  static_assert(NBINS == NSLOT + 2, "bins");

  E* Wsm = reinterpret_cast<E*>(smem);              // W table (and staging, and FFT if full)
  E* Z = HALF ? reinterpret_cast<E*>(cta_scratch) : Wsm;  // FFT buffer
  C* tw = reinterpret_cast<C*>(smem + L::tw_off);
  using Syn = typename IO::Syn;
  Syn* syn = reinterpret_cast<Syn*>(smem + L::syn_off);
  Cand<A>* slots = reinterpret_cast<Cand<A>*>(smem + L::slot_off);
  TraceSm<A>* tr = reinterpret_cast<TraceSm<A>*>(smem + L::tr_off);
  C* ex = reinterpret_cast<C*>(smem + L::ex_off);  // the two bins beyond the slot grid

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const PlanDev& P = args.plan;
  const fofse_block bd = args.blocks[blk];
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
      fence_proxy_async();  // earlier generic writes to this area before the async copies
      mbar_expect_tx(mbar, (unsigned)(bytesF + args.box_a * Ls));
      tma_load_2d(stF, tmF, fx0, ly0, mbar);
      tma_load_2d(stA, tmA, ax0, ly0, mbar);
    }
    bool done = false;
    for (unsigned it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(mbar, tma_phase);
    if (!done) {
      atomicOr(args.err, kErrTimeout);
      // wait (bounded again) for the copy in flight before giving up on the block
      for (unsigned it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(mbar, tma_phase);
    }
    tma_phase ^= 1u;
    if (!__syncthreads_and(done)) {
      if (tid == 0 && args.status) args.status[blk] = kBlkTimeout;
      return;
    }
  }

  // ---- 2. weighting and the packed input z = w f + j w (bit-reversed) -------
  constexpr int PER = (T * T + NT - 1) / NT;
  using Mask = typename std::conditional<(PER > 32), unsigned long long, unsigned>::type;
  float fv[PER];
  Mask use = 0;
  bool bad = false, nzf = false;
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
          use |= Mask(1) << s;
          fv[s] = f;
          bad |= !isfinite(f);
          nzf |= f != 0.f;
        }
      }
    }
  }
  int any_bad = __syncthreads_or(bad);  // the staging area may be overwritten below
  // f = 0 on the whole support: R_w = DFT(w f) is exactly zero (the packed
  // transform would leave W's rounding in it)
  const bool zero_f = !__syncthreads_or(nzf);
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int e = tid + s * NT;
    if (e < T * T) {
      const int r = e >> LOGT, c = e & (T - 1);
      C z = A::zero();
      if (use & (Mask(1) << s)) {
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

  C W0c;
  int st;
  {
  // ---- split: R_w[k] = (Z[k] + conj Z[-k]) / 2 into registers ---------------
  C R[NB];
  int kc[NB];  // x_k | code << 16
#pragma unroll
  for (int i = 0; i <= NB; ++i) {
    if (i == NB && tid >= 2) break;
    const int x = i < NB ? slot_xk<T>(tid + i * NT) : extra_xk<T>(tid);
    const int k1 = x >> (LOGT + 1), k2 = x & (T2 - 1);
    const int mx = ((T - k1) & (T - 1)) * T2 + ((T - k2) & (T - 1));
    const C a = A::load(Z, x, T), m = A::load(Z, mx, T);
    const C r = zero_f ? A::zero() : A::half(A::add(a, A::conj(m)));
    if (!A::finite(r)) bad = true;
    if (i < NB) {
      kc[i] = x | (code_of<T>(x) << 16);
      R[i] = r;
    } else {
      ex[tid] = r;
    }
  }
  any_bad |= __syncthreads_or(bad);
    build_wtab<A, T, NT, HALF>(Z, Wsm);
    __syncthreads();
    W0c = WT::at0(Wsm);
    st = FOFSE_BLK_OK;
    if (IO::w0_zero(W0c)) st = FOFSE_BLK_NO_SUPPORT;
    else if (any_bad || !IO::w0_finite(W0c)) st = FOFSE_BLK_NONFINITE;
  if (st == FOFSE_BLK_OK) {
    const auto inv = IO::inv_w0(IO::gamma(P), W0c.re);
    Cand<A> best = empty_cand<A>();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const Cand<A> c = make_cand(R[i], kc[i] >> 16);
      if (better(c, best)) best = c;
    }
    if (tid < 2) {
      const int x = extra_xk<T>(tid);
      const Cand<A> c = make_cand(ex[tid], code_of<T>(x));
      if (better(c, best)) best = c;
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
          const int x = kc[i] & 0xffff;
          const C Wm = WT::minus(Wsm, x, y);
          const C Wp = WT::plus(Wsm, x, y);
          Upd<A>::pair(R[i], c, Wm, Wp);
          const Cand<A> cd = make_cand(R[i], kc[i] >> 16);
          if (better(cd, best)) best = cd;
        }
      } else {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const C Wm = WT::minus(Wsm, kc[i] & 0xffff, y);
          Upd<A>::single(R[i], c, Wm);
          const Cand<A> cd = make_cand(R[i], kc[i] >> 16);
          if (better(cd, best)) best = cd;
        }
      }
      if (tid < 2) {  // the two bins kept in shared memory (only this thread touches its own)
        const int x = extra_xk<T>(tid);
        C r = ex[tid];
        const C Wm = WT::minus(Wsm, x, y);
        if (!sc) Upd<A>::pair(r, c, Wm, WT::plus(Wsm, x, y));
        else Upd<A>::single(r, c, Wm);
        ex[tid] = r;
        const Cand<A> cd = make_cand(r, code_of<T>(x));
        if (better(cd, best)) best = cd;
      }
    }
  }
    }
  __syncthreads();

  // ---- 5. synthesis of B (Eq. 1) and outputs ---------------------------------
  // The packed output row of a block is out_ld x out_ld (the largest block side
  // of the call); B_hat fills its top-left b x b corner, the rest is zero.
  using SA = typename IO::SynAcc;
  const int nIt = (st == FOFSE_BLK_OK) ? iters : 0;
  const int ld = args.out_ld;
  for (int p = tid; p < ld * ld; p += NT) {
    const int bm = p / ld, bn = p - bm * ld;
    float v = 0.f;
    if (bm < b && bn < b) {
      const int m = br + bm, n = br + bn;
      SA acc = 0;
      for (int i = 0; i < nIt; ++i) {
        const TraceSm<A> t = tr[i];
        const int ph = ((t.u >> 16) * m + (t.u & 0xffff) * n) & (T - 1);
        const Syn cs = syn[ph];
        acc += t.re * cs.x - t.im * cs.y;
      }
      v = (float)acc;
      if (args.out_frame) {
        const int fy = bd.y + bm, fx = bd.x + bn;
        if (fy >= 0 && fy < args.height && fx >= 0 && fx < args.width)
          args.out_frame[(size_t)fy * args.pitch + fx] = v;
      }
    }
    if (args.out_blocks) args.out_blocks[(size_t)blk * args.out_stride + p] = v;
  }
  if (args.trace) {  // the whole row: entries past this plan's iterations are zero
    for (int i = tid; i < args.trace_stride; i += NT) {
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
  __syncthreads();  // shared memory is reused by the next block
}

// Persistent kernel: each CTA takes blocks from the work queue of its plan (an
// atomic counter over the block list; entries of other plans are skipped)
// until the list is exhausted.  Without a queue, block i goes to CTA i mod grid.
template <class A, int T, int NT, int MINB, bool HALF>
__global__ void __launch_bounds__(NT, MINB) fofse_forward_kernel(const __grid_constant__ FwdArgs args,
                                                           const __grid_constant__ CUtensorMap tmF,
                                                           const __grid_constant__ CUtensorMap tmA) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t mbar;
  __shared__ int s_item;
  unsigned tma_phase = 0;
  if (args.use_tma) {
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  unsigned char* cta_scratch = nullptr;
  if (HALF)
    cta_scratch = static_cast<unsigned char*>(args.scratch) +
                  (size_t)blockIdx.x * FwdLayout<A, T, NT, HALF>::scratch_bytes;
  int next = blockIdx.x;
  for (;;) {
    int item;
    if (args.queue) {
      if (threadIdx.x == 0) s_item = atomicAdd(args.queue, 1);
      __syncthreads();
      item = s_item;
      __syncthreads();
    } else {
      item = next;
      next += gridDim.x;
    }
    if (item >= args.n_blocks) break;
    if (args.blocks[item].plan != args.plan_index) continue;
    forward_block<A, T, NT, HALF>(args, &tmF, &tmA, item, smem, &mbar, tma_phase, cta_scratch);
  }
}

template <class A, int T, int NT, int MINB, bool HALF> struct Variant {
  static constexpr size_t per_cta = FwdLayout<A, T, NT, HALF>::scratch_bytes;
  static cudaError_t prepare(int iters, size_t* smem, int* max_ctas) {
    *smem = FwdLayout<A, T, NT, HALF>::bytes(iters);
    return prepare_kernel(fofse_forward_kernel<A, T, NT, MINB, HALF>, NT, *smem, max_ctas);
  }
  static cudaError_t scratch(int iters, size_t* bytes) {
    size_t sm;
    int ctas;
    cudaError_t e = prepare(iters, &sm, &ctas);
    *bytes = e == cudaSuccess ? per_cta * (size_t)ctas : 0;
    return e;
  }
  static cudaError_t launch(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta,
                            cudaStream_t s) {
    size_t sm;
    int grid;
    cudaError_t e = prepare(a.plan.iters, &sm, &grid);
    if (e != cudaSuccess) return e;
    if (per_cta > 0) {  // one scratch slot per persistent CTA
      const size_t fit = a.scratch ? a.scratch_bytes / per_cta : 0;
      if (fit < 1) return cudaErrorInvalidValue;
      if ((size_t)grid > fit) grid = (int)fit;
    }
    if (grid > a.n_blocks) grid = a.n_blocks;
    if (grid < 1) return cudaSuccess;
    fofse_forward_kernel<A, T, NT, MINB, HALF><<<grid, NT, sm, s>>>(a, *tf, *ta);
    return cudaGetLastError();
  }
};

// Kernel choice per (precision, T).  FOFSE_FP32 runs the register-blocked
// filtered-exact kernel (fofse_fwd3.cu) when the workspace's scratch is given,
// and this all-bins float-float kernel otherwise (also FOFSE_FP32_FULLFF);
// FOFSE_FP64_VALIDATE runs it in IEEE double.
template <int T> struct Pick;
template <> struct Pick<32> {
  using FF = Variant<ArFF, 32, 128, 6, false>;
  using F64 = Variant<ArF64, 32, 128, 1, false>;
};
template <> struct Pick<64> {
  using FF = Variant<ArFF, 64, 256, 3, false>;
  using F64 = Variant<ArF64, 64, 256, 1, false>;
};
template <> struct Pick<128> {
  using FF = Variant<ArFF, 128, 512, 1, true>;
  using F64 = Variant<ArF64, 128, 512, 1, true>;
};

template <int T>
cudaError_t launch_T(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta, cudaStream_t s) {
  using Pk = Pick<T>;
  switch (a.plan.precision) {
    case FOFSE_FP64_VALIDATE: return Pk::F64::launch(a, tf, ta, s);
    case FOFSE_FP32_FULLFF: return Pk::FF::launch(a, tf, ta, s);
    default:  // FOFSE_FP32
      if (!a.scratch || a.scratch_bytes < forward_f3_scratch_bytes(a.plan))
        return Pk::FF::launch(a, tf, ta, s);
      return launch_forward_f3(a, tf, ta, s);
  }
}
// Scratch of the plan's kernel (for FOFSE_FP32, the largest launch shape).
template <int T> cudaError_t scratch_T(const PlanDev& p, size_t* bytes) {
  using Pk = Pick<T>;
  switch (p.precision) {
    case FOFSE_FP64_VALIDATE: return Pk::F64::scratch(p.iters, bytes);
    case FOFSE_FP32_FULLFF: return Pk::FF::scratch(p.iters, bytes);
    default:
      *bytes = forward_f3_scratch_bytes(p);
      return *bytes ? cudaSuccess : cudaErrorInvalidValue;
  }
}
template <int T> int variants_T(const PlanDev& p) {
  return p.precision == FOFSE_FP32 ? forward_f3_variant_count(p) : 1;
}

}  // namespace

size_t forward_scratch_bytes(const PlanDev& p) {
  if (p.basis == FOFSE_BASIS_DCT) return 0;  // everything in shared memory
  size_t b = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (p.T == 32) e = scratch_T<32>(p, &b);
  if (p.T == 64) e = scratch_T<64>(p, &b);
  if (p.T == 128) e = scratch_T<128>(p, &b);
  return e == cudaSuccess ? b : 0;
}

bool forward_needs_scratch(const PlanDev& p) { return p.T == 128 && p.basis != FOFSE_BASIS_DCT; }

int forward_variant_count(const PlanDev& p) {
  if (p.basis == FOFSE_BASIS_DCT) return forward_dct_variant_count(p);
  if (p.T == 32) return variants_T<32>(p);
  if (p.T == 64) return variants_T<64>(p);
  if (p.T == 128) return variants_T<128>(p);
  return 1;
}

cudaError_t launch_forward(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta,
                           cudaStream_t s) {
  if (a.plan.basis == FOFSE_BASIS_DCT) return launch_forward_dct(a, s);
  if (a.plan.T == 128) return launch_T<128>(a, tf, ta, s);
  if (a.plan.T == 64) return launch_T<64>(a, tf, ta, s);
  if (a.plan.T == 32) return launch_T<32>(a, tf, ta, s);
  return cudaErrorInvalidValue;
}

}  // namespace fofse
