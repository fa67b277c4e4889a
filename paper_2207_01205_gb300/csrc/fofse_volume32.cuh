// FOFSE over video volumes in FP32 with exact decisions: the product kernel of
// fofse_extrapolate_volume_batch (Sec. 1: the method carried over to
// three-dimensional sets; the transform-domain recursion of Sec. 2 on a
// T x T x Tt grid).
//
// The design is the one of the register-blocked 2-D kernel (fofse_fwd3.cuh)
// on the 3-D grid:
//   * setup: z = w f + j w per frame of the volume at bit-reversed positions,
//     a float-float 2-D FFT per frame (in chunks through shared memory), then
//     the Tt-point DFT over the frames per (k1, k2), all in a per-CTA slot of
//     global scratch; the Hermitian split gives the exact initial spectrum R0
//     (kept per held bin in the scratch, its FP32 rounding in registers) and
//     the exact W (in place; its FP32 plane copied to shared memory);
//   * held bins: the 2-D slot grid of the register-blocked kernel (one bin
//     per 2-D conjugate pair) times every temporal frequency k3.  For the four
//     2-D self-conjugate (k1, k2) both members (k3 and -k3) of a temporal pair
//     are held; the one with k3 > Tt/2 is not canonical and takes no part in
//     the selection;
//   * each iteration: the block's FP32 top-2 decide the argmax of Eq. 9 when
//     they are further apart than the running error bound allows, otherwise
//     every bin within the band is evaluated exactly and compared in
//     float-float (ties: smallest lin(k) = (k1 T + k2) Tt + k3); the
//     coefficient (Eq. 5, Eq. 14) comes from the exact value of the winner by
//     the triangular recurrence over the distinct selected indices (64-bit
//     fixed point); every held bin gets the FP32 update
//     R32[k] -= c W[k - u] + s(u) conj(c) W[k + u] from the FP32 plane of W.
// The error analysis of the 2-D kernel holds unchanged (one update of the same
// form per bin and iteration, |W[k]| <= W[0]).
#pragma once
#include "fofse_fwd3.cuh"

namespace fofse {
namespace {

struct VolArgs32 {
  int block, border, depth, Ls, Lt, iters;
  float gamma_h, gamma_l;  // gamma as a float pair
  const float2* w_ff;      // Lt x Ls x Ls: rho^d as (hi, lo)
  PlanTables tab;          // tw_ff: exp(-j 2 pi e / T), e < T/2
  const float4* twt_ff;    // Tt: exp(-j 2 pi p / Tt) as (re.h, im.h, re.l, im.l)
  const float2* syn;       // T Tt: (cos, sin)(2 pi p / (T Tt))
  const fofse_volume_block* blocks;
  int n_blocks;
  const float* video;
  const uint8_t* avail;
  int frames, height, width, pitch;
  float* out;       // n x block x block
  int32_t* path;    // n x iters x 3, nullable
  double* coef;     // n x iters x 2, nullable
  double* w0;       // n, nullable
  int32_t* status;  // n, nullable
  int* queue;       // work-queue counter (zeroed before the launch)
  void* scratch;
  size_t scratch_bytes;
};

template <int T, int TT, int NT> struct V3 {
  static constexpr int LOGT = ilog2(T), LOGTT = ilog2(TT), T2 = 2 * T;
  static constexpr int K = T * T * TT;
  static constexpr int NW = NT / 32, NS2 = T * T / 2, NB2 = NS2 / NT;
  static constexpr int NB = NB2 * TT;      // held bins per thread (threads 0, 1: + TT extras)
  static constexpr int RS = 2 * NT / T;    // rows between a thread's consecutive 2-D bins
  static constexpr int IB = NB2 / 2;       // the 2-D bin whose row is T/2 + r_t
  static constexpr int LIST = 16;          // near-tie candidates per pass
  // packed index of a bin for the exact terms: k2 | k1 << (LOGT + 1) | k3 << (2 LOGT + 2),
  // one guard bit above each field so that componentwise differences and sums
  // are one add and one AND
  static constexpr int SH1 = LOGT + 1, SH3 = 2 * LOGT + 2;
  static constexpr int PM = ((TT - 1) << SH3) | ((T - 1) << SH1) | (T - 1);
  static constexpr int PG = (TT << SH3) | (T << SH1) | T;
  static_assert((1 << LOGT) == T && (1 << LOGTT) == TT && NB2 >= 2 && NB <= 32 && NT >= 2 * TT &&
                    PM <= 0xFFFF &&
                    NW <= 32,
                "grid");
  // shared memory, bytes from a 128-aligned base
  static constexpr size_t w_bytes = sizeof(float2) * (size_t)K;     // FP32 plane of W [k3][k1][k2]
  static constexpr size_t t2_off = w_bytes;                         // uint4 [2][NW]
  static constexpr size_t red_off = t2_off + 32 * NW;               // longlong2 [NW]
  static constexpr size_t wtot_off = red_off + 16 * NW;             // int [NW]
  static constexpr size_t list_off = (wtot_off + 4 * NW + 15) & ~size_t(15);  // int4 [LIST]
  static constexpr size_t ww_off = list_off + 16 * LIST;            // float4 [NW], int2 [NW]
  static constexpr size_t nd_off = ww_off + 24 * NW;                // int
  static constexpr size_t trc_off = (nd_off + 4 + 15) & ~size_t(15);  // float4 [iters]
  __host__ __device__ static size_t try_off(int iters) { return trc_off + 16 * (size_t)iters; }
  __host__ __device__ static size_t bytes(int iters) { return 128 + try_off(iters) + 2 * (size_t)iters; }
  // per-CTA global scratch: the 3-D packed transform, then the exact W
  // ([k3][k1] rows of 2T float2: hi plane, lo plane), and R0 per held bin
  static constexpr size_t z_bytes = sizeof(float2) * (size_t)K * 2;
  static constexpr size_t scratch_bytes = z_bytes + sizeof(float4) * (size_t)(NS2 + 2) * TT;
};

// index conversions (k1, k2, k3) <-> storage
template <int T, int TT, int NT> struct VIdx {
  using G = V3<T, TT, NT>;
  __device__ __forceinline__ static int pack(int k1, int k2, int k3) {
    return (k3 << G::SH3) | (k1 << G::SH1) | k2;
  }
  // hi-plane element of the global table
  __device__ __forceinline__ static int gidx(int a) {
    return ((((a >> G::SH3) << G::LOGT) | ((a >> G::SH1) & (T - 1))) << (G::LOGT + 1)) | (a & (T - 1));
  }
  // element of the shared FP32 plane
  __device__ __forceinline__ static int sidx(int a) {
    return ((((a >> G::SH3) << G::LOGT) | ((a >> G::SH1) & (T - 1))) << G::LOGT) | (a & (T - 1));
  }
  __device__ __forceinline__ static int lin(int a) {  // (k1 T + k2) Tt + k3
    return ((((a >> G::SH1) & (T - 1)) * T + (a & (T - 1))) << G::LOGTT) | (a >> G::SH3);
  }
  __device__ __forceinline__ static int neg(int a) {  // packed -k
    return (G::PG - a) & G::PM;
  }
  __device__ __forceinline__ static bool selfconj(int a) {
    const int k1 = (a >> G::SH1) & (T - 1), k2 = a & (T - 1), k3 = a >> G::SH3;
    return (k1 & (T / 2 - 1)) == 0 && (k2 & (T / 2 - 1)) == 0 && (TT == 1 || (k3 & (TT / 2 - 1)) == 0);
  }
};

// exact W[a] (packed a): hi part from the shared FP32 plane, lo part from the
// global table
template <int T, int TT, int NT>
__device__ __forceinline__ ArFF::C vwex(const float2* Whi, const float2* Zg, int a) {
  using I = VIdx<T, TT, NT>;
  const float2 h = Whi[I::sidx(a)];
  const float2 l = Zg[I::gidx(a) + T];
  return {{h.x, l.x}, {h.y, l.y}};
}

// sum over j in {j0, j0 + stride, ...} < j1 of C_j W[x - u_j] + s_j conj(C_j) W[x + u_j]
// (float-float terms), added to sre / sim in fixed point with unit 1/scale
template <int T, int TT, int NT>
__device__ __forceinline__ void vrecur(const float2* Whi, const float2* Zg, const unsigned short* ty,
                                       const float4* tc, int x, int j0, int j1, int stride,
                                       float scale, long long& sre, long long& sim) {
  using G = V3<T, TT, NT>;
  using I = VIdx<T, TT, NT>;
  ff are = {0.f, 0.f}, aim = {0.f, 0.f};
  for (int j = j0; j < j1; j += stride) {
    const int y = ty[j];
    const float4 c4 = tc[j];
    const ArFF::C c = {{c4.x, c4.y}, {c4.z, c4.w}};
    const ArFF::C Wm = vwex<T, TT, NT>(Whi, Zg, (x + G::PG - y) & G::PM);
    ff tre, tim;
    if (!I::selfconj(y)) {
      const ArFF::C Wp = vwex<T, TT, NT>(Whi, Zg, (x + y) & G::PM);
      const ff s1 = ff_add_raw(Wm.re, Wp.re), s2 = ff_sub_raw(Wm.im, Wp.im);
      const ff s3 = ff_sub_raw(Wm.re, Wp.re), s4 = ff_add_raw(Wm.im, Wp.im);
      tre = ff_dot2(c.re, s1, ff_neg(c.im), s2);
      tim = ff_dot2(c.re, s4, c.im, s3);
    } else {
      tre = ff_mul(c.re, Wm.re);
      tim = ff_mul(c.re, Wm.im);
    }
    are = ff_add(are, tre);
    aim = ff_add(aim, tim);
  }
  if (j0 < j1) {
    sre += fx_round(are.h * scale) + fx_round(are.l * scale);
    sim += fx_round(aim.h * scale) + fx_round(aim.l * scale);
  }
}

// The rebase of the FP32 loop (out of line: it runs rarely and keeps the hot
// loop's code small): the exact values of thread tid's held bins, R0 minus
// the terms nb .. nd of the list, written over R0 in the scratch (Rx); returns
// the thread's best live bin (exact comparison, ties to the smallest lin of
// the canonical member) as (slot, 0, lin, packed index), lin 0x7fffffff if
// none.
template <int T, int TT, int NT>
__device__ __noinline__ int4 vol_rebase_bins(const float2* Whi, const float2* Zg, const unsigned short* trY,
                                             const float4* trC, float4* Rx, int tid, int nb, int nd,
                                             float scale, float iscale, unsigned dead, bool hasx, bool xdead) {
  using G = V3<T, TT, NT>;
  using I = VIdx<T, TT, NT>;
  ffc wb = {{0.f, 0.f}, {0.f, 0.f}};
  int wbc = 0x7fffffff, wbx = 0, wbs = 0;
  for (int i = 0; i <= G::NB; ++i) {
    if (i == G::NB && !hasx) break;
    const int2 kk = i < G::NB ? f3_bin<T, NT>(tid, i / TT) : f3_extra<T>(tid & 1);
    const int k3 = i < G::NB ? i % TT : tid >> 1;
    const int slot = i < G::NB ? (tid + (i / TT) * NT) * TT + k3 : (G::NS2 + (tid & 1)) * TT + k3;
    const int pk = I::pack(kk.x, kk.y, k3);
    const int cl = kk.x > T / 2 ? I::lin(I::neg(pk)) : I::lin(pk);
    const float4 r0 = Rx[slot];
    long long sre = 0, sim = 0;
    vrecur<T, TT, NT>(Whi, Zg, trY, trC, pk, nb, nd, 1, scale, sre, sim);
    const ffc v = {ff_sub(ff{r0.x, r0.y}, fx_to_ff(sre, iscale)), ff_sub(ff{r0.z, r0.w}, fx_to_ff(sim, iscale))};
    Rx[slot] = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
    const bool live = i < G::NB ? !((dead >> i) & 1u) : !xdead;
    if (live && (wbc == 0x7fffffff || exact_better(v, cl, wb, wbc))) {
      wb = v;
      wbc = cl;
      wbx = pk;
      wbs = slot;
    }
  }
  return make_int4(wbs, 0, wbc, wbx);
}

template <int T, int TT, int NT>
__device__ __forceinline__ void volume_block_f32(const VolArgs32& a, int blk, unsigned char* dsm,
                                                 float2* Whi, float2* Zg, float4* Rx) {
  using A = ArFF;
  using C = ArFF::C;
  using G = V3<T, TT, NT>;
  using I = VIdx<T, TT, NT>;
  constexpr int T2 = G::T2, LOGT = G::LOGT, NS2 = G::NS2, NB2 = G::NB2, NB = G::NB, NW = G::NW;
  constexpr int IB = G::IB, LIST = G::LIST, K = G::K;
  constexpr float kU = 5.9604644775390625e-08f;  // 2^-24
  constexpr float kDn = 1.f - 16.f * kU, kUp = 1.f + 256.f * kU, kUpB = 1.f + 16.f * kU;
  constexpr float kTiny = 7.888609052210118e-31f;
  constexpr float kTinySqrt = 8.881784197001252e-16f;
  constexpr float kA = 2.1f * kU, kB = 12.f * kU;
  constexpr int ROWB = T * 8, PLANEB = T * T * 8;  // bytes per row / plane of the FP32 plane

  uint4* t2s = reinterpret_cast<uint4*>(dsm + G::t2_off);
  longlong2* red = reinterpret_cast<longlong2*>(dsm + G::red_off);
  int* wtot = reinterpret_cast<int*>(dsm + G::wtot_off);
  int4* list = reinterpret_cast<int4*>(dsm + G::list_off);
  float4* wwv = reinterpret_cast<float4*>(dsm + G::ww_off);
  int2* wwc = reinterpret_cast<int2*>(dsm + G::ww_off + 16 * NW);
  int* nd_s = reinterpret_cast<int*>(dsm + G::nd_off);
  const int iters = a.iters;
  float4* trC = reinterpret_cast<float4*>(dsm + G::trc_off);
  // packed indices of the recurrence's terms (16 bits hold every supported grid's)
  unsigned short* trY = reinterpret_cast<unsigned short*>(dsm + G::try_off(iters));
  int nd = 0;
  // entries before nb belong to coefficients taken into R0 by a rebase
  // (below): they count for the synthesis only
  int nb = 0;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int rt = tid >> (LOGT - 1), ct = tid & (T / 2 - 1);
  const int chi = ct == 0 ? T / 2 : ct;
  const fofse_volume_block bd = a.blocks[blk];
  const int b = a.block, br = a.border, Ls = a.Ls, Lt = a.Lt, D = a.depth;

  // ---- 1. z = w f + j w per frame at bit-reversed positions; planes tau >= Lt zero ----
  bool bad = false, nzf = false;
  for (int e = tid; e < K; e += NT) {
    const int tau = e >> (2 * LOGT), r = (e >> LOGT) & (T - 1), cc = e & (T - 1);
    const int m = __brev(r) >> (32 - LOGT), n = __brev(cc) >> (32 - LOGT);
    C z = A::zero();
    if (tau < Lt && m < Ls && n < Ls) {
      const bool inB = tau == D && m >= br && m < br + b && n >= br && n < br + b;
      const int ft = bd.t - D + tau, fy = bd.y - br + m, fx = bd.x - br + n;
      if (!inB && ft >= 0 && ft < a.frames && fy >= 0 && fy < a.height && fx >= 0 && fx < a.width) {
        const long long o = ((long long)ft * a.height + fy) * a.pitch + fx;
        if (a.avail[o]) {
          const float f0 = a.video[o];
          const float2 w = a.w_ff[(tau * Ls + m) * Ls + n];
          // a non-finite sample marks the block and enters as 0, so that the
          // transform of w (W[0] among it) stays finite
          bad |= !isfinite(f0);
          const float f = isfinite(f0) ? f0 : 0.f;
          nzf |= f != 0.f;
          ff x = ff_two_prod(w.x, f);
          x.l = __fmaf_rn(w.y, f, x.l);
          z = {ff_fast_two_sum(x.h, x.l), {w.x, w.y}};
        }
      }
    }
    A::store(Zg, ((tau << LOGT) | r) * T2 + cc, T, z);
  }
  int any_bad = __syncthreads_or(bad);
  // f = 0 on the whole support: R0 = DFT(w f) is exactly zero (the packed
  // transform would leave W's rounding in it, about 1e-16 of |W|)
  const bool zero_f = !__syncthreads_or(nzf);

  // ---- 2. 2-D FFT per frame (float-float), then the DFT over the frames ----
  for (int tau = 0; tau < Lt; ++tau) fft2d_chunked<T, NT>(Zg + (size_t)tau * T * T2, Whi, a.tab, Ls);
  for (int col = tid; col < T * T; col += NT) {
    const int k1 = col >> LOGT, k2 = col & (T - 1);
    C zt[TT];
#pragma unroll
    for (int tau = 0; tau < TT; ++tau)
      zt[tau] = tau < Lt ? A::load(Zg, ((tau << LOGT) | k1) * T2 + k2, T) : A::zero();
#pragma unroll
    for (int k3 = 0; k3 < TT; ++k3) {
      C s = zt[0];
#pragma unroll
      for (int tau = 1; tau < TT; ++tau) {
        if (tau >= Lt) break;
        const float4 tw = a.twt_ff[(k3 * tau) & (TT - 1)];
        s = A::add(s, A::mul_norm(C{{tw.x, tw.z}, {tw.y, tw.w}}, zt[tau]));
      }
      A::store(Zg, ((k3 << LOGT) | k1) * T2 + k2, T, s);
    }
  }
  __syncthreads();

  // ---- 3. split: exact R0 -> scratch, FP32 copy -> registers, first top-2 ----
  // local bin i = i2 TT + k3 (i2 < NB2); the 2 TT bins of the two 2-D bins
  // outside the slot grid, (0, T/2) and (T/2, T/2), are held one per thread by
  // threads e < 2 TT (2-D bin e & 1, k3 = e >> 1) as local bin NB.  "Dead"
  // bins (the non-canonical member of a temporal pair held twice) get no key.
  float2 R32[NB];
  float2 rex = make_float2(0.f, 0.f);
  unsigned m1k = 0u, m2k = 0u;
  unsigned dead = 0u;
  const bool hasx = tid < 2 * TT;
  bool xdead = false;
  auto split_bin = [&](int k1, int k2, int k3, int slot) -> float2 {
    const int x = ((k3 << LOGT) | k1) * T2 + k2;
    const int mx = ((((TT - k3) & (TT - 1)) << LOGT) | ((T - k1) & (T - 1))) * T2 + ((T - k2) & (T - 1));
    const C za = A::load(Zg, x, T), zm = A::load(Zg, mx, T);
    const C r = zero_f ? A::zero() : A::half(A::add(za, A::conj(zm)));
    if (!A::finite(r)) bad = true;
    Rx[slot] = make_float4(r.re.h, r.re.l, r.im.h, r.im.l);
    return make_float2(r.re.h, r.im.h);
  };
#pragma unroll
  for (int i2 = 0; i2 < NB2; ++i2) {
    const int2 kk = f3_bin<T, NT>(tid, i2);
    const bool sc2 = (kk.x & (T / 2 - 1)) == 0 && (kk.y & (T / 2 - 1)) == 0;
#pragma unroll
    for (int k3 = 0; k3 < TT; ++k3) {
      const float2 r32 = split_bin(kk.x, kk.y, k3, (tid + i2 * NT) * TT + k3);
      R32[i2 * TT + k3] = r32;
      if (sc2 && TT > 1 && k3 > TT / 2) dead |= 1u << (i2 * TT + k3);
      else key_insert(m1k, m2k, m32(r32), i2 * TT + k3);
    }
  }
  if (hasx) {
    const int2 kk = f3_extra<T>(tid & 1);
    const int k3 = tid >> 1;
    rex = split_bin(kk.x, kk.y, k3, (NS2 + (tid & 1)) * TT + k3);
    xdead = TT > 1 && k3 > TT / 2;  // both extra 2-D bins are self-conjugate
    if (!xdead) key_insert(m1k, m2k, m32(rex), NB);
  }
  any_bad |= __syncthreads_or(bad);
  // exact W in place: W[k] = (Z[k] - conj Z[-k]) / (2 j) over the pairs (k, -k)
  for (int e = tid; e < K; e += NT) {
    const int k3 = e >> (2 * LOGT), k1 = (e >> LOGT) & (T - 1), k2 = e & (T - 1);
    const int m3 = (TT - k3) & (TT - 1), m1 = (T - k1) & (T - 1), m2 = (T - k2) & (T - 1);
    const int me = (((m3 << LOGT) | m1) << LOGT) | m2;
    if (e <= me) {
      const int xa = ((k3 << LOGT) | k1) * T2 + k2, xm = ((m3 << LOGT) | m1) * T2 + m2;
      const C za = A::load(Zg, xa, T), zm = A::load(Zg, xm, T);
      const C d = A::sub(za, A::conj(zm));  // W = -j d / 2
      C wv;
      wv.re = d.im;
      wv.im = d.re;
      wv = A::conj(A::half(wv));
      A::store(Zg, xa, T, wv);
      if (me != e) A::store(Zg, xm, T, A::conj(wv));
    }
  }
  __syncthreads();
  for (int e = tid; e < K; e += NT) Whi[e] = Zg[(e >> LOGT) * T2 + (e & (T - 1))];
  __syncthreads();
  const C W0c = A::load(Zg, 0, T);
  int st = FOFSE_BLK_OK;
  if (W0c.re.h == 0.f) st = FOFSE_BLK_NO_SUPPORT;
  else if (any_bad || !isfinite(W0c.re.h)) st = FOFSE_BLK_NONFINITE;

  int done_it = 0;  // iterations the loop ran (any later one repeats a zero residual's (0, 0, 0), 0)
  if (st == FOFSE_BLK_OK) {
    const ff inv = ff_div(ff{a.gamma_h, a.gamma_l}, W0c.re);
    const float W0f = W0c.re.h * (1.f + 1e-6f);
    const char* wb8 = reinterpret_cast<const char*>(Whi);
    float bnd = 0.f, prevabs = 0.f, csum = 0.f;
    int it = 0;
#pragma unroll 1
    for (; it < iters; ++it) {
      // ---- top-2 over the block (packed keys) ----
      const unsigned wm1 = __reduce_max_sync(kFull, m1k);
      const unsigned hold = __ballot_sync(kFull, m1k == wm1);
      const int ldr = __ffs(hold) - 1;
      const unsigned wm2 = __reduce_max_sync(kFull, lane == ldr ? m2k : m1k);
      uint4* ts = t2s + (it & 1) * NW;
      if (lane == 0) ts[warp] = make_uint4(wm1, wm2, (unsigned)(warp * 32 + ldr), (unsigned)nd);
      __syncthreads();
      uint4 g = ts[0];
      nd = (int)g.w;  // warp 0's count, after its update of the previous iteration
#pragma unroll
      for (int w = 1; w < NW; ++w) {
        const uint4 o = ts[w];
        if (o.x > g.x) {
          g.y = max(g.x, o.y);
          g.x = o.x;
          g.z = o.z;
        } else {
          g.y = max(g.y, o.x);
        }
      }
      const float m1 = __uint_as_float(g.x & ~kKeyMask), m2 = __uint_as_float(g.y & ~kKeyMask);
      const bool n1 = m1 >= kTiny, n2 = m2 >= kTiny;
      const float r1 = m1 * rsqrtf(n1 ? m1 : 1.f), r2 = m2 * rsqrtf(n2 ? m2 : 1.f);
      const float sM1 = n1 ? r1 : 0.f, sM1u = n1 ? r1 * kUp : kTinySqrt;
      const float sM2 = n2 ? r2 : kTinySqrt;
      bnd += kA * sM1u + kB * W0f * prevabs;
      const bool certain = (sM1 * kDn - bnd * kUpB) > (sM2 * kUp + bnd * kUpB);
      const int sh = fx_shift(4.f * W0f * csum);
      const float scale = pow2f(sh), iscale = pow2f(-sh);

      int wk1, wk2, wk3;  // the held winner
      ffc Rt;
      if (certain) {
        const int wt = (int)g.z, li = (int)(g.x & kKeyMask);
        const int2 kk = li < NB ? f3_bin<T, NT>(wt, li / TT) : f3_extra<T>(wt & 1);
        const int k3 = li < NB ? li % TT : wt >> 1;
        wk1 = kk.x;
        wk2 = kk.y;
        wk3 = k3;
        const int wslot = li < NB ? (wt + (li / TT) * NT) * TT + k3 : (NS2 + (wt & 1)) * TT + k3;
        const float4 r0 = Rx[wslot];
        long long sre = 0, sim = 0, Sr = 0, Si = 0;
        if (warp * 32 < nd - nb) {
          vrecur<T, TT, NT>(Whi, Zg, trY, trC, I::pack(wk1, wk2, wk3), nb + tid, nd, NT, scale, sre, sim);
          sre = redux_sum64(sre);
          sim = redux_sum64(sim);
        }
        if (lane == 0) red[warp] = make_longlong2(sre, sim);
        __syncthreads();
        {
          const longlong2 v = lane < NW ? red[lane] : make_longlong2(0, 0);
          Sr = redux_sum64(v.x);
          Si = redux_sum64(v.y);
        }
        Rt = {ff_sub(ff{r0.x, r0.y}, fx_to_ff(Sr, iscale)), ff_sub(ff{r0.z, r0.w}, fx_to_ff(Si, iscale))};
      } else {
        // ---- near-tie: exact values of every bin within the band ----
        const float Lb = (sM1 * kDn - 2.f * bnd * kUpB) * kDn;
        const float thr = Lb > 0.f ? Lb * Lb * kDn : -1.f;
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < NB; ++i) cnt += (!((dead >> i) & 1u) && m32(R32[i]) >= thr) ? 1 : 0;
        if (hasx && !xdead && m32(rex) >= thr) ++cnt;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += v;
        }
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int v = wtot[w];
          before += w < warp ? v : 0;
          total += v;
        }
        const int rank0 = before + incl - cnt;
        ffc wb = {{0.f, 0.f}, {0.f, 0.f}};
        int wbc = 0x7fffffff, wbx = 0;
        // a candidate: (packed held index, lin of its canonical member, slot)
        auto cand = [&](int k1, int k2, int k3, int slot) -> int4 {
          const int p = I::pack(k1, k2, k3);
          const int cl = k1 > T / 2 ? I::lin(I::neg(p)) : I::lin(p);
          return make_int4(p, cl, slot, 0);
        };
        const bool rebase = total > T * T * TT / 8;
        if (rebase) {
          // ---- rebase: the bound has grown to the size of the residual
          // (a residual that decays far, as over flat content) and nearly
          // every bin is a candidate.  Each thread evaluates its own bins
          // exactly; these values become R0 (the recurrence continues from
          // entry nb), R32 their FP32 roundings, and the bound restarts.
          {
            const int4 r = vol_rebase_bins<T, TT, NT>(Whi, Zg, trY, trC, Rx, tid, nb, nd, scale, iscale,
                                                      dead, hasx, xdead);
            wbc = r.z;
            wbx = r.w;
            const float4 v = Rx[r.x];  // the best value, as written
            wb = {{v.x, v.y}, {v.z, v.w}};
          }
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const float4 r = Rx[(tid + (i / TT) * NT) * TT + i % TT];
            R32[i] = make_float2(r.x, r.z);
          }
          if (hasx) {
            const float4 r = Rx[(NS2 + (tid & 1)) * TT + (tid >> 1)];
            rex = make_float2(r.x, r.z);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const ffc ov = ffc_shfl(wb, o);
            const int oc = __shfl_xor_sync(kFull, wbc, o), ox = __shfl_xor_sync(kFull, wbx, o);
            if (oc != 0x7fffffff && (wbc == 0x7fffffff || exact_better(ov, oc, wb, wbc))) {
              wb = ov;
              wbc = oc;
              wbx = ox;
            }
          }
          nb = nd;
          csum = 0.f;
        }
        for (int pass = 0; !rebase && pass < total; pass += LIST) {
          int r = rank0;
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            if (!((dead >> i) & 1u) && m32(R32[i]) >= thr) {
              if (r >= pass && r < pass + LIST) {
                const int2 kk = f3_bin<T, NT>(tid, i / TT);
                list[r - pass] = cand(kk.x, kk.y, i % TT, (tid + (i / TT) * NT) * TT + i % TT);
              }
              ++r;
            }
          }
          if (hasx && !xdead && m32(rex) >= thr && r >= pass && r < pass + LIST) {
            const int2 kk = f3_extra<T>(tid & 1);
            list[r - pass] = cand(kk.x, kk.y, tid >> 1, (NS2 + (tid & 1)) * TT + (tid >> 1));
          }
          __syncthreads();
          const int n = min(LIST, total - pass);
          for (int c = warp; c < n; c += NW) {
            const int4 e = list[c];
            const float4 r0 = Rx[e.z];
            long long sre = 0, sim = 0;
            vrecur<T, TT, NT>(Whi, Zg, trY, trC, e.x, nb + lane, nd, 32, scale, sre, sim);
            sre = redux_sum64(sre);
            sim = redux_sum64(sim);
            const ffc v = {ff_sub(ff{r0.x, r0.y}, fx_to_ff(sre, iscale)),
                           ff_sub(ff{r0.z, r0.w}, fx_to_ff(sim, iscale))};
            if (wbc == 0x7fffffff || exact_better(v, e.y, wb, wbc)) {
              wb = v;
              wbc = e.y;
              wbx = e.x;
            }
          }
          __syncthreads();
        }
        if (lane == 0) {
          wwv[warp] = make_float4(wb.re.h, wb.re.l, wb.im.h, wb.im.l);
          wwc[warp] = make_int2(wbc, wbx);
        }
        __syncthreads();
        int wcode = 0x7fffffff, wx = 0;
        Rt = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int2 cs = wwc[w];
          if (cs.x == 0x7fffffff) continue;
          const float4 v4 = wwv[w];
          const ffc v = {{v4.x, v4.y}, {v4.z, v4.w}};
          if (wcode == 0x7fffffff || exact_better(v, cs.x, Rt, wcode)) {
            Rt = v;
            wcode = cs.x;
            wx = cs.y;
          }
        }
        wk1 = (wx >> G::SH1) & (T - 1);
        wk2 = wx & (T - 1);
        wk3 = wx >> G::SH3;
        // after a rebase the bound restarts: the roundings of the new R0 to
        // FP32 (u of the largest value, the winner's) are covered by the
        // first increment, as for the first R0
        if (rebase) bnd = kA * (fabsf(Rt.re.h) + fabsf(Rt.im.h)) * kUp;
      }
      // ---- exact coefficient (Eq. 5, Eq. 14) of the held winner ----
      const int wp = I::pack(wk1, wk2, wk3);
      const bool mir = wk1 > T / 2;  // the held bin is the mirror of the canonical u
      const int up = mir ? I::neg(wp) : wp;
      const bool sc = I::selfconj(wp);
      C c;
      c.re = ff_mul(Rt.re, inv);
      c.im = sc ? ff{0.f, 0.f} : ff_mul(Rt.im, inv);
      // ---- record: the output path and coefficient, the recurrence's term ----
      if (warp == 0) {
        const float4 cc = mir ? make_float4(c.re.h, c.re.l, -c.im.h, -c.im.l)
                              : make_float4(c.re.h, c.re.l, c.im.h, c.im.l);
        int pos = -1;
        for (int j0 = nb; j0 < nd; j0 += 32) {
          const int j = j0 + lane;
          const unsigned hit = __ballot_sync(kFull, j < nd && trY[j] == up);
          if (hit) {
            pos = j0 + __ffs(hit) - 1;
            break;
          }
        }
        if (lane == 0) {
          if (pos >= 0) {
            const float4 o = trC[pos];
            const ff sr = ff_add(ff{o.x, o.y}, ff{cc.x, cc.y}), si = ff_add(ff{o.z, o.w}, ff{cc.z, cc.w});
            trC[pos] = make_float4(sr.h, sr.l, si.h, si.l);
          } else {
            trY[nd] = (unsigned short)up;
            trC[nd] = cc;
          }
          const size_t o = (size_t)blk * iters + it;
          if (a.path) {
            a.path[3 * o] = (up >> G::SH1) & (T - 1);
            a.path[3 * o + 1] = up & (T - 1);
            a.path[3 * o + 2] = up >> G::SH3;
          }
          if (a.coef) {
            a.coef[2 * o] = (double)cc.x + (double)cc.y;
            a.coef[2 * o + 1] = (double)cc.z + (double)cc.w;
          }
        }
        if (pos < 0) ++nd;
      }
      // The winner is the exact maximum, so an exactly zero winner means a
      // zero residual in every bin: every later iteration selects the
      // smallest index, (0, 0, 0) (which this one did), with a zero
      // coefficient; they are written as such at the end instead of being run.
      if (Rt.re.h == 0.f && Rt.re.l == 0.f && Rt.im.h == 0.f && Rt.im.l == 0.f) {
        ++it;
        break;
      }
      // ---- FP32 update of the working spectrum + next top-2 keys ----
      const float p = c.re.h, q = c.im.h;
      prevabs = fabsf(p) + fabsf(q);
      csum += prevabs;
      // byte offsets in the FP32 plane [k3][k1][k2]: per 2-D bin the row, per
      // k3 the plane, per thread the column
      const int rm0 = ((rt - wk1) & (T - 1)) * ROWB, rp0 = ((rt + wk1) & (T - 1)) * ROWB;
      const int pm0 = ((-wk3) & (TT - 1)) * PLANEB, pp0 = (wk3 & (TT - 1)) * PLANEB;
      const int cml = ((ct - wk2) & (T - 1)) << 3, cmh = ((chi - wk2) & (T - 1)) << 3;
      const int cpl = ((ct + wk2) & (T - 1)) << 3, cph = ((chi + wk2) & (T - 1)) << 3;
      unsigned k1a = 0u, k2a = 0u;
      const unsigned long long npp = f3_pair(-p);
#pragma unroll
      for (int i2 = 0; i2 < NB2; ++i2) {
        const int rowm = (rm0 + i2 * G::RS * ROWB) & (PLANEB - 1);
        const int rowp = (rp0 + i2 * G::RS * ROWB) & (PLANEB - 1);
        const int colm = i2 < IB ? cml : (i2 == IB ? (rt > 0 ? cmh : cml) : cmh);
        const int colp = i2 < IB ? cpl : (i2 == IB ? (rt > 0 ? cph : cpl) : cph);
#pragma unroll
        for (int k3 = 0; k3 < TT; ++k3) {
          const int i = i2 * TT + k3;
          const int plm = (pm0 + k3 * PLANEB) & (TT * PLANEB - 1);
          const float2 Wm = *reinterpret_cast<const float2*>(wb8 + (plm + rowm + colm));
          if (!sc) {
            const int plp = (pp0 + k3 * PLANEB) & (TT * PLANEB - 1);
            const float2 Wp = *reinterpret_cast<const float2*>(wb8 + (plp + rowp + colp));
            f3_update_bin(R32[i], Wm, Wp, q, npp);
          } else {
            f3_update_bin_sc(R32[i], Wm, npp);
          }
          // the bins that can be dead are those of the 2-D self-conjugate
          // (k1, k2) held by thread 0 (rows 0 and T/2 of column 0)
          const bool maybe_dead = TT > 1 && k3 > TT / 2 && (i2 == 0 || i2 * G::RS == T / 2);
          if (!(maybe_dead && ((dead >> i) & 1u))) key_insert(k1a, k2a, m32(R32[i]), i);
        }
      }
      if (hasx) {
        const int2 kk = f3_extra<T>(tid & 1);
        const int k3 = tid >> 1;
        const int sm = ((((k3 - wk3) & (TT - 1)) << LOGT) | ((kk.x - wk1) & (T - 1))) * T + ((kk.y - wk2) & (T - 1));
        const float2 Wm = Whi[sm];
        float2 Wp = make_float2(0.f, 0.f);
        if (!sc) {
          const int sp = ((((k3 + wk3) & (TT - 1)) << LOGT) | ((kk.x + wk1) & (T - 1))) * T + ((kk.y + wk2) & (T - 1));
          Wp = Whi[sp];
        }
        const float aa = Wm.x + Wp.x, bb = Wm.y - Wp.y, cc = Wm.y + Wp.y, d = Wm.x - Wp.x;
        rex.x = __fmaf_rn(-p, aa, __fmaf_rn(q, bb, rex.x));
        rex.y = __fmaf_rn(-p, cc, __fmaf_rn(-q, d, rex.y));
        if (!xdead) key_insert(k1a, k2a, m32(rex), NB);
      }
      m1k = k1a;
      m2k = k2a;
    }
    done_it = it;
  }
  if (tid == 0) *nd_s = nd;  // thread 0 is in warp 0, which holds the count
  __syncthreads();

  // ---- synthesis of B in frame tau = depth (Eq. 1) from the exact coefficients ----
  const int nTerms = (st == FOFSE_BLK_OK) ? *nd_s : 0;
  for (int pidx = tid; pidx < b * b; pidx += NT) {
    const int bm = pidx / b, bn = pidx - bm * b;
    const int m = br + bm, n = br + bn;
    float acc = 0.f;
    for (int i = 0; i < nTerms; ++i) {
      const int yy = trY[i];
      const int u1 = (yy >> G::SH1) & (T - 1), u2 = yy & (T - 1), u3 = yy >> G::SH3;
      const float4 c4 = trC[i];
      const float mult = I::selfconj(yy) ? 1.f : 2.f;
      const int ph = ((((u1 * m + u2 * n) & (T - 1)) << G::LOGTT) + ((u3 * D) & (TT - 1)) * T) & (T * TT - 1);
      const float2 cs = __ldg(&a.syn[ph]);
      acc += mult * (c4.x * cs.x - c4.z * cs.y);
    }
    a.out[(size_t)blk * b * b + pidx] = acc;
  }
  {  // the iterations that did not run: (0, 0, 0) with a zero coefficient
    for (int i = done_it + tid; i < iters; i += NT) {
      const size_t o = (size_t)blk * iters + i;
      if (a.path) a.path[3 * o] = a.path[3 * o + 1] = a.path[3 * o + 2] = 0;
      if (a.coef) a.coef[2 * o] = a.coef[2 * o + 1] = 0.0;
    }
  }
  if (tid == 0) {
    // W[0] as computed (a block with a non-finite sample still has its weights)
    if (a.w0) a.w0[blk] = st == FOFSE_BLK_NO_SUPPORT ? 0.0 : (double)W0c.re.h + (double)W0c.re.l;
    if (a.status) a.status[blk] = st;
  }
  __syncthreads();
}

template <int T, int TT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fofse_volume_f32_kernel(const __grid_constant__ VolArgs32 a) {
  using G = V3<T, TT, NT>;
  extern __shared__ __align__(16) unsigned char smem_v32[];  // 16-byte slots, no TMA
  unsigned char* dsm = smem_v32;
  __shared__ int s_item;
  float2* Whi = reinterpret_cast<float2*>(dsm);
  unsigned char* slot = static_cast<unsigned char*>(a.scratch) + (size_t)blockIdx.x * G::scratch_bytes;
  float2* Zg = reinterpret_cast<float2*>(slot);
  float4* Rx = reinterpret_cast<float4*>(slot + G::z_bytes);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.n_blocks) break;
    volume_block_f32<T, TT, NT>(a, item, dsm, Whi, Zg, Rx);
  }
}

// Launch shapes: threads per block NT (held bins per thread NB = K / (2 NT))
// and the minimum resident blocks per SM that the register allocation is held
// to.  Shape 0: 32 bins per thread with at least two warps (measured best or
// tied on every grid: 1.20 ms against 1.26 ms with 16 bins per thread on the
// 32 x 32 x 4 video batch, where it fits six CTAs per SM and the 804 blocks in
// one wave); shape 1: twice the threads; shape 2: half the threads.  A shape
// exists where the 2-D slot grid still gives every thread two rows
// (NB2 >= 2), a block has at least one warp and a thread at most 32 bins.
template <int T, int TT, int V> struct V3Shape {
  static constexpr int K = T * T * TT;
  static constexpr int NTA = K / 64 > 64 ? K / 64 : 64;
  static constexpr int NT = V == 0 ? NTA : (V == 1 ? NTA * 2 : NTA / 2);
  static constexpr bool valid = NT >= 32 && NT <= 1024 && NT <= T * T / 4 && K / (2 * NT) <= 32 &&
                                K / (2 * NT) >= 1;
  static constexpr int NB = K / (2 * NT);
  static constexpr int REGS = 2 * NB + 104 > 255 ? 255 : 2 * NB + 104;  // register target
  static constexpr int BY_REGS = 65536 / (NT * ((REGS + 7) & ~7));
  // the SM's 228 KB over W's plane, about 5 KB of slots and term list (200
  // iterations) and the 1 KB the hardware reserves per CTA
  static constexpr int BY_SMEM = 233472 / (K * 8 + 6 * 1024);
  static constexpr int MINB0 = BY_REGS < BY_SMEM ? BY_REGS : BY_SMEM;
  static constexpr int MINB = MINB0 < 1 ? 1 : (MINB0 > 8 ? 8 : MINB0);
};

template <int T, int TT, int V> struct VariantV3 {
  static constexpr int NT = V3Shape<T, TT, V>::NT;
  static constexpr int MINB = V3Shape<T, TT, V>::MINB;
  using G = V3<T, TT, NT>;
  static constexpr size_t per_cta = G::scratch_bytes;
  static cudaError_t prepare(int iters, size_t* smem, int* max_ctas) {
    *smem = G::bytes(iters);
    return prepare_kernel(fofse_volume_f32_kernel<T, TT, NT, MINB>, NT, *smem, max_ctas);
  }
  static cudaError_t scratch(int iters, size_t* bytes) {
    size_t sm;
    int ctas;
    cudaError_t e = prepare(iters, &sm, &ctas);
    *bytes = e == cudaSuccess ? per_cta * (size_t)ctas : 0;
    return e;
  }
  static cudaError_t launch(const VolArgs32& a, cudaStream_t s) {
    size_t sm;
    int grid;
    cudaError_t e = prepare(a.iters, &sm, &grid);
    if (e != cudaSuccess) return e;
    const size_t fit = a.scratch ? a.scratch_bytes / per_cta : 0;
    if (fit < 1) return cudaErrorInvalidValue;
    if ((size_t)grid > fit) grid = (int)fit;
    if (grid > a.n_blocks) grid = a.n_blocks;
    if (grid < 1) return cudaSuccess;
    fofse_volume_f32_kernel<T, TT, NT, MINB><<<grid, NT, sm, s>>>(a);
    return cudaGetLastError();
  }
};

}  // namespace
}  // namespace fofse
