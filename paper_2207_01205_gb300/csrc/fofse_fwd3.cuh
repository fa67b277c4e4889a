// Filtered-exact forward kernel, register-blocked layout: the product kernel
// of FOFSE_FP32 when a workspace is given (instantiated in fofse_fwd3.cu for
// the constant compensation of Eq. 14 and in fofse_ofse.cu for OFSE's
// compensation of Eq. 10-13).
//
// The method is the one of the filtered variant in fofse_fwd.cu: the working
// spectrum R32 is FP32 (registers) with a running bound B on its distance to
// the exact recursion; the block's FP32 top-2 decide the argmax of Eq. 9 when
// they are further apart than the bound allows, otherwise every bin inside
// the band is evaluated exactly and compared in float-float; the coefficient
// of Eq. 5 / Eq. 14 always comes from the exact value of the winner, given by
// the triangular recurrence
//   R~[k] = R0[k] - sum_{j<i} (c_j W[k - u_j] + s_j conj(c_j) W[k + u_j]).
// What this layout changes is the cost of each iteration:
//   * slot grid.  Bin i of thread t is the bin in row r_t + i*RS, column c_t of
//     the half spectrum (r_t = t / (T/2), c_t = t mod (T/2), RS = 2 NT / T).
//     The shifted gathers W[k -+ u] of one thread are then one base per
//     iteration plus a compile-time step: one add and one AND per gather.
//     Column 0 holds the bins (r, 0) for r <= T/2 and, in rows r > T/2, the
//     bins (r, T/2) (mirrors of the canonical (T - r, T/2)); (0, T/2) and
//     (T/2, T/2) are held by threads 0 and 1 outside the grid.
//   * W's FP32 plane in shared memory with row stride T (static shared memory
//     for T <= 64, so that its address folds into the load instruction).
//   * top-2 tracking with packed keys: the bits of |R32|^2 with the low seven
//     replaced by the bin's local index, three unsigned min/max per bin, the
//     warp's top-2 by redux.sync.
//   * the recurrence sum accumulated in 64-bit fixed point: each float-float
//     term is rounded to a multiple of 2^-s, s chosen per iteration from the
//     running sum of the coefficient magnitudes so that no partial sum can
//     overflow; warp and block reductions are then exact integer adds.
//
// Error bound (first order, u = 2^-24, |W[k]| <= W[0]).  One FP32 update
// R.x <- fma(-p, a, fma(q, b, R.x)) with a = Wm.x + Wp.x, b = Wm.y - Wp.y (and
// the same shape for R.y) errs by at most 2u |R_new| + 5.66u (|p| + |q|) W[0];
// rounding W and c to FP32 adds 2u (|p| + |q|) W[0] each.  The kernel adds
// 2.1u max|R32| + 12u (|p| + |q|) W[0] to B per iteration (max|R32| after the
// update bounds |R_new|; the first term of the first iteration also covers the
// rounding of R0).
#pragma once
#include "fofse_fwd_common.cuh"

namespace fofse {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int T, int NT> struct F3 {
  static constexpr int LOGT = ilog2(T), T2 = 2 * T;
  static constexpr int NW = NT / 32, NSLOT = T * T / 2, NB = NSLOT / NT;
  static constexpr int RS = 2 * NT / T;  // rows between a thread's consecutive bins
  static constexpr int IB = NB / 2;      // the bin whose row is T/2 + r_t
  static constexpr int LIST = 32;        // near-tie candidates per pass
  // near-tie candidates beyond which the exact values of every bin are taken
  // as a new R0 instead (evaluating them all costs about as much)
  static constexpr int REBASE = NSLOT / 4;
  static constexpr bool STATIC_W = T <= 64;
  static_assert(NSLOT % NT == 0 && NB >= 2 && NB <= 64 && NW >= 1 && (NW & (NW - 1)) == 0,
                "slot grid");
  // dynamic shared memory, bytes from a 128-aligned base
  static constexpr size_t w_bytes = STATIC_W ? 0 : sizeof(float2) * (size_t)T * T;
  static constexpr size_t t2_off = w_bytes;                                // uint4 [2][NW]
  static constexpr size_t red_off = t2_off + 32 * NW;                      // longlong2 [2][NW]
  static constexpr size_t wtot_off = red_off + 32 * NW;                    // int [NW]
  static constexpr size_t list_off = (wtot_off + 4 * NW + 15) & ~size_t(15);  // int4 [LIST]
  static constexpr size_t ww_off = list_off + 16 * LIST;                   // float4 [NW], int2 [NW]
  static constexpr size_t nd_off = ww_off + 24 * NW;                       // int: terms in the list
  static constexpr size_t trc_off = (nd_off + 4 + 15) & ~size_t(15);       // float4 [iters]
  __host__ __device__ static size_t try_off(int iters) { return trc_off + 16 * (size_t)iters; }
  // Where W's FP32 plane is dynamic (fft_size 128, one block per SM), the low
  // parts of the exact W also live in shared memory when they fit, as the
  // Hermitian half k2 <= T/2 (W[-k] = conj(W[k]) holds bit for bit in the
  // table the setup builds), so that the recurrence reads no global memory
  // for W.
  static constexpr int LO_LD = T / 2 + 1;
  static constexpr size_t lo_bytes = sizeof(float2) * (size_t)T * LO_LD;
  __host__ __device__ static size_t lo_off(int iters) {
    return (try_off(iters) + 2 * (((size_t)iters + 7) & ~size_t(7)) + 15) & ~size_t(15);
  }
  __host__ __device__ static bool lo_smem(int iters) {
    return !STATIC_W && 128 + lo_off(iters) + lo_bytes <= 231 * 1024;
  }
  __host__ __device__ static size_t bytes(int iters) {  // + alignment slack
    return 128 + (lo_smem(iters) ? lo_off(iters) + lo_bytes
                                 : try_off(iters) + 2 * (((size_t)iters + 7) & ~size_t(7)));
  }
  // per-CTA global scratch: the packed FFT (then the exact W), exact R0 per slot
  static constexpr size_t z_bytes = sizeof(float2) * (size_t)T * 2 * T;
  static constexpr size_t scratch_bytes = z_bytes + sizeof(float4) * (size_t)(NSLOT + 2);
  // OFSE adds the same two regions again: the packed FFT of w^2 f + j w^2
  // (then the exact V = DFT(w^2)), and the exact Q0 = DFT(w^2 f) per slot
  static constexpr size_t scratch_bytes_ofse = 2 * scratch_bytes;
};

// held bin (k1, k2) of local bin i of thread t
template <int T, int NT> __device__ __forceinline__ int2 f3_bin(int t, int i) {
  const int k1 = (t >> (ilog2(T) - 1)) + i * F3<T, NT>::RS;
  const int c = t & (T / 2 - 1);
  return make_int2(k1, (c == 0 && k1 > T / 2) ? T / 2 : c);
}
// the two bins outside the grid, held by threads 0 and 1
template <int T> __device__ __forceinline__ int2 f3_extra(int e) {
  return make_int2(e ? T / 2 : 0, T / 2);
}
// slot (tid + i * NT, or NSLOT + e for the extras) of a held bin (k1, k2)
template <int T, int NT> __device__ __forceinline__ int f3_slot(int k1, int k2) {
  using G = F3<T, NT>;
  if (k2 == T / 2 && (k1 == 0 || k1 == T / 2)) return G::NSLOT + (k1 ? 1 : 0);
  const int ct = k2 == T / 2 ? 0 : k2;
  const int t = (k1 & (G::RS - 1)) * (T / 2) + ct;
  return t + (k1 / G::RS) * NT;
}
// 2 * canonical index + (the held bin is the mirror of the canonical one)
template <int T> __device__ __forceinline__ int f3_code(int k1, int k2) {
  const bool mir = k1 > T / 2;
  const int canon = mir ? (((T - k1) & (T - 1)) * T + ((T - k2) & (T - 1))) : (k1 * T + k2);
  return canon * 2 + (mir ? 1 : 0);
}

// low bits of a key that hold the bin's local index (up to 64 bins per thread
// plus one extra); truncating them lowers |R32|^2 by less than 2^-16 relative
constexpr unsigned kKeyMask = 127u;

__device__ __forceinline__ void key_insert(unsigned& k1, unsigned& k2, float m, int i) {
  const unsigned key = (__float_as_uint(m) & ~kKeyMask) | (unsigned)i;  // m >= 0: monotone bits
  k2 = max(k2, min(k1, key));
  k1 = max(k1, key);
}

// The FP32 update of one held bin, R -= c W[k - u] + conj(c) W[k + u] with
// c = p + j q:
//   R.x = fma(-p, Wm.x + Wp.x, fma( q, Wm.y - Wp.y, R.x))
//   R.y = fma(-p, Wm.y + Wp.y, fma(-q, Wm.x - Wp.x, R.y))
// with the sum, the difference and the p terms as packed FP32x2 operations
// (each lane rounds as the scalar instruction does, so the result is that of
// the scalar form bit for bit).  npp = (-p, -p) as one 64-bit pair.
__device__ __forceinline__ unsigned long long f3_pair(float v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void f3_update_bin(float2& R, float2 Wm, float2 Wp, float q,
                                              unsigned long long npp) {
  asm("{\n\t.reg .b64 m, w, s, d, r;\n\t.reg .f32 dx, dy, rx, ry;\n\t"
      "mov.b64 m, {%2, %3};\n\tmov.b64 w, {%4, %5};\n\t"
      "add.rn.f32x2 s, m, w;\n\tsub.rn.f32x2 d, m, w;\n\t"
      "mov.b64 {dx, dy}, d;\n\t"
      "fma.rn.f32 rx, %6, dy, %0;\n\tfma.rn.f32 ry, %7, dx, %1;\n\t"
      "mov.b64 r, {rx, ry};\n\tfma.rn.f32x2 r, %8, s, r;\n\t"
      "mov.b64 {%0, %1}, r;\n\t}"
      : "+f"(R.x), "+f"(R.y)
      : "f"(Wm.x), "f"(Wm.y), "f"(Wp.x), "f"(Wp.y), "f"(q), "f"(-q), "l"(npp));
}
// the same for a self-conjugate u (c real): R = fma(-p, Wm, R)
__device__ __forceinline__ void f3_update_bin_sc(float2& R, float2 Wm, unsigned long long npp) {
  asm("{\n\t.reg .b64 m, r;\n\tmov.b64 m, {%2, %3};\n\tmov.b64 r, {%0, %1};\n\t"
      "fma.rn.f32x2 r, %4, m, r;\n\tmov.b64 {%0, %1}, r;\n\t}"
      : "+f"(R.x), "+f"(R.y)
      : "f"(Wm.x), "f"(Wm.y), "l"(npp));
}

// 2^s with bound * 2^s < 2^62 and s <= 126 (bound finite, >= 0)
__device__ __forceinline__ int fx_shift(float bound) {
  const int eb = (__float_as_int(bound) >> 23) & 0xff;  // bound < 2^(eb - 126)
  return min(188 - eb, 126);
}
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((s + 127) << 23); }
// Conversions between FP32 and the 64-bit fixed-point sums use 32-bit
// conversion instructions only (the 64-bit ones go through the FP64 pipe,
// two lanes per clock on this GPU).
// Nearest integer to v, |v| < 2^62.  For |v| >= 2^30, v is a multiple of 2^7,
// so v = h 2^31 + r with h = floor(v / 2^31) and r = v - h 2^31 in [0, 2^31)
// both exact in FP32.
__device__ __forceinline__ long long fx_round(float v) {
  const bool big = fabsf(v) >= 1073741824.f;                   // 2^30
  const float h = floorf(v * 4.656612873077393e-10f);          // v / 2^31
  const float r = __fmaf_rn(-h, 2147483648.f, v);
  const long long vb = ((long long)__float2int_rn(h) << 31) + (long long)__float2uint_rn(r);
  const long long vs = (long long)__float2int_rn(v);
  return big ? vb : vs;
}
// Float-float value of v / scale (|v| < 2^62): v split into a signed 20-bit
// limb and two 21-bit limbs, each exact in FP32, summed in float-float.
__device__ __forceinline__ ff fx_to_ff(long long v, float inv_scale) {
  const int a = (int)(v >> 42);
  const int b = (int)((v >> 21) & 0x1FFFFF), c = (int)(v & 0x1FFFFF);
  const ff t = ff_add(ff_two_sum(__int2float_rn(a) * 4398046511104.f, __int2float_rn(b) * 2097152.f),
                      ff{__int2float_rn(c), 0.f});
  return {t.h * inv_scale, t.l * inv_scale};
}
__device__ __forceinline__ void warp_sum64(long long& a, long long& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    b += __shfl_xor_sync(kFull, b, o);
  }
}
// The same sum by redux.sync on three 21-bit limbs (|v| < 2^62: the limb sums
// of 32 lanes fit in 32 bits); shorter latency than five shuffle rounds.
__device__ __forceinline__ long long redux_sum64(long long v) {
  const int l0 = (int)(v & 0x1FFFFF), l1 = (int)((v >> 21) & 0x1FFFFF), l2 = (int)(v >> 42);
  const long long s0 = __reduce_add_sync(kFull, l0), s1 = __reduce_add_sync(kFull, l1);
  const long long s2 = __reduce_add_sync(kFull, l2);
  return s2 * 4398046511104LL + s1 * 2097152LL + s0;  // 2^42, 2^21
}

// sum over j in {j0, j0 + stride, ...} < j1 of c_j W[k - u_j] + s_j conj(c_j) W[k + u_j]
// (float-float terms, exact W from the global table), added to sre / sim in
// fixed point with unit 1/scale.  HI_GLOBAL: both planes of the table are
// read from Zg (a table without an FP32 copy in shared memory).  Wlo: the low
// parts as the Hermitian half in shared memory (row stride T/2 + 1), or null
// for the global table.
template <int T, bool HI_GLOBAL = false>
__device__ __forceinline__ void recur_fixed(const float2* Whi, const float2* Zg, const float2* Wlo,
                                            const short* ty, const float4* tc, int x, int j0, int j1,
                                            int stride, float scale, long long& sre, long long& sim) {
  constexpr int LOGT = ilog2(T), M = (T - 1) * 2 * T + (T - 1), LD = T / 2 + 1;
  // exact W: hi part from the FP32 plane in shared memory (row stride T), lo
  // part from the global table (two planes of row stride 2T) or the half
  // plane in shared memory (k2 > T/2: the conjugate of the mirror -k)
  auto wex = [&](int a) -> ArFF::C {  // a = packed a1 * 2T + a2
    const int a1 = a >> (LOGT + 1), a2 = a & (T - 1);
    const float2 h = HI_GLOBAL ? Zg[a] : Whi[(a1 << LOGT) | a2];
    float2 l;
    if (Wlo) {
      const bool mr = a2 > T / 2;
      l = Wlo[(mr ? (T - a1) & (T - 1) : a1) * LD + (mr ? T - a2 : a2)];
      if (mr) l.y = -l.y;
    } else {
      l = Zg[a + T];
    }
    return {{h.x, l.x}, {h.y, l.y}};
  };
  // a thread's few terms are summed in float-float and converted once
  ff are = {0.f, 0.f}, aim = {0.f, 0.f};
  for (int j = j0; j < j1; j += stride) {
    const int y = ty[j];
    const float4 c4 = tc[j];
    const ArFF::C c = {{c4.x, c4.y}, {c4.z, c4.w}};
    const int u1 = y >> (ilog2(T) + 1), u2 = y & (2 * T - 1);
    const bool sc = ((u1 & (T / 2 - 1)) == 0) && ((u2 & (T / 2 - 1)) == 0);
    const ArFF::C Wm = wex((x + T - y) & M);
    ff tre, tim;
    if (!sc) {
      const ArFF::C Wp = wex((x + y) & M);
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

// 2-D FFT of the packed block, which sits in the per-CTA global scratch
// (two-plane float-float layout, input at bit-reversed positions, storage
// rows brev(m), m < Ls, nonzero), through shared memory: the row pass in
// chunks of T/2 storage rows, the column pass in chunks of T/2 columns, each
// chunk loaded into `buf` (8 T^2 bytes: the region of W's FP32 plane, free
// during the setup), transformed there by decimation-in-time stages (radix-4
// pairs of stages from fft_size 64 on, radix-2 otherwise) and written
// back.  Two reads and three writes of the scratch instead of one read and
// one write per stage.  Twiddles exp(-j 2 pi e / T) come from the plan table.
// exp(-j 2 pi e / T) for 0 <= e < T (the plan's table covers e < T/2; the
// rest is its negative)
template <int T> __device__ __forceinline__ ArFF::C twiddle_full(const PlanTables& tab, int e) {
  const ArFF::C w = PlanIO<ArFF>::twiddle(tab, e & (T / 2 - 1));
  return e >= T / 2 ? ArFF::C{ff_neg(w.re), ff_neg(w.im)} : w;
}

// One radix-4 decimation-in-time butterfly (two radix-2 stages of distance h
// and 2h merged): inputs at offsets 0, h, 2h, 3h (stride `st` elements apart
// per unit of h), twiddles W^j, W^2j, W^3j with W = exp(-j 2 pi / (4h)).
template <int T>
__device__ __forceinline__ void radix4(float2* buf, int i0, int hs, int ld, int e1, const PlanTables& tab) {
  using A = ArFF;
  using C = ArFF::C;
  const C a = A::load(buf, i0, ld);
  C b = A::load(buf, i0 + hs, ld), c = A::load(buf, i0 + 2 * hs, ld), d = A::load(buf, i0 + 3 * hs, ld);
  if (e1 != 0) {
    b = A::mul_norm(twiddle_full<T>(tab, 2 * e1), b);
    c = A::mul_norm(twiddle_full<T>(tab, e1), c);
    d = A::mul_norm(twiddle_full<T>(tab, 3 * e1), d);
  }
  const C s0 = A::add(a, b), s1 = A::sub(a, b), s2 = A::add(c, d), s3 = A::sub(c, d);
  const C is3 = {s3.im, ff_neg(s3.re)};  // -j (c - d)
  A::store(buf, i0, ld, A::add(s0, s2));
  A::store(buf, i0 + hs, ld, A::add(s1, is3));
  A::store(buf, i0 + 2 * hs, ld, A::sub(s0, s2));
  A::store(buf, i0 + 3 * hs, ld, A::sub(s1, is3));
}

template <int T, int NT>
__device__ __forceinline__ void fft2d_chunked(float2* Z, float2* buf, const PlanTables& tab, int Ls) {
  using A = ArFF;
  using C = ArFF::C;
  using IO = PlanIO<A>;
  constexpr int LOGT = ilog2(T), T2 = 2 * T, CH = T / 2;
  // radix-4 stages from fft_size 64 on (measured faster there; at 32, with
  // one warp per block, slower than radix-2)
  constexpr int R4 = T >= 64 ? (LOGT & ~1) : 0;  // stages done in radix-4 pairs
  const int tid = threadIdx.x;
  // ---- rows: chunk rows are storage rows brev(rr), rr in [r0, r0 + CH) ----
#pragma unroll 1
  for (int r0 = 0; r0 < Ls; r0 += CH) {
    const int nr = min(CH, Ls - r0);
    for (int e = tid; e < nr * T; e += NT) {
      const int lr = e >> LOGT, c = e & (T - 1);
      const int row = __brev(r0 + lr) >> (32 - LOGT);
      A::store(buf, lr * T2 + c, T, A::load(Z, row * T2 + c, T));
    }
    __syncthreads();
#pragma unroll 1
    for (int lh = 0; lh + 1 < R4; lh += 2) {
      const int h = 1 << lh;
      for (int it = tid; it < nr * (T / 4); it += NT) {
        const int lr = it >> (LOGT - 2), q = it & (T / 4 - 1);
        const int j = q & (h - 1);
        radix4<T>(buf, lr * T2 + (((q >> lh) << (lh + 2)) | j), h, T, j << (LOGT - 2 - lh), tab);
      }
      __syncthreads();
    }
#pragma unroll 1
    for (int lh = R4; lh < LOGT; ++lh) {
      const int h = 1 << lh;
      for (int it = tid; it < nr * (T / 2); it += NT) {
        const int lr = it >> (LOGT - 1), q = it & (T / 2 - 1);
        const int i = ((q >> lh) << (lh + 1)) | (q & (h - 1));
        const int ia = lr * T2 + i, ib = ia + h;
        const C a = A::load(buf, ia, T), bb = A::load(buf, ib, T);
        const C wb = A::mul_norm(IO::twiddle(tab, (q & (h - 1)) << (LOGT - 1 - lh)), bb);
        A::store(buf, ia, T, A::add(a, wb));
        A::store(buf, ib, T, A::sub(a, wb));
      }
      __syncthreads();
    }
    for (int e = tid; e < nr * T; e += NT) {
      const int lr = e >> LOGT, c = e & (T - 1);
      const int row = __brev(r0 + lr) >> (32 - LOGT);
      A::store(Z, row * T2 + c, T, A::load(buf, lr * T2 + c, T));
    }
    __syncthreads();
  }
  // ---- columns: chunk of CH columns, all T rows, rows of 2 CH elements ----
#pragma unroll 1
  for (int c0 = 0; c0 < T; c0 += CH) {
    for (int e = tid; e < T * CH; e += NT) {
      const int r = e / CH, lc = e - r * CH;
      A::store(buf, r * 2 * CH + lc, CH, A::load(Z, r * T2 + c0 + lc, T));
    }
    __syncthreads();
#pragma unroll 1
    for (int lh = 0; lh + 1 < R4; lh += 2) {
      const int h = 1 << lh;
      for (int it = tid; it < CH * (T / 4); it += NT) {
        const int lc = it % CH, q = it / CH;
        const int j = q & (h - 1);
        radix4<T>(buf, (((q >> lh) << (lh + 2)) | j) * 2 * CH + lc, h * 2 * CH, CH, j << (LOGT - 2 - lh), tab);
      }
      __syncthreads();
    }
#pragma unroll 1
    for (int lh = R4; lh < LOGT; ++lh) {
      const int h = 1 << lh;
      for (int it = tid; it < CH * (T / 2); it += NT) {
        const int lc = it % CH, q = it / CH;
        const int i = ((q >> lh) << (lh + 1)) | (q & (h - 1));
        const int ia = i * 2 * CH + lc, ib = ia + h * 2 * CH;
        const C a = A::load(buf, ia, CH), bb = A::load(buf, ib, CH);
        const C wb = A::mul_norm(IO::twiddle(tab, (q & (h - 1)) << (LOGT - 1 - lh)), bb);
        A::store(buf, ia, CH, A::add(a, wb));
        A::store(buf, ib, CH, A::sub(a, wb));
      }
      __syncthreads();
    }
    for (int e = tid; e < T * CH; e += NT) {
      const int r = e / CH, lc = e - r * CH;
      A::store(Z, r * T2 + c0 + lc, T, A::load(buf, r * 2 * CH + lc, CH));
    }
    __syncthreads();
  }
}

// The rebase of the FP32 loop (out of line: it runs rarely and keeps the hot
// loop's code small): the exact values of thread tid's held bins, R0 minus
// the terms nb .. nd of the list, written over R0 in the scratch (Rx); returns
// the thread's best of them (exact comparison) as (slot, 0, code, packed
// index).
template <int T, int NT>
__device__ __noinline__ int4 f3_rebase_bins(const float2* Whi, const float2* Zg, const float2* Wlo,
                                            const short* trY, const float4* trC, float4* Rx, int tid,
                                            int nb, int nd, float scale, float iscale) {
  using G = F3<T, NT>;
  constexpr int T2 = 2 * T;
  ffc wb = {{0.f, 0.f}, {0.f, 0.f}};
  int wbc = 0x7fffffff, wbx = 0, wbs = 0;
  for (int i = 0; i <= G::NB; ++i) {
    if (i == G::NB && tid >= 2) break;
    const int2 kk = i < G::NB ? f3_bin<T, NT>(tid, i) : f3_extra<T>(tid);
    const int x = kk.x * T2 + kk.y, slot = i < G::NB ? tid + i * NT : G::NSLOT + tid;
    long long sre = 0, sim = 0;
    recur_fixed<T>(Whi, Zg, Wlo, trY, trC, x, nb, nd, 1, scale, sre, sim);
    const float4 r0 = Rx[slot];
    const ffc v = {ff_sub(ff{r0.x, r0.y}, fx_to_ff(sre, iscale)), ff_sub(ff{r0.z, r0.w}, fx_to_ff(sim, iscale))};
    Rx[slot] = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
    const int code = f3_code<T>(kk.x, kk.y);
    if (wbc == 0x7fffffff || exact_better(v, code, wb, wbc)) {
      wb = v;
      wbc = code;
      wbx = x;
      wbs = slot;
    }
  }
  return make_int4(wbs, 0, wbc, wbx);
}

template <int T, int NT, bool OFSE>
__device__ __forceinline__ void forward_block_f3(const FwdArgs& args, const CUtensorMap* tmF,
                                                 const CUtensorMap* tmA, int blk, float2* Whi,
                                                 unsigned char* dsm, uint64_t* mbar,
                                                 unsigned& tma_phase, unsigned char* cta_scratch) {
  using A = ArFF;
  using C = ArFF::C;
  using IO = PlanIO<A>;
  using G = F3<T, NT>;
  constexpr int T2 = G::T2, LOGT = G::LOGT, NSLOT = G::NSLOT, NB = G::NB, NW = G::NW;
  constexpr int IB = G::IB, LIST = G::LIST;
  // with 32 or more bins per thread the top-2 keys run in two independent
  // chains (even and odd bins), merged after the update loop: a shorter
  // dependency chain (measured faster there, slower with 16 bins)
  constexpr bool kTwoChains = NB >= 32;
  constexpr int STEP8 = G::RS * T * 8, MSK8 = T * T * 8 - 8;
  constexpr float kU = 5.9604644775390625e-08f;  // 2^-24
  constexpr float kDn = 1.f - 16.f * kU, kUp = 1.f + 256.f * kU, kUpB = 1.f + 16.f * kU;
  constexpr float kTiny = 7.888609052210118e-31f;     // 2^-100: below it, sqrt is bounded by
  constexpr float kTinySqrt = 8.881784197001252e-16f; // 2^-50

  uint4* t2s = reinterpret_cast<uint4*>(dsm + G::t2_off);
  longlong2* red = reinterpret_cast<longlong2*>(dsm + G::red_off);
  int* wtot = reinterpret_cast<int*>(dsm + G::wtot_off);
  int4* list = reinterpret_cast<int4*>(dsm + G::list_off);
  float4* wwv = reinterpret_cast<float4*>(dsm + G::ww_off);
  int2* wwc = reinterpret_cast<int2*>(dsm + G::ww_off + 16 * NW);
  const PlanDev& P = args.plan;
  const int iters = P.iters;
  // The recurrence's terms: one entry per distinct selected index, in order
  // of first selection, with the sum of that index's coefficients (float-float,
  // canonical orientation).  A pair picked again adds to its entry, so the
  // exact recurrence sums over the distinct indices (about 40 % of the
  // iterations on natural content) instead of over every earlier iteration.
  float4* trC = reinterpret_cast<float4*>(dsm + G::trc_off);
  short* trY = reinterpret_cast<short*>(dsm + G::try_off(iters));
  int* nd_s = reinterpret_cast<int*>(dsm + G::nd_off);
  float2* Wlo = G::lo_smem(iters) ? reinterpret_cast<float2*>(dsm + G::lo_off(iters)) : nullptr;
  int nd = 0;  // entries in the list (warp 0 maintains it; the others read it each iteration)
  // entries before nb belong to coefficients taken into R0 by a rebase (below):
  // they count for the synthesis only, the recurrence sums entries nb .. nd
  int nb = 0;
  float2* Zg = reinterpret_cast<float2*>(cta_scratch);
  float4* Rx = reinterpret_cast<float4*>(cta_scratch + G::z_bytes);
  // OFSE: the packed FFT of w^2 f + j w^2, then the exact V = DFT(w^2) (the
  // layout of Zg), and the exact Q0 = DFT(w^2 f) per slot (the layout of Rx)
  float2* Vg = reinterpret_cast<float2*>(cta_scratch + G::scratch_bytes);
  float4* Qx = reinterpret_cast<float4*>(cta_scratch + G::scratch_bytes + G::z_bytes);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int rt = tid >> (LOGT - 1), ct = tid & (T / 2 - 1);
  const int chi = ct == 0 ? T / 2 : ct;
  const fofse_block bd = args.blocks[blk];
  const int b = P.block, br = P.border, Ls = P.Ls;
  const int ly0 = bd.y - br, lx0 = bd.x - br;

  // ---- 1. stage the support tile into shared memory (TMA) -------------------
  float* stF = reinterpret_cast<float*>(Whi);
  const int bytesF = args.box_f * Ls * 4;
  uint8_t* stA = reinterpret_cast<uint8_t*>(Whi) + ((bytesF + 127) & ~127);
  const int fx0 = lx0 & ~3, fo = lx0 - fx0;
  const int ax0 = lx0 & ~15, ao = lx0 - ax0;
  if (args.use_tma) {
    if (tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(mbar, (unsigned)(bytesF + args.box_a * Ls));
      tma_load_2d(stF, tmF, fx0, ly0, mbar);
      tma_load_2d(stA, tmA, ax0, ly0, mbar);
    }
    bool done = false;
    for (unsigned it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(mbar, tma_phase);
    if (!done) {
      atomicOr(args.err, kErrTimeout);
      for (unsigned it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(mbar, tma_phase);
    }
    tma_phase ^= 1u;
    if (!__syncthreads_and(done)) {
      if (tid == 0 && args.status) args.status[blk] = kBlkTimeout;
      return;
    }
  }

  // ---- 2. z = w f + j w at bit-reversed positions of the global FFT buffer --
  bool bad = false, nzf = false;
  for (int e = tid; e < T * T; e += NT) {
    const int r = e >> LOGT, cc = e & (T - 1);
    const int m = __brev(r) >> (32 - LOGT), n = __brev(cc) >> (32 - LOGT);
    C z = A::zero(), z2 = A::zero();
    if (m < Ls && n < Ls) {
      const bool inB = m >= br && m < br + b && n >= br && n < br + b;
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
        bad |= !isfinite(f);
        nzf |= f != 0.f;
        C wd;
        z = IO::weighted(P.tab, m * Ls + n, f, wd);
        if constexpr (OFSE) {
          const ff w2 = ff_mul(wd.re, wd.re);
          z2 = {ff_mul(w2, ff{f, 0.f}), w2};
        }
      }
    }
    A::store(Zg, r * T2 + cc, T, z);
    if constexpr (OFSE) A::store(Vg, r * T2 + cc, T, z2);
  }
  // the staging tiles are read: the W region becomes the FFT's chunk buffer
  int any_bad = __syncthreads_or(bad);
  // f = 0 on the whole support: R0 = DFT(w f) is exactly zero (the packed
  // transform would leave W's rounding in it, about 1e-16 of |W|)
  const bool zero_f = !__syncthreads_or(nzf);

  // ---- 3. FFT (float-float), through shared memory in chunks -------------------
  fft2d_chunked<T, NT>(Zg, Whi, P.tab, Ls);
  if constexpr (OFSE) fft2d_chunked<T, NT>(Vg, Whi, P.tab, Ls);

  // ---- split: exact R0 -> scratch, FP32 copy -> registers, first top-2 -------
  float2 R32[NB];
  float2 rex = make_float2(0.f, 0.f);
  unsigned m1k = 0u, m2k = 0u;
#pragma unroll
  for (int i = 0; i <= NB; ++i) {
    if (i == NB && tid >= 2) break;
    const int2 kk = i < NB ? f3_bin<T, NT>(tid, i) : f3_extra<T>(tid);
    const int x = kk.x * T2 + kk.y;
    const int mx = ((T - kk.x) & (T - 1)) * T2 + ((T - kk.y) & (T - 1));
    const C a = A::load(Zg, x, T), mm = A::load(Zg, mx, T);
    const C r = zero_f ? A::zero() : A::half(A::add(a, A::conj(mm)));
    if (!A::finite(r)) bad = true;
    const int slot = i < NB ? tid + i * NT : NSLOT + tid;
    Rx[slot] = make_float4(r.re.h, r.re.l, r.im.h, r.im.l);
    const float2 r32 = make_float2(r.re.h, r.im.h);
    if (i < NB) R32[i] = r32;
    else rex = r32;
    key_insert(m1k, m2k, m32(r32), i);
    if constexpr (OFSE) {
      const C qa = A::load(Vg, x, T), qm = A::load(Vg, mx, T);
      const C qv = zero_f ? A::zero() : A::half(A::add(qa, A::conj(qm)));
      Qx[slot] = make_float4(qv.re.h, qv.re.l, qv.im.h, qv.im.l);
    }
  }
  any_bad |= __syncthreads_or(bad);
  build_wtab<A, T, NT, false>(Zg, nullptr);  // exact W in place (global)
  if constexpr (OFSE) build_wtab<A, T, NT, false>(Vg, nullptr);  // exact V = DFT(w^2)
  __syncthreads();
  for (int e = tid; e < T * T; e += NT) Whi[e] = Zg[(e >> LOGT) * T2 + (e & (T - 1))];
  if (Wlo)
    for (int e = tid; e < T * G::LO_LD; e += NT) {
      const int r = e / G::LO_LD, c = e - r * G::LO_LD;
      Wlo[e] = Zg[r * T2 + c + T];
    }
  __syncthreads();
  const C W0c = A::load(Zg, 0, T);
  int st = FOFSE_BLK_OK;
  if (IO::w0_zero(W0c)) st = FOFSE_BLK_NO_SUPPORT;
  else if (any_bad || !IO::w0_finite(W0c)) st = FOFSE_BLK_NONFINITE;

  int done_it = 0;  // iterations the loop ran (any later one repeats a zero residual's (0, 0), 0)
  if (st == FOFSE_BLK_OK) {
    const ff inv = IO::inv_w0(IO::gamma(P), W0c.re);
    const float W0f = W0c.re.h * (1.f + 1e-6f);
    const char* wb8 = reinterpret_cast<const char*>(Whi);
    float bnd = 0.f, prevabs = 0.f, csum = 0.f;
    bool dc_run = true;   // every winner so far was the DC bin
    float kA = 2.1f * kU, kB = 12.f * kU;  // bound increments (raised once after a refresh)
    // The iteration loop runs in two stretches: the first ends at the first
    // winner that is not the DC bin, where the working spectrum is refreshed
    // from exact values (below, outside the hot loop), then the loop resumes.
    // Only at fft_size 128 (400 iterations, where near-ties are frequent
    // enough to repay it; at 32 and 64 the extra code costs more than it saves).
    constexpr bool kRefresh = T >= 128;
    int it = 0, wk1 = 0, wk2 = 0;
    bool sc = false;
    float p = 0.f, q = 0.f;
#pragma unroll 1
    for (;;) {
      bool refresh = false;
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
        // square roots from the hardware reciprocal square root (relative
        // error a few ulp, inside the 16u / 256u margins): sM1 is a lower and
        // sM1u an upper bound of the largest |R32|, sM2 an upper bound of the rest
        const float m1 = __uint_as_float(g.x & ~kKeyMask), m2 = __uint_as_float(g.y & ~kKeyMask);
        const bool n1 = m1 >= kTiny, n2 = m2 >= kTiny;
        const float r1 = m1 * rsqrtf(n1 ? m1 : 1.f), r2 = m2 * rsqrtf(n2 ? m2 : 1.f);
        const float sM1 = n1 ? r1 : 0.f, sM1u = n1 ? r1 * kUp : kTinySqrt;
        const float sM2 = n2 ? r2 : kTinySqrt;
        bnd += kA * sM1u + kB * W0f * prevabs;
        kA = 2.1f * kU;
        kB = 12.f * kU;
        const bool certain = (sM1 * kDn - bnd * kUpB) > (sM2 * kUp + bnd * kUpB);
        // fixed-point unit of the recurrence: every partial sum is below
        // 2 W0 sum_j (|Re c_j| + |Im c_j|) <= 4 W0f csum
        const int sh = fx_shift(4.f * W0f * csum);
        const float scale = pow2f(sh), iscale = pow2f(-sh);

        ffc Rt;
        if (certain) {
          const int wt = (int)g.z, li = (int)(g.x & kKeyMask);
          int wslot;
          if (li < NB) {
            const int2 kk = f3_bin<T, NT>(wt, li);
            wk1 = kk.x;
            wk2 = kk.y;
            wslot = wt + li * NT;
          } else {
            const int2 kk = f3_extra<T>(wt);
            wk1 = kk.x;
            wk2 = kk.y;
            wslot = NSLOT + wt;
          }
          const float4 r0 = Rx[wslot];
          // one term per thread and iteration at most; up to four warps the
          // partial sums go through shuffles and a short block sum, beyond
          // that through redux.sync (warp and block level)
          long long sre = 0, sim = 0;
          long long Sr = 0, Si = 0;
          if constexpr (NW <= 4) {
            if (warp * 32 < nd - nb) {  // warp-uniform: this warp holds terms
              recur_fixed<T>(Whi, Zg, Wlo, trY, trC, wk1 * T2 + wk2, nb + tid, nd, NT, scale, sre, sim);
              warp_sum64(sre, sim);
            }
            if (lane == 0) red[warp] = make_longlong2(sre, sim);
            __syncthreads();
#pragma unroll
            for (int w = 0; w < NW; ++w) {
              const longlong2 v = red[w];
              Sr += v.x;
              Si += v.y;
            }
          } else {
            if (warp * 32 < nd - nb) {
              recur_fixed<T>(Whi, Zg, Wlo, trY, trC, wk1 * T2 + wk2, nb + tid, nd, NT, scale, sre, sim);
              sre = redux_sum64(sre);
              sim = redux_sum64(sim);
            }
            if (lane == 0) red[warp] = make_longlong2(sre, sim);
            __syncthreads();
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
          for (int i = 0; i < NB; ++i) cnt += m32(R32[i]) >= thr ? 1 : 0;
          if (tid < 2) cnt += m32(rex) >= thr ? 1 : 0;
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
          if (!OFSE && total > G::REBASE) {
            // ---- rebase: when the bound has grown to the size of the
            // residual (a residual that decays far, as over flat content)
            // nearly every bin is a candidate.  Each thread then evaluates
            // its own bins exactly, these values become R0 (the coefficients
            // so far are folded in: the recurrence continues from entry nb),
            // R32 their FP32 roundings, and the bound restarts from their
            // rounding.  The winner is their exact maximum.
            {
              const int4 r = f3_rebase_bins<T, NT>(Whi, Zg, Wlo, trY, trC, Rx, tid, nb, nd, scale, iscale);
              wbc = r.z;
              wbx = r.w;
              const float4 v = Rx[r.x];  // the best value, as written
              wb = {{v.x, v.y}, {v.z, v.w}};
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) {
              const float4 r = Rx[tid + i * NT];
              R32[i] = make_float2(r.x, r.z);
            }
            if (tid < 2) {
              const float4 r = Rx[NSLOT + tid];
              rex = make_float2(r.x, r.z);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const ffc ov = ffc_shfl(wb, o);
              const int oc = __shfl_xor_sync(kFull, wbc, o), ox = __shfl_xor_sync(kFull, wbx, o);
              if (exact_better(ov, oc, wb, wbc)) {
                wb = ov;
                wbc = oc;
                wbx = ox;
              }
            }
            nb = nd;
            csum = 0.f;
          } else {
          for (int pass = 0; pass < total; pass += LIST) {
            int r = rank0;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
              if (m32(R32[i]) >= thr) {
                if (r >= pass && r < pass + LIST) {
                  const int2 kk = f3_bin<T, NT>(tid, i);
                  list[r - pass] = make_int4(kk.x * T2 + kk.y, f3_code<T>(kk.x, kk.y), tid + i * NT, 0);
                }
                ++r;
              }
            }
            if (tid < 2 && m32(rex) >= thr && r >= pass && r < pass + LIST) {
              const int2 kk = f3_extra<T>(tid);
              list[r - pass] = make_int4(kk.x * T2 + kk.y, f3_code<T>(kk.x, kk.y), NSLOT + tid, 0);
            }
            __syncthreads();
            const int n = min(LIST, total - pass);
            for (int c = warp; c < n; c += NW) {
              const int4 e = list[c];
              const float4 r0 = Rx[e.z];
              long long sre = 0, sim = 0;
              recur_fixed<T>(Whi, Zg, Wlo, trY, trC, e.x, nb + lane, nd, 32, scale, sre, sim);
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
          wk1 = wx >> (LOGT + 1);
          wk2 = wx & (T2 - 1);
          // after a rebase the bound restarts: the roundings of the new R0 to
          // FP32 (u of the largest value, the winner's) are covered by the
          // first increment, as for the first R0
          if (!OFSE && total > G::REBASE) bnd = kA * (fabsf(Rt.re.h) + fabsf(Rt.im.h)) * kUp;
        }
        // ---- exact coefficient (Eq. 5, Eq. 14) of the held winner ----
        const bool mir = wk1 > T / 2;
        const int u1 = mir ? ((T - wk1) & (T - 1)) : wk1;
        const int u2 = mir ? ((T - wk2) & (T - 1)) : wk2;
        sc = ((wk1 & (T / 2 - 1)) == 0) && ((wk2 & (T / 2 - 1)) == 0);
        C c;
        if constexpr (!OFSE) {
          c.re = ff_mul(Rt.re, inv);
          c.im = sc ? ff{0.f, 0.f} : ff_mul(Rt.im, inv);
        } else {
          // OFSE's compensation (Eq. 10-13) with the DFT basis: with
          // Q[u] = sum_l P[l] W[u - l] = T^2 DFT(w^2 r)[u], c = P[u]^2 / Q[u] and
          // gamma_u = W0 P[u] / Q[u].  DFT(w^2 r) at the winner comes from the
          // same triangular recurrence as R~, with V = DFT(w^2) for W
          // (|V[k]| <= V[0] <= W[0], so the fixed-point unit above holds):
          //   Q~[k] = Q0[k] - sum_{j<i} (c_j V[k - u_j] + s_j conj(c_j) V[k + u_j]).
          const float4 q0 = Qx[f3_slot<T, NT>(wk1, wk2)];
          const int xw = wk1 * T2 + wk2;
          longlong2* red2 = red + NW;
          long long sre = 0, sim = 0, Sr = 0, Si = 0;
          if constexpr (NW <= 4) {
            if (warp * 32 < nd - nb) {
              recur_fixed<T, true>(Whi, Vg, nullptr, trY, trC, xw, nb + tid, nd, NT, scale, sre, sim);
              warp_sum64(sre, sim);
            }
            if (lane == 0) red2[warp] = make_longlong2(sre, sim);
            __syncthreads();
#pragma unroll
            for (int w = 0; w < NW; ++w) {
              const longlong2 v = red2[w];
              Sr += v.x;
              Si += v.y;
            }
          } else {
            if (warp * 32 < nd - nb) {
              recur_fixed<T, true>(Whi, Vg, nullptr, trY, trC, xw, nb + tid, nd, NT, scale, sre, sim);
              sre = redux_sum64(sre);
              sim = redux_sum64(sim);
            }
            if (lane == 0) red2[warp] = make_longlong2(sre, sim);
            __syncthreads();
            const longlong2 v = lane < NW ? red2[lane] : make_longlong2(0, 0);
            Sr = redux_sum64(v.x);
            Si = redux_sum64(v.y);
          }
          const ff qr = ff_sub(ff{q0.x, q0.y}, fx_to_ff(Sr, iscale));
          const ff qi = sc ? ff{0.f, 0.f} : ff_sub(ff{q0.z, q0.w}, fx_to_ff(Si, iscale));
          const ff rr = Rt.re, ri = sc ? ff{0.f, 0.f} : Rt.im;
          const ff den = ff_add(ff_mul(qr, qr), ff_mul(qi, qi));
          const ff nr = ff_sub(ff_mul(rr, rr), ff_mul(ri, ri)), ni = ff_scale(ff_mul(rr, ri), 2.f);
          constexpr float kInvT2 = 1.f / (float)(T * T);  // a power of two
          if (den.h > 0.f) {  // Q = 0 (a zero residual): c = 0
            c.re = ff_scale(ff_div(ff_add(ff_mul(nr, qr), ff_mul(ni, qi)), den), kInvT2);
            c.im = ff_scale(ff_div(ff_sub(ff_mul(ni, qr), ff_mul(nr, qi)), den), kInvT2);
          } else {
            c.re = c.im = ff{0.f, 0.f};
          }
          if (tid == 0 && args.gamma_out) {
            float2 gm = make_float2(0.f, 0.f);
            if (den.h > 0.f) {
              gm.x = ff_scale(ff_mul(W0c.re, ff_div(ff_add(ff_mul(rr, qr), ff_mul(ri, qi)), den)), kInvT2).h;
              gm.y = ff_scale(ff_mul(W0c.re, ff_div(ff_sub(ff_mul(ri, qr), ff_mul(rr, qi)), den)), kInvT2).h;
            }
            args.gamma_out[(size_t)blk * args.trace_stride + it] = mir ? make_float2(gm.x, -gm.y) : gm;
          }
        }
        // ---- record: the trace entry, and the term of the recurrence ----
        // (every read of the list in this iteration lies before a barrier
        // that precedes this update)
        if (warp == 0) {
          const float4 cc = mir ? make_float4(c.re.h, c.re.l, -c.im.h, -c.im.l)
                                : make_float4(c.re.h, c.re.l, c.im.h, c.im.l);
          const short y = (short)(u1 * T2 + u2);
          int pos = -1;
          for (int j0 = nb; j0 < nd; j0 += 32) {
            const int j = j0 + lane;
            const unsigned hit = __ballot_sync(kFull, j < nd && trY[j] == y);
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
              trY[nd] = y;
              trC[nd] = cc;
            }
            if (args.trace) {
              fofse_trace_entry e;
              e.u1 = (int16_t)u1;
              e.u2 = (int16_t)u2;
              e.dc_re = cc.x;
              e.dc_im = cc.z;
              args.trace[(size_t)blk * args.trace_stride + it] = e;
            }
          }
          if (pos < 0) ++nd;
        }
        // The winner is the exact maximum, so an exactly zero winner means
        // the exact residual is zero in every bin: every later iteration
        // selects the smallest index, (0, 0) (which this one did), with a zero
        // coefficient and changes nothing.  They are written as such at the
        // end instead of being run (each would resolve a near-tie over every
        // bin).
        if (Rt.re.h == 0.f && Rt.re.l == 0.f && Rt.im.h == 0.f && Rt.im.l == 0.f) {
          ++it;
          break;
        }
        p = c.re.h;
        q = c.im.h;
        if (kRefresh && dc_run && !(wk1 == 0 && wk2 == 0)) {
          dc_run = false;
          if (it > 0) {
            refresh = true;
            break;
          }
        }
        // ---- FP32 update of the working spectrum + next top-2 keys ----
        prevabs = fabsf(p) + fabsf(q);
        csum += prevabs;
        const int rm = ((rt - wk1) & (T - 1)) << LOGT, rp = ((rt + wk1) & (T - 1)) << LOGT;
        const int bml = (rm | ((ct - wk2) & (T - 1))) << 3, bmh = (rm | ((chi - wk2) & (T - 1))) << 3;
        const int bpl = (rp | ((ct + wk2) & (T - 1))) << 3, bph = (rp | ((chi + wk2) & (T - 1))) << 3;
        const int bmi = rt > 0 ? bmh : bml, bpi = rt > 0 ? bph : bpl;
        unsigned k1a = 0u, k2a = 0u, k1b = 0u, k2b = 0u;  // two key chains (even / odd bins)
        const unsigned long long npp = f3_pair(-p);
        if (!sc) {
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const int bm = i < IB ? bml : (i == IB ? bmi : bmh);
            const int bp = i < IB ? bpl : (i == IB ? bpi : bph);
            const float2 Wm = *reinterpret_cast<const float2*>(wb8 + ((bm + i * STEP8) & MSK8));
            const float2 Wp = *reinterpret_cast<const float2*>(wb8 + ((bp + i * STEP8) & MSK8));
            f3_update_bin(R32[i], Wm, Wp, q, npp);
            if (kTwoChains && (i & 1)) key_insert(k1b, k2b, m32(R32[i]), i);
            else key_insert(k1a, k2a, m32(R32[i]), i);
          }
        } else {
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const int bm = i < IB ? bml : (i == IB ? bmi : bmh);
            const float2 Wm = *reinterpret_cast<const float2*>(wb8 + ((bm + i * STEP8) & MSK8));
            f3_update_bin_sc(R32[i], Wm, npp);
            if (kTwoChains && (i & 1)) key_insert(k1b, k2b, m32(R32[i]), i);
            else key_insert(k1a, k2a, m32(R32[i]), i);
          }
        }
        if (tid < 2) {
          const int2 kk = f3_extra<T>(tid);
          const float2 Wm = Whi[(((kk.x - wk1) & (T - 1)) << LOGT) | ((kk.y - wk2) & (T - 1))];
          float2 Wp = make_float2(0.f, 0.f);
          if (!sc) Wp = Whi[(((kk.x + wk1) & (T - 1)) << LOGT) | ((kk.y + wk2) & (T - 1))];
          const float a = Wm.x + Wp.x, bb = Wm.y - Wp.y, cc = Wm.y + Wp.y, d = Wm.x - Wp.x;
          rex.x = __fmaf_rn(-p, a, __fmaf_rn(q, bb, rex.x));
          rex.y = __fmaf_rn(-p, cc, __fmaf_rn(-q, d, rex.y));
          key_insert(k1a, k2a, m32(rex), NB);
        }
        m1k = max(k1a, k1b);
        m2k = max(max(k2a, k2b), min(k1a, k1b));
      }
      if (!refresh) break;
      // ---- refresh after the initial run of DC picks ----
      // The first picks are usually the DC bin (u = 0, real c_j), with large
      // coefficients whose FP32 rounding dominates the bound.  At the first
      // other winner the working spectrum is rebuilt from the exact values,
      // R~[k] = R0[k] - C W[k] with C = sum_{j<it} c_j, and the bound restarts:
      // the rounding of R~ (u |R~| <= u (max|R32| + 2 |c| W[0]) after this
      // iteration's update) is added with the next increment.
      {
        // every earlier pick was the DC bin: its single list entry holds the
        // sum C (the entry is not written in this iteration)
        const float4 c0 = nd > nb ? trC[nb] : make_float4(0.f, 0.f, 0.f, 0.f);
        const ff Cs = {c0.x, c0.y};
#pragma unroll
        for (int i = 0; i <= NB; ++i) {
          if (i == NB && tid >= 2) break;
          const int2 kk = i < NB ? f3_bin<T, NT>(tid, i) : f3_extra<T>(tid);
          const int x = kk.x * T2 + kk.y;
          const float4 r0 = Rx[i < NB ? tid + i * NT : NSLOT + tid];
          const float2 wh = Zg[x], wl = Zg[x + T];
          const float2 r = make_float2(ff_sub(ff{r0.x, r0.y}, ff_mul(Cs, ff{wh.x, wl.x})).h,
                                       ff_sub(ff{r0.z, r0.w}, ff_mul(Cs, ff{wh.y, wl.y})).h);
          if (i < NB) R32[i] = r;
          else rex = r;
        }
        bnd = 0.f;
        kA = (2.1f + 1.1f) * kU;
        kB = (12.f + 2.1f) * kU;
      }
      // this iteration's update, then back to the loop
      // ---- FP32 update of the working spectrum + next top-2 keys ----
      prevabs = fabsf(p) + fabsf(q);
      csum += prevabs;
      const int rm = ((rt - wk1) & (T - 1)) << LOGT, rp = ((rt + wk1) & (T - 1)) << LOGT;
      const int bml = (rm | ((ct - wk2) & (T - 1))) << 3, bmh = (rm | ((chi - wk2) & (T - 1))) << 3;
      const int bpl = (rp | ((ct + wk2) & (T - 1))) << 3, bph = (rp | ((chi + wk2) & (T - 1))) << 3;
      const int bmi = rt > 0 ? bmh : bml, bpi = rt > 0 ? bph : bpl;
      unsigned k1a = 0u, k2a = 0u, k1b = 0u, k2b = 0u;  // two key chains (even / odd bins)
      const unsigned long long npp = f3_pair(-p);
      if (!sc) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const int bm = i < IB ? bml : (i == IB ? bmi : bmh);
          const int bp = i < IB ? bpl : (i == IB ? bpi : bph);
          const float2 Wm = *reinterpret_cast<const float2*>(wb8 + ((bm + i * STEP8) & MSK8));
          const float2 Wp = *reinterpret_cast<const float2*>(wb8 + ((bp + i * STEP8) & MSK8));
          f3_update_bin(R32[i], Wm, Wp, q, npp);
          if (kTwoChains && (i & 1)) key_insert(k1b, k2b, m32(R32[i]), i);
            else key_insert(k1a, k2a, m32(R32[i]), i);
        }
      } else {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const int bm = i < IB ? bml : (i == IB ? bmi : bmh);
          const float2 Wm = *reinterpret_cast<const float2*>(wb8 + ((bm + i * STEP8) & MSK8));
          f3_update_bin_sc(R32[i], Wm, npp);
          if (kTwoChains && (i & 1)) key_insert(k1b, k2b, m32(R32[i]), i);
            else key_insert(k1a, k2a, m32(R32[i]), i);
        }
      }
      if (tid < 2) {
        const int2 kk = f3_extra<T>(tid);
        const float2 Wm = Whi[(((kk.x - wk1) & (T - 1)) << LOGT) | ((kk.y - wk2) & (T - 1))];
        float2 Wp = make_float2(0.f, 0.f);
        if (!sc) Wp = Whi[(((kk.x + wk1) & (T - 1)) << LOGT) | ((kk.y + wk2) & (T - 1))];
        const float a = Wm.x + Wp.x, bb = Wm.y - Wp.y, cc = Wm.y + Wp.y, d = Wm.x - Wp.x;
        rex.x = __fmaf_rn(-p, a, __fmaf_rn(q, bb, rex.x));
        rex.y = __fmaf_rn(-p, cc, __fmaf_rn(-q, d, rex.y));
        key_insert(k1a, k2a, m32(rex), NB);
      }
      m1k = max(k1a, k1b);
      m2k = max(max(k2a, k2b), min(k1a, k1b));
      ++it;
    }
    done_it = it;
  }
  if (tid == 0) *nd_s = nd;  // thread 0 is in warp 0, which holds the count
  __syncthreads();

  // ---- synthesis of B (Eq. 1) from the exact coefficients; outputs ----------
  const int nIt = (st == FOFSE_BLK_OK) ? iters : 0;
  const int nTerms = (st == FOFSE_BLK_OK) ? *nd_s : 0;
  const int ld = args.out_ld;
  const float2* syn = P.tab.syn_f32;
  for (int pidx = tid; pidx < ld * ld; pidx += NT) {
    const int bm = pidx / ld, bn = pidx - bm * ld;
    float v = 0.f;
    if (bm < b && bn < b) {
      const int m = br + bm, n = br + bn;
      if constexpr (!OFSE) {
        float acc = 0.f;
        for (int i = 0; i < nTerms; ++i) {
          const int yy = trY[i];
          const int a1 = yy >> (LOGT + 1), a2 = yy & (T2 - 1);
          const float4 c4 = trC[i];
          const float mult = (((a1 & (T / 2 - 1)) == 0) && ((a2 & (T / 2 - 1)) == 0)) ? 1.f : 2.f;
          const float2 cs = __ldg(&syn[(a1 * m + a2 * n) & (T - 1)]);
          acc += mult * (c4.x * cs.x - c4.z * cs.y);
        }
        v = acc;
      } else {
        // OFSE's coefficients are larger and alternate in sign (factors up
        // to tens), so the FP32 sum would lose more than the output
        // tolerance: float-float terms and sum
        ff acc = {0.f, 0.f};
        for (int i = 0; i < nTerms; ++i) {
          const int yy = trY[i];
          const int a1 = yy >> (LOGT + 1), a2 = yy & (T2 - 1);
          const float4 c4 = trC[i];
          const float mult = (((a1 & (T / 2 - 1)) == 0) && ((a2 & (T / 2 - 1)) == 0)) ? 1.f : 2.f;
          const float4 cs = __ldg(&P.tab.syn_ff[(a1 * m + a2 * n) & (T - 1)]);
          const ff t = ff_dot2(ff{c4.x, c4.y}, ff{cs.x, cs.z}, ff{-c4.z, -c4.w}, ff{cs.y, cs.w});
          acc = ff_add(acc, ff{mult * t.h, mult * t.l});
        }
        v = acc.h + acc.l;
      }
      if (args.out_frame) {
        const int fy = bd.y + bm, fx = bd.x + bn;
        if (fy >= 0 && fy < args.height && fx >= 0 && fx < args.width)
          args.out_frame[(size_t)fy * args.pitch + fx] = v;
      }
    }
    if (args.out_blocks) args.out_blocks[(size_t)blk * args.out_stride + pidx] = v;
  }
  if (args.trace) {  // entries of the iterations that ran were written as they ran
    for (int i = done_it + tid; i < args.trace_stride; i += NT) {
      fofse_trace_entry e;
      e.u1 = e.u2 = 0;
      e.dc_re = e.dc_im = 0.f;
      args.trace[(size_t)blk * args.trace_stride + i] = e;
    }
  }
  if (args.gamma_out) {  // the compensation factor of each iteration (Eq. 13)
    for (int i = tid; i < args.trace_stride; i += NT) {
      float2* gp = args.gamma_out + (size_t)blk * args.trace_stride + i;
      if (i >= (OFSE ? done_it : nIt)) *gp = make_float2(0.f, 0.f);
      else if (!OFSE) *gp = make_float2(IO::gamma(P).h, 0.f);  // OFSE: written per iteration
    }
  }
  if (tid == 0) {
    if (args.w0) args.w0[blk] = st == FOFSE_BLK_OK ? W0c.re.h + W0c.re.l : 0.f;
    if (args.status) args.status[blk] = st;
  }
  __syncthreads();
}

template <int T, int NT, int MINB, bool OFSE>
__global__ void __launch_bounds__(NT, MINB) fofse_forward_f3_kernel(const __grid_constant__ FwdArgs args,
                                                              const __grid_constant__ CUtensorMap tmF,
                                                              const __grid_constant__ CUtensorMap tmA) {
  using G = F3<T, NT>;
  // dynamic shared memory: 16-byte alignment serves its slots; where W's
  // plane lives there (fft_size 128) it is the TMA staging target and starts
  // on a 128-byte boundary
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* dsm;
  float2* Whi;
  if constexpr (G::STATIC_W) {
    __shared__ __align__(128) float2 s_whi[G::STATIC_W ? T * T : 1];
    Whi = s_whi;
    dsm = smem_raw;
  } else {
    dsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    Whi = reinterpret_cast<float2*>(dsm);
  }
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
  unsigned char* cta_scratch =
      static_cast<unsigned char*>(args.scratch) +
      (size_t)blockIdx.x * (OFSE ? G::scratch_bytes_ofse : G::scratch_bytes);
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
    forward_block_f3<T, NT, OFSE>(args, &tmF, &tmA, item, Whi, dsm, &mbar, tma_phase, cta_scratch);
  }
}

template <int T, int NT, int MINB, bool OFSE = false> struct VariantF3 {
  static constexpr size_t per_cta = OFSE ? F3<T, NT>::scratch_bytes_ofse : F3<T, NT>::scratch_bytes;
  static cudaError_t prepare(int iters, size_t* smem, int* max_ctas) {
    *smem = F3<T, NT>::bytes(iters);
    return prepare_kernel(fofse_forward_f3_kernel<T, NT, MINB, OFSE>, NT, *smem, max_ctas);
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
    const size_t fit = a.scratch ? a.scratch_bytes / per_cta : 0;
    if (fit < 1) return cudaErrorInvalidValue;
    if ((size_t)grid > fit) grid = (int)fit;
    if (grid > a.n_blocks) grid = a.n_blocks;
    if (grid < 1) return cudaSuccess;
    fofse_forward_f3_kernel<T, NT, MINB, OFSE><<<grid, NT, sm, s>>>(a, *tf, *ta);
    return cudaGetLastError();
  }
};

}  // namespace
}  // namespace fofse
