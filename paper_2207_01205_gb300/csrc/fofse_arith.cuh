// Arithmetic back-ends of the FOFSE kernels.
//
//  * ArFF  -- compensated "float-float" arithmetic: every real is an unevaluated
//             sum hi + lo of two FP32 numbers (about 48 significant bits).  Only
//             FP32 instructions are issued.  The selection path of FOFSE is
//             decided by an argmax over |R_w|^2 (Sec. 2, Eq. 9); near-ties make
//             plain FP32 diverge from the exact path, so this is the product's
//             arithmetic.
//  * ArF64 -- IEEE double, for the FP64 validation mode.
//  * ArF32 -- plain FP32, the arithmetic of the frozen-path backward (linear
//             along the path: no decision to keep exact).
//
// The error-free transformations are Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA-based TwoProduct; intrinsics with explicit rounding (__fadd_rn ...)
// keep the compiler from contracting or reassociating them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fofse {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ ff ff_from(float a) { return {a, 0.f}; }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
// sum with an absolute error of order 2^-46 (|a| + |b|)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return ff_fast_two_sum(s.h, e);
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
// the same sum without the final renormalisation (feeds products only)
__device__ __forceinline__ ff ff_add_raw(ff a, ff b) {
  ff s = ff_two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ ff ff_sub_raw(ff a, ff b) { return ff_add_raw(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_two_prod(a.h, b.h);
  float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return ff_fast_two_sum(p.h, e);
}
__device__ __forceinline__ ff ff_scale(ff a, float s) {  // s exact power of two
  return {a.h * s, a.l * s};
}
// a / b (one Newton correction)
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  float q1 = __fdiv_rn(a.h, b.h);
  ff r = ff_sub(a, ff_mul(b, ff_from(q1)));
  float q2 = __fdiv_rn(r.h, b.h);
  return ff_fast_two_sum(q1, q2);
}
// a.x * b.x - a.y * b.y style dot product of two ff pairs: p*x + q*y
__device__ __forceinline__ ff ff_dot2(ff p, ff x, ff q, ff y) {
  ff P1 = ff_two_prod(p.h, x.h);
  ff P2 = ff_two_prod(q.h, y.h);
  ff s = ff_two_sum(P1.h, P2.h);
  float lo = __fadd_rn(s.l, __fadd_rn(P1.l, P2.l));
  lo = __fmaf_rn(p.h, x.l, lo);
  lo = __fmaf_rn(p.l, x.h, lo);
  lo = __fmaf_rn(q.h, y.l, lo);
  lo = __fmaf_rn(q.l, y.h, lo);
  return {s.h, lo};
}
// |z|^2 of a complex ff, normalised
__device__ __forceinline__ ff ff_norm2(ff re, ff im) {
  ff a = ff_two_prod(re.h, re.h);
  ff b = ff_two_prod(im.h, im.h);
  ff s = ff_two_sum(a.h, b.h);
  float lo = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  lo = __fmaf_rn(2.f * re.h, re.l, lo);
  lo = __fmaf_rn(2.f * im.h, im.l, lo);
  return ff_fast_two_sum(s.h, lo);
}

// ---------------------------------------------------------------------------
// Back-end traits.  Each provides:
//   S           real scalar;   C  complex {S re, im}
//   E           element type of the shared-memory spectra (two planes per row)
//   load/store  a complex at spectrum index idx (part 0 at idx, part 1 at idx+T)
//   add/sub/mul complex arithmetic, half(), from_double()
// ---------------------------------------------------------------------------

struct ArFF {
  using S = ff;
  struct C { ff re, im; };
  using E = float2;  // part0 = (re.h, im.h), part1 = (re.l, im.l)
  static constexpr int kBytes = 16;
  __device__ __forceinline__ static C load(const E* b, int idx, int T) {
    float2 h = b[idx], l = b[idx + T];
    return {{h.x, l.x}, {h.y, l.y}};
  }
  __device__ __forceinline__ static void store(E* b, int idx, int T, C v) {
    b[idx] = make_float2(v.re.h, v.im.h);
    b[idx + T] = make_float2(v.re.l, v.im.l);
  }
  __device__ __forceinline__ static C zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
  __device__ __forceinline__ static C add(C a, C b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
  __device__ __forceinline__ static C sub(C a, C b) { return {ff_sub(a.re, b.re), ff_sub(a.im, b.im)}; }
  __device__ __forceinline__ static C mul(C a, C b) {
    return {ff_dot2(a.re, b.re, ff_neg(a.im), b.im), ff_dot2(a.re, b.im, a.im, b.re)};
  }
  __device__ __forceinline__ static C mul_norm(C a, C b) {  // normalised result
    C r = mul(a, b);
    return {ff_fast_two_sum(r.re.h, r.re.l), ff_fast_two_sum(r.im.h, r.im.l)};
  }
  __device__ __forceinline__ static C conj(C a) { return {a.re, ff_neg(a.im)}; }
  __device__ __forceinline__ static C half(C a) { return {ff_scale(a.re, 0.5f), ff_scale(a.im, 0.5f)}; }
  __device__ __forceinline__ static bool finite(C a) { return isfinite(a.re.h) && isfinite(a.im.h); }
  __device__ __forceinline__ static float approx_re(C a) { return a.re.h; }
  __device__ __forceinline__ static float approx_im(C a) { return a.im.h; }
};

struct ArF64 {
  using S = double;
  struct C { double re, im; };
  using E = double;  // part0 = re, part1 = im
  static constexpr int kBytes = 16;
  __device__ __forceinline__ static C load(const E* b, int idx, int T) { return {b[idx], b[idx + T]}; }
  __device__ __forceinline__ static void store(E* b, int idx, int T, C v) {
    b[idx] = v.re;
    b[idx + T] = v.im;
  }
  __device__ __forceinline__ static C zero() { return {0.0, 0.0}; }
  __device__ __forceinline__ static C add(C a, C b) { return {a.re + b.re, a.im + b.im}; }
  __device__ __forceinline__ static C sub(C a, C b) { return {a.re - b.re, a.im - b.im}; }
  __device__ __forceinline__ static C mul(C a, C b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  }
  __device__ __forceinline__ static C mul_norm(C a, C b) { return mul(a, b); }
  __device__ __forceinline__ static C conj(C a) { return {a.re, -a.im}; }
  __device__ __forceinline__ static C half(C a) { return {0.5 * a.re, 0.5 * a.im}; }
  __device__ __forceinline__ static bool finite(C a) { return isfinite(a.re) && isfinite(a.im); }
  __device__ __forceinline__ static double approx_re(C a) { return a.re; }
  __device__ __forceinline__ static double approx_im(C a) { return a.im; }
};

struct ArF32 {
  using S = float;
  struct C { float re, im; };
  using E = float;  // part0 = re, part1 = im
  static constexpr int kBytes = 8;
  __device__ __forceinline__ static C load(const E* b, int idx, int T) { return {b[idx], b[idx + T]}; }
  __device__ __forceinline__ static void store(E* b, int idx, int T, C v) {
    b[idx] = v.re;
    b[idx + T] = v.im;
  }
  __device__ __forceinline__ static C zero() { return {0.f, 0.f}; }
  __device__ __forceinline__ static C add(C a, C b) { return {a.re + b.re, a.im + b.im}; }
  __device__ __forceinline__ static C sub(C a, C b) { return {a.re - b.re, a.im - b.im}; }
  __device__ __forceinline__ static C mul(C a, C b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  }
  __device__ __forceinline__ static C mul_norm(C a, C b) { return mul(a, b); }
  __device__ __forceinline__ static C conj(C a) { return {a.re, -a.im}; }
  __device__ __forceinline__ static C half(C a) { return {0.5f * a.re, 0.5f * a.im}; }
  __device__ __forceinline__ static bool finite(C a) { return isfinite(a.re) && isfinite(a.im); }
  __device__ __forceinline__ static float approx_re(C a) { return a.re; }
  __device__ __forceinline__ static float approx_im(C a) { return a.im; }
};

}  // namespace fofse
