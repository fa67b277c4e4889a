// FOFSE with the real basis of the 2-D DCT-II (Sec. 2: like the DFT, the
// DCT admits the complete transform-domain formulation).  On the T x T grid
// with the area L at its origin,
//   phi_k[m,n] = cos(pi k1 (2m+1) / (2T)) cos(pi k2 (2n+1) / (2T)),
// and with C[a1,a2] = sum w cos(pi a1 (2m+1)/(2T)) cos(pi a2 (2n+1)/(2T)) for
// 0 <= a < 2T - 1, the product-to-sum identities give
//   sum w phi_k phi_u = 1/4 sum_{+-,+-} C[|k1 +- u1|, |k2 +- u2|],
// so one iteration of the method is, on the working spectrum
// R[k] = sum w r phi_k (all T^2 bins, real):
//   u = argmax_k e_k R[k]^2,  e_k = (k1 > 0 ? 2 : 1)(k2 > 0 ? 2 : 1)
//       (the orthonormal DCT's magnitude, Eq. 9; ties: smallest k1 T + k2)
//   c = gamma R[u] / N_u,  N_u = 1/4 (C[0,0] + C[2u1,0] + C[0,2u2] + C[2u1,2u2])
//       (Eq. 5 with the weighted norm sum w phi_u^2, Eq. 14)
//   R[k] -= c/4 sum_{+-,+-} C[|k1 +- u1|, |k2 +- u2|]     for every k.
// C is kept in float-float (pairs of FP32, about 48 bits) in shared memory.
// Two iteration loops: the product one keeps the working spectrum in FP32 in
// registers with a rigorous bound on its distance to the exact recursion and
// takes every decision and coefficient from exact values (as the DFT's
// register-blocked kernel does); the other keeps every bin in float-float and
// compares exactly.  Either way the decisions are those of the exact
// algorithm up to float-float rounding.  Setup per block: R0 = DCT of w f and
// the table C of w, both by separable float-float sums over the rows of L in
// chunks (cosines from integer phases, table of the plan).  The model of B is
// rebuilt from the coefficients.
#include "fofse_fwd3.cuh"  // fixed-point recurrence sums, packed top-2 keys

namespace fofse {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

template <int T, int NT> struct Dct {
  // C[a1, a2] is needed for 0 <= a < 2T - 1; since C[2T - a1, a2] =
  // -C[a1, a2] (and the same in a2), the table holds a in [0, T] only
  static constexpr int TC = T + 1;          // rows / columns of the table
  static constexpr int S = T + 2;           // row stride of the table (float pairs)
  static constexpr int NB = T * T / NT;     // bins per thread
  static constexpr int RS = NT / T;         // rows between a thread's bins
  static constexpr int NW = NT / 32;
  static constexpr int CH = 16;             // rows of L per setup chunk
  static_assert(T * T % NT == 0 && NT % T == 0 && NB >= 1, "bin grid");
  static constexpr size_t ct_bytes = sizeof(float2) * (size_t)TC * S;  // (hi, lo) pairs
  static constexpr size_t cos_off = ct_bytes;                          // float2 [4T]
  static constexpr size_t red_off = cos_off + sizeof(float2) * 4 * T;  // float4 [2][NW], float2 [2][NW]
  // the FP32 loop's exchange slots: the same bytes as uint4 [2][NW] top-2 keys
  // and longlong2 [NW] recurrence sums, then (aux) int [NW] near-tie counts,
  // int4 [LIST] candidates, float4 [NW] + int2 [NW] warp results, int count
  static constexpr int LIST = 32;
  static constexpr size_t aux_off = red_off + 48 * NW;
  static constexpr size_t wtot_off = aux_off;
  static constexpr size_t list_off = (wtot_off + 4 * NW + 15) & ~size_t(15);
  static constexpr size_t ww_off = list_off + 16 * LIST;
  static constexpr size_t ndx_off = ww_off + 24 * NW;
  static constexpr size_t chunk_off = (ndx_off + 4 + 15) & ~size_t(15);
  // setup chunk: masked w and x = w f (CH x T each), then the row sums of C
  // (CH x TC) and of R0 (CH x T), all float-float
  static constexpr size_t chunk_bytes = sizeof(float2) * (size_t)CH * (T + T + TC + T);
  __host__ __device__ static size_t trace_bytes(int iters) { return 10 * (size_t)iters + 16; }
  // the FP32 loop keeps the exact R0 of every bin (float-float, by slot) and
  // the term list (distinct index, summed coefficient) in the chunk region
  static constexpr size_t r0x_bytes = sizeof(float2) * (size_t)T * T;
  __host__ __device__ static size_t filt_bytes(int iters) {
    return r0x_bytes + ((2 * (size_t)iters + 15) & ~size_t(15)) + 8 * (size_t)iters;
  }
  __host__ __device__ static size_t bytes(int iters, bool filt) {
    const size_t tb = filt ? filt_bytes(iters) : trace_bytes(iters);
    return 128 + chunk_off + (chunk_bytes > tb ? chunk_bytes : tb);
  }
};

// float-float accumulation of a product of two float-float numbers, without
// renormalising the sum at every step (a few dozen terms)
__device__ __forceinline__ void ff_mac(ff& acc, ff a, ff b) {
  const ff p = ff_two_prod(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  const ff s = ff_two_sum(acc.h, p.h);
  acc = {s.h, s.l + (acc.l + e)};
}
__device__ __forceinline__ ff ff_norm(ff a) { return ff_fast_two_sum(a.h, a.l); }

// One element of the row sums of the masked weights over n (row r of the
// chunk), zc[r][a] = sum_n w[r][n] cos(pi a (2n+1) / (2T)), and one element of
// C's accumulation over the chunk's rows, C[a1][a2] += sum_r cos(a1, m0 + r)
// zc[r][a2] (the order of each element's sum is fixed; the split of elements
// over threads does not enter).
template <int T, class Cos>
__device__ __forceinline__ float2 dct_row_sum(const float2* src, int a, int Ls, Cos cosv) {
  ff acc = {0.f, 0.f};
  for (int n = 0; n < Ls; ++n) {
    const float2 v = src[n];
    ff_mac(acc, ff{v.x, v.y}, cosv(a, n));
  }
  acc = ff_norm(acc);
  return make_float2(acc.h, acc.l);
}
template <int T, class Cos>
__device__ __forceinline__ float2 dct_c_accumulate(float2 c0, const float2* zc, int a1, int a2,
                                                   int m0, int nr, Cos cosv) {
  constexpr int TC = T + 1;
  ff acc = {c0.x, c0.y};
  for (int r = 0; r < nr; ++r) {
    const float2 v = zc[r * TC + a2];
    ff_mac(acc, cosv(a1, m0 + r), ff{v.x, v.y});
  }
  acc = ff_norm(acc);
  return make_float2(acc.h, acc.l);
}
// KB independent elements of either kind at once (interleaved chains for
// latency; each element's own sum runs in the order of the one-element forms
// above, so the values are the same bit for bit).  Elements with on[k] false
// are computed on a valid stand-in and not stored by the caller.
template <int T, int KB, class Cos>
__device__ __forceinline__ void dct_row_sums(const float2* (&src)[KB], const int (&a)[KB], int Ls,
                                             Cos cosv, float2 (&out)[KB]) {
  ff acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = {0.f, 0.f};
  for (int n = 0; n < Ls; ++n) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const float2 v = src[k][n];
      ff_mac(acc[k], ff{v.x, v.y}, cosv(a[k], n));
    }
  }
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const ff r = ff_norm(acc[k]);
    out[k] = make_float2(r.h, r.l);
  }
}
template <int T, int KB, class Cos>
__device__ __forceinline__ void dct_c_accumulates(float2 (&c)[KB], const float2* zc, const int (&a1)[KB],
                                                  const int (&a2)[KB], int m0, int nr, Cos cosv) {
  constexpr int TC = T + 1;
  ff acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = {c[k].x, c[k].y};
  for (int r = 0; r < nr; ++r) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const float2 v = zc[r * TC + a2[k]];
      ff_mac(acc[k], cosv(a1[k], m0 + r), ff{v.x, v.y});
    }
  }
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const ff r = ff_norm(acc[k]);
    c[k] = make_float2(r.h, r.l);
  }
}

// The table index of C's index a in [0, 2T - 1) and its sign: C[2T - a] =
// -C[a], since cos(pi (2T - a)(2m+1) / (2T)) = -cos(pi a (2m+1) / (2T))
template <int T> __device__ __forceinline__ int dct_fold(int a, float& sign) {
  const bool hi = a > T;
  sign = hi ? -1.f : 1.f;
  return hi ? 2 * T - a : a;
}
__device__ __forceinline__ ff ff_sign(ff a, float s) { return {a.h * s, a.l * s}; }

// (m, n) of L in the support shape and outside B
__device__ __forceinline__ bool dct_in_support(int support, int m, int n, int b, int br) {
  const bool inB = m >= br && m < br + b && n >= br && n < br + b;
  bool inS = true;
  if (support == FOFSE_SUPPORT_CAUSAL_L) inS = (m < br) ? (n < br + b) : (m < br + b ? n < br : false);
  return inS && !inB;
}

// (a, b) better than (c, d): larger value, or equal value and smaller index
__device__ __forceinline__ bool better(ff a, int ia, ff b, int ib) {
  return a.h > b.h || (a.h == b.h && (a.l > b.l || (a.l == b.l && ia < ib)));
}

// The exact value's correction at bin (k1, k2) from the terms j in {j0, j0 +
// stride, ...} < j1 of the term list (distinct index v_j, summed coefficient
// c_j, float-float):  sum_j c_j / 4 sum_{+-,+-} C[|k1 +- v1|, |k2 +- v2|],
// each term in float-float from the table C in shared memory, returned in
// fixed point with unit 1/scale (so that warp and block sums are exact).
template <int T>
__device__ __forceinline__ long long dct_recur(const float2* ct, const short* ty, const float2* tc,
                                               int k1, int k2, int j0, int j1, int stride,
                                               float scale) {
  constexpr int S = T + 2, LOGT = ilog2(T);
  ff acc = {0.f, 0.f};
  for (int j = j0; j < j1; j += stride) {
    const int y = ty[j];
    const int v1 = y >> LOGT, v2 = y & (T - 1);
    const float2 cj = tc[j];
    float sr, sc;
    const int rp = dct_fold<T>(k1 + v1, sr) * S, rm = abs(k1 - v1) * S;
    const int cp = dct_fold<T>(k2 + v2, sc), cm = abs(k2 - v2);
    const float2 a = ct[rp + cp], b = ct[rp + cm], c = ct[rm + cp], d = ct[rm + cm];
    const ff sum = ff_add(ff_sign(ff_add(ff_sign(ff{a.x, a.y}, sc), ff{b.x, b.y}), sr),
                          ff_add(ff_sign(ff{c.x, c.y}, sc), ff{d.x, d.y}));
    acc = ff_add(acc, ff_mul(ff{cj.x, cj.y}, sum));
  }
  const float sq = 0.25f * scale;  // the 1/4, exactly
  return fx_round(acc.h * sq) + fx_round(acc.l * sq);
}

// e_k R^2 in float-float (the comparison value of Eq. 9 with the orthonormal
// DCT's magnitude), e a power of two
__device__ __forceinline__ ff dct_energy(ff r, float e) {
  const ff q = ff_two_prod(r.h, r.h);
  const ff e2 = ff_fast_two_sum(q.h, __fmaf_rn(2.f * r.h, r.l, q.l));
  return {e2.h * e, e2.l * e};
}

template <int T, int NT, bool FILT>
__device__ __forceinline__ void forward_block_dct(const FwdArgs& args, int blk, unsigned char* dsm) {
  using G = Dct<T, NT>;
  using IO = PlanIO<ArFF>;
  constexpr int TC = G::TC, S = G::S, NB = G::NB, RS = G::RS, NW = G::NW, CH = G::CH;
  float2* ct = reinterpret_cast<float2*>(dsm);
  float2* cosT = reinterpret_cast<float2*>(dsm + G::cos_off);
  float4* redv = reinterpret_cast<float4*>(dsm + G::red_off);             // [2][NW]: e.h, e.l, idx, -
  float2* redr = reinterpret_cast<float2*>(dsm + G::red_off + 32 * NW);  // [2][NW]: R[idx]
  unsigned char* chunk = dsm + G::chunk_off;
  float2* wsm = reinterpret_cast<float2*>(chunk);                  // [CH][T]
  float2* xsm = wsm + CH * T;                                      // [CH][T]
  float2* zc = xsm + CH * T;                                       // [CH][TC]
  float2* yc = zc + CH * TC;                                       // [CH][T]
  const PlanDev& P = args.plan;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int iters = P.iters, b = P.block, br = P.border, Ls = P.Ls;
  const fofse_block bd = args.blocks[blk];
  const int ly0 = bd.y - br, lx0 = bd.x - br;
  auto cosv = [&](int a, int m) -> ff {  // cos(pi a (2m+1) / (2T))
    const float2 v = cosT[(a * (2 * m + 1)) & (4 * T - 1)];
    return {v.x, v.y};
  };

  // ---- setup: C and R0 by chunks of CH rows of L ----------------------------
  // C is linear in w.  With the complete-support table C_full of the plan (or
  // of the call's rho), a block starts from C_full and subtracts the
  // contribution of its missing samples (in the support shape, outside B, but
  // not usable), summed over the chunks of rows that hold any: a block whose
  // support is complete only copies the table.  Without a table, C is summed
  // over every chunk from the usable samples.
  const bool have_table = P.tab.dct_c_full != nullptr;
  for (int e = tid; e < 4 * T; e += NT) cosT[e] = P.tab.dct_cos_ff[e];
  if (have_table) {
    const float4* src = reinterpret_cast<const float4*>(P.tab.dct_c_full);
    float4* dst = reinterpret_cast<float4*>(ct);
    for (int e = tid; e < TC * S / 2; e += NT) dst[e] = src[e];
  } else {
    for (int e = tid; e < TC * S; e += NT) ct[e] = make_float2(0.f, 0.f);
  }
  const int k2 = tid & (T - 1), r0 = tid / T;  // bins (r0 + j RS, k2)
  ff R[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) R[j] = {0.f, 0.f};
  bool bad = false, use = false;
  __syncthreads();
  for (int m0 = 0; m0 < Ls; m0 += CH) {
    const int nr = min(CH, Ls - m0);
    // weights for C (with a table: the missing samples' weights, negated;
    // else the usable samples' weights) and weighted samples of rows
    // m0 .. m0 + nr (zero beyond Ls)
    bool cmiss = false;
    for (int e = tid; e < CH * T; e += NT) {
      const int r = e / T, n = e - r * T, m = m0 + r;
      float2 wv = make_float2(0.f, 0.f), xv = make_float2(0.f, 0.f);
      if (r < nr && n < Ls && dct_in_support(P.support, m, n, b, br)) {
        const int fy = ly0 + m, fx = lx0 + n;
        const bool in = fy >= 0 && fy < args.height && fx >= 0 && fx < args.width;
        if (in && args.avail[(size_t)fy * args.pitch + fx]) {
          const float f = args.frame[(size_t)fy * args.pitch + fx];
          bad |= !isfinite(f);
          use = true;
          ArFF::C wd;
          const ArFF::C z = IO::weighted(P.tab, m * Ls + n, f, wd);
          if (!have_table) wv = make_float2(wd.re.h, wd.re.l);
          xv = make_float2(z.re.h, z.re.l);
        } else if (have_table) {
          const float2 w = P.tab.w_ff[m * Ls + n];
          wv = make_float2(-w.x, -w.y);
          cmiss = true;
        }
      }
      wsm[e] = wv;
      xsm[e] = xv;
    }
    // this chunk's rows change C (a barrier either way)
    const bool full = have_table && !__syncthreads_or(cmiss);
    // row sums over n: zc[r][a2] = sum_n w cos(a2, n) (only for chunks that
    // change C), yc[r][k] = sum_n x cos(k, n)
    // (KB elements per thread and pass)
    constexpr int KB = 4;
    {
      const int e0 = full ? CH * TC : 0, e1 = CH * (TC + T);
      for (int eb = e0 + tid; eb < e1; eb += KB * NT) {
        const float2* src[KB];
        int a[KB], dst[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const int e = eb + k * NT;
          const bool on = e < e1;
          const int ec = on ? e : e0;
          const bool isz = ec < CH * TC;
          const int ee = isz ? ec : ec - CH * TC;
          const int r = isz ? ee / TC : ee / T;
          a[k] = isz ? ee - r * TC : ee - r * T;
          src[k] = (isz ? wsm : xsm) + r * T;
          dst[k] = on ? (isz ? r * TC + a[k] : CH * TC + r * T + a[k]) : -1;  // zc, then yc
        }
        float2 v[KB];
        dct_row_sums<T, KB>(src, a, Ls, cosv, v);
#pragma unroll
        for (int k = 0; k < KB; ++k)
          if (dst[k] >= 0) zc[dst[k]] = v[k];  // yc follows zc in the chunk region
      }
    }
    __syncthreads();
    // C[a1][a2] += sum_r cos(a1, m0 + r) zc[r][a2]
    if (!full) {
      for (int eb = tid; eb < TC * TC; eb += KB * NT) {
        int a1[KB], a2[KB];
        float2 c[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const int e = eb + k * NT, ec = e < TC * TC ? e : 0;
          a1[k] = ec / TC;
          a2[k] = ec - a1[k] * TC;
          c[k] = ct[a1[k] * S + a2[k]];
        }
        dct_c_accumulates<T, KB>(c, zc, a1, a2, m0, nr, cosv);
#pragma unroll
        for (int k = 0; k < KB; ++k)
          if (eb + k * NT < TC * TC) ct[a1[k] * S + a2[k]] = c[k];
      }
    }
    // R0 of the held bins: R[k1][k2] += sum_r cos(k1, m0 + r) yc[r][k2]
    // (the bins' chains interleaved, each over r in order)
    {
      ff acc[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) acc[j] = R[j];
      for (int r = 0; r < nr; ++r) {
        const float2 v = yc[r * T + k2];
#pragma unroll
        for (int j = 0; j < NB; ++j) ff_mac(acc[j], cosv(r0 + j * RS, m0 + r), ff{v.x, v.y});
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) R[j] = ff_norm(acc[j]);
    }
    __syncthreads();
  }
  const int any_bad = __syncthreads_or(bad);
  // no usable sample: C_full minus every sample's part need not round to 0
  const int any_use = __syncthreads_or(use);
  // the chunk region now holds the trace: packed index and coefficient
  short* trU = reinterpret_cast<short*>(chunk);
  float2* trC = reinterpret_cast<float2*>(chunk + ((2 * (size_t)iters + 15) & ~size_t(15)));
  const ff W0 = {ct[0].x, ct[0].y};  // C[0,0] = sum w
  int st = FOFSE_BLK_OK;
  if (!any_use || W0.h == 0.f) st = FOFSE_BLK_NO_SUPPORT;
  else if (any_bad || !isfinite(W0.h)) st = FOFSE_BLK_NONFINITE;

  int done_it = 0;  // iterations the FP32 loop ran (any later one repeats a zero residual's (0, 0), 0)
  if (st == FOFSE_BLK_OK) {
    if constexpr (FILT) {
      // ---- FP32 working spectrum with exact decisions ----
      // As in the register-blocked DFT kernel: R32 (FP32, registers) with a
      // running bound B on its distance to the exact recursion; the block's
      // FP32 top-2 of e_k R32[k]^2 decide the argmax when further apart than
      // the bound allows (sqrt(e_k) <= 2 scales B), otherwise every bin that
      // can still win is evaluated exactly and compared in float-float; the
      // winner's exact value comes from the recurrence
      //   R~[k] = R0[k] - sum_j c_j / 4 sum_{+-,+-} C[|k1 +- v1|, |k2 +- v2|]
      // over the distinct selected indices v_j (summed coefficients c_j).
      // Bound per update R <- fma(-c/4, s, R), s the FP32 sum of the four
      // C entries (hi parts; |C[a]| <= C[0,0] = W[0]): rounding C to FP32
      // (u W[0] each), the two-level sum (8u W[0]), c to FP32 (u |c|) and the
      // fma (u |R_new|) give u |R_new| + 4u |c| W[0]; the kernel adds
      // 1.5u max|R32| + 6u |c| W[0] per iteration (the first term of the
      // first iteration also covers the rounding of R0 to FP32).
      constexpr int LIST = G::LIST;
      constexpr float kU = 5.9604644775390625e-08f;  // 2^-24
      constexpr float kDn = 1.f - 16.f * kU, kUp = 1.f + 256.f * kU, kUpB = 1.f + 16.f * kU;
      constexpr float kTiny = 7.888609052210118e-31f;     // 2^-100
      constexpr float kTinySqrt = 8.881784197001252e-16f; // 2^-50
      constexpr float kA = 1.5f * kU, kB = 6.f * kU;
      uint4* t2s = reinterpret_cast<uint4*>(dsm + G::red_off);                  // [2][NW]
      longlong2* redx = reinterpret_cast<longlong2*>(dsm + G::red_off + 32 * NW);  // [NW]
      int* wtot = reinterpret_cast<int*>(dsm + G::wtot_off);
      int4* list = reinterpret_cast<int4*>(dsm + G::list_off);
      float4* wwv = reinterpret_cast<float4*>(dsm + G::ww_off);
      int2* wwc = reinterpret_cast<int2*>(dsm + G::ww_off + 16 * NW);
      int* ndx = reinterpret_cast<int*>(dsm + G::ndx_off);
      float2* R0x = reinterpret_cast<float2*>(chunk);  // exact R0 by slot tid + j NT
      short* trY = reinterpret_cast<short*>(chunk + G::r0x_bytes);
      float2* trCm = reinterpret_cast<float2*>(chunk + G::r0x_bytes + ((2 * (size_t)iters + 15) & ~size_t(15)));
      const ff gam = IO::gamma(P);
      const float W0f = W0.h * (1.f + 1e-6f);
      float R32[NB], ew[NB];
      unsigned m1k = 0u, m2k = 0u;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        R0x[tid + j * NT] = make_float2(R[j].h, R[j].l);
        R32[j] = R[j].h;
        ew[j] = (r0 + j * RS > 0 ? 2.f : 1.f) * (k2 > 0 ? 2.f : 1.f);
        key_insert(m1k, m2k, ew[j] * (R32[j] * R32[j]), j);
      }
      float bnd = 0.f, prevabs = 0.f, csum = 0.f;
      int nd = 0;  // terms in the list (warp 0 maintains it; the others read it each iteration)
      // entries before nb belong to coefficients taken into R0 by a rebase
      // (below): they count for the synthesis only
      int nb = 0;
      __syncthreads();
      int it = 0;
#pragma unroll 1
      for (; it < iters; ++it) {
        // ---- top-2 over the block (packed keys) ----
        const unsigned wm1 = __reduce_max_sync(kFullMask, m1k);
        const unsigned hold = __ballot_sync(kFullMask, m1k == wm1);
        const int ldr = __ffs(hold) - 1;
        const unsigned wm2 = __reduce_max_sync(kFullMask, lane == ldr ? m2k : m1k);
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
        const float q1 = m1 * rsqrtf(n1 ? m1 : 1.f), q2 = m2 * rsqrtf(n2 ? m2 : 1.f);
        const float sM1 = n1 ? q1 : 0.f, sM1u = n1 ? q1 * kUp : kTinySqrt;
        const float sM2 = n2 ? q2 : kTinySqrt;
        bnd += kA * sM1u + kB * W0f * prevabs;
        const float bw = 2.f * bnd;  // bound of sqrt(e_k) |R32[k] - R~[k]|
        const bool certain = (sM1 * kDn - bw * kUpB) > (sM2 * kUp + bw * kUpB);
        const int sh = fx_shift(4.f * W0f * csum);
        const float scale = pow2f(sh), iscale = pow2f(-sh);
        int u1, u2;
        ff Rt;
        if (certain) {
          const int wt = (int)g.z, li = (int)(g.x & kKeyMask);
          u1 = wt / T + li * RS;
          u2 = wt & (T - 1);
          const float2 rx = R0x[wt + li * NT];
          long long sv = 0;
          if (warp * 32 < nd - nb) {  // warp-uniform: this warp holds terms
            sv = dct_recur<T>(ct, trY, trCm, u1, u2, nb + tid, nd, NT, scale);
            sv = redux_sum64(sv);
          }
          if (lane == 0) redx[warp] = make_longlong2(sv, 0);
          __syncthreads();
          const longlong2 v = lane < NW ? redx[lane] : make_longlong2(0, 0);
          Rt = ff_sub(ff{rx.x, rx.y}, fx_to_ff(redux_sum64(v.x), iscale));
        } else {
          // ---- near-tie: exact values of every bin that can still win ----
          const float Lb = (sM1 * kDn - 2.f * bw * kUpB) * kDn;
          const float thr = Lb > 0.f ? Lb * Lb * kDn : -1.f;
          int cnt = 0;
#pragma unroll
          for (int j = 0; j < NB; ++j) cnt += ew[j] * (R32[j] * R32[j]) >= thr ? 1 : 0;
          int incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFullMask, incl, o);
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
          ff wbe = {-1.f, 0.f}, wbr = {0.f, 0.f};
          int wbl = 0x7fffffff;
          const bool rebase = total > T * T / 4;
          if (rebase) {
            // ---- rebase: the bound has grown to the size of the residual
            // (a residual that decays far, as over flat content) and nearly
            // every bin is a candidate.  Each thread evaluates its own bins
            // exactly; these values become R0 (the recurrence continues from
            // entry nb), R32 their FP32 roundings, and the bound restarts.
#pragma unroll 1
            for (int j = 0; j < NB; ++j) {
              const int k1 = r0 + j * RS, lin = k1 * T + k2;
              const float2 rx = R0x[tid + j * NT];
              const long long sv = dct_recur<T>(ct, trY, trCm, k1, k2, nb, nd, 1, scale);
              const ff rv = ff_sub(ff{rx.x, rx.y}, fx_to_ff(sv, iscale));
              R0x[tid + j * NT] = make_float2(rv.h, rv.l);
              const ff ev = dct_energy(rv, (k1 > 0 ? 2.f : 1.f) * (k2 > 0 ? 2.f : 1.f));
              if (better(ev, lin, wbe, wbl)) {
                wbe = ev;
                wbl = lin;
                wbr = rv;
              }
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) R32[j] = R0x[tid + j * NT].x;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const ff oe = {__shfl_xor_sync(kFullMask, wbe.h, o), __shfl_xor_sync(kFullMask, wbe.l, o)};
              const ff orv = {__shfl_xor_sync(kFullMask, wbr.h, o), __shfl_xor_sync(kFullMask, wbr.l, o)};
              const int ol = __shfl_xor_sync(kFullMask, wbl, o);
              if (better(oe, ol, wbe, wbl)) {
                wbe = oe;
                wbl = ol;
                wbr = orv;
              }
            }
            nb = nd;
            csum = 0.f;
          }
          for (int pass = 0; !rebase && pass < total; pass += LIST) {
            int r = rank0;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
              if (ew[j] * (R32[j] * R32[j]) >= thr) {
                if (r >= pass && r < pass + LIST)
                  list[r - pass] = make_int4((r0 + j * RS) * T + k2, tid + j * NT, __float_as_int(ew[j]), 0);
                ++r;
              }
            }
            __syncthreads();
            const int n = min(LIST, total - pass);
            for (int c = warp; c < n; c += NW) {
              const int4 e = list[c];
              const int c1 = e.x / T, c2 = e.x - c1 * T;
              const float2 rx = R0x[e.y];
              long long sv = dct_recur<T>(ct, trY, trCm, c1, c2, nb + lane, nd, 32, scale);
              sv = redux_sum64(sv);
              const ff rv = ff_sub(ff{rx.x, rx.y}, fx_to_ff(sv, iscale));
              const ff ev = dct_energy(rv, __int_as_float(e.z));
              if (better(ev, e.x, wbe, wbl)) {
                wbe = ev;
                wbl = e.x;
                wbr = rv;
              }
            }
            __syncthreads();
          }
          if (lane == 0) {
            wwv[warp] = make_float4(wbe.h, wbe.l, wbr.h, wbr.l);
            wwc[warp] = make_int2(wbl, 0);
          }
          __syncthreads();
          ff be = {-1.f, 0.f};
          int bl = 0x7fffffff;
          Rt = {0.f, 0.f};
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            const float4 v4 = wwv[w];
            const int l = wwc[w].x;
            if (l != 0x7fffffff && better(ff{v4.x, v4.y}, l, be, bl)) {
              be = {v4.x, v4.y};
              bl = l;
              Rt = {v4.z, v4.w};
            }
          }
          if (bl == 0x7fffffff) bl = 0;  // no candidate (cannot happen for finite data)
          u1 = bl / T;
          u2 = bl - u1 * T;
          // after a rebase the bound restarts from the roundings of the new
          // R0 to FP32: u |R[k]| <= 2u |R[u]| (e_u R[u]^2 is the largest
          // e_k R[k]^2 and e_k / e_u >= 1/4)
          if (rebase) bnd = 2.f * kA * fabsf(Rt.h) * kUp;
        }
        // ---- coefficient (Eq. 5, Eq. 14) ----
        float s1n, s2n;
        const int f1 = dct_fold<T>(2 * u1, s1n) * S, f2 = dct_fold<T>(2 * u2, s2n);
        const float2 n0 = ct[0], n1c = ct[f1], n2c = ct[f2], n3 = ct[f1 + f2];
        ff nrm = ff_add(ff_add(ff{n0.x, n0.y}, ff_sign(ff{n1c.x, n1c.y}, s1n)),
                        ff_add(ff_sign(ff{n2c.x, n2c.y}, s2n), ff_sign(ff{n3.x, n3.y}, s1n * s2n)));
        nrm = ff_scale(nrm, 0.25f);
        const ff cff = nrm.h > 0.f ? ff_div(ff_mul(gam, Rt), nrm) : ff{0.f, 0.f};
        // ---- record: the trace entry, and the term of the recurrence ----
        // (every read of the list in this iteration lies before a barrier
        // that precedes this update)
        if (warp == 0) {
          const short y = (short)(u1 * T + u2);
          int pos = -1;
          for (int j0 = nb; j0 < nd; j0 += 32) {
            const int jj = j0 + lane;
            const unsigned hit = __ballot_sync(kFullMask, jj < nd && trY[jj] == y);
            if (hit) {
              pos = j0 + __ffs(hit) - 1;
              break;
            }
          }
          if (lane == 0) {
            if (pos >= 0) {
              const float2 o = trCm[pos];
              const ff sm = ff_add(ff{o.x, o.y}, cff);
              trCm[pos] = make_float2(sm.h, sm.l);
            } else {
              trY[nd] = y;
              trCm[nd] = make_float2(cff.h, cff.l);
            }
            if (args.trace) {
              fofse_trace_entry e;
              e.u1 = (int16_t)u1;
              e.u2 = (int16_t)u2;
              e.dc_re = cff.h;
              e.dc_im = 0.f;
              args.trace[(size_t)blk * args.trace_stride + it] = e;
            }
          }
          if (pos < 0) ++nd;
        }
        // an exactly zero winner (the exact maximum of e_k R~[k]^2) means a
        // zero residual in every bin: every later iteration selects (0, 0),
        // as this one did, with a zero coefficient; they are written as such
        // at the end instead of being run
        if (Rt.h == 0.f && Rt.l == 0.f) {
          ++it;
          break;
        }
        // ---- FP32 update R -= c/4 sum C[|k1 +- u1|, |k2 +- u2|] + next keys ----
        const float p = cff.h, c4 = 0.25f * p;
        prevabs = fabsf(p);
        csum += prevabs;
        float sgc;
        const int cp = dct_fold<T>(k2 + u2, sgc), cm = abs(k2 - u2);
        m1k = 0u;
        m2k = 0u;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const int k1 = r0 + j * RS;
          float sgr;
          const int rp = dct_fold<T>(k1 + u1, sgr) * S, rm = abs(k1 - u1) * S;
          // the four entries with their signs: sums of the same shape and
          // rounding as without the folding (the signs are exact)
          const float sv = __fmaf_rn(sgr, __fmaf_rn(sgc, ct[rp + cp].x, ct[rp + cm].x),
                                     __fmaf_rn(sgc, ct[rm + cp].x, ct[rm + cm].x));
          R32[j] = __fmaf_rn(-c4, sv, R32[j]);
          key_insert(m1k, m2k, ew[j] * (R32[j] * R32[j]), j);
        }
      }
      done_it = it;
      if (tid == 0) *ndx = nd;  // thread 0 is in warp 0, which holds the count
    } else {
      const ff gam = IO::gamma(P);
      // this thread's best bin by e_k R[k]^2 (exact comparison in float-float),
      // found again after every update
      ff best = {-1.f, 0.f}, bestR = {0.f, 0.f};
      int bidx = 0x7fffffff;
      // the thread's best bin: every bin's value, then a pairwise tree (the
      // order "larger value, then smaller index" is total, so the tree finds the
      // bin a scan would, with a dependency depth of log2(NB) instead of NB)
      auto thread_best = [&]() {
        ff ev[NB], rv[NB];
        int ix[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const int k1 = r0 + j * RS;
          const float sc = (k1 > 0 ? 2.f : 1.f) * (k2 > 0 ? 2.f : 1.f);
          const ff q = ff_two_prod(R[j].h, R[j].h);
          const ff e2 = ff_fast_two_sum(q.h, __fmaf_rn(2.f * R[j].h, R[j].l, q.l));
          ev[j] = {e2.h * sc, e2.l * sc};
          ix[j] = k1 * T + k2;
          rv[j] = R[j];
        }
#pragma unroll
        for (int w = 1; w < NB; w *= 2) {
#pragma unroll
          for (int j = 0; j + w < NB; j += 2 * w) {
            if (better(ev[j + w], ix[j + w], ev[j], ix[j])) {
              ev[j] = ev[j + w];
              ix[j] = ix[j + w];
              rv[j] = rv[j + w];
            }
          }
        }
        best = ev[0];
        bidx = ix[0];
        bestR = rv[0];
      };
      thread_best();
#pragma unroll 1
      for (int it = 0; it < iters; ++it) {
        // ---- block argmax ----
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const ff ob = {__shfl_xor_sync(kFullMask, best.h, o), __shfl_xor_sync(kFullMask, best.l, o)};
          const int oi = __shfl_xor_sync(kFullMask, bidx, o);
          const ff orr = {__shfl_xor_sync(kFullMask, bestR.h, o), __shfl_xor_sync(kFullMask, bestR.l, o)};
          if (better(ob, oi, best, bidx)) {
            best = ob;
            bidx = oi;
            bestR = orr;
          }
        }
        float4* rv = redv + (it & 1) * NW;
        float2* rr = redr + (it & 1) * NW;
        if (lane == 0) {
          rv[warp] = make_float4(best.h, best.l, __int_as_float(bidx), 0.f);
          rr[warp] = make_float2(bestR.h, bestR.l);
        }
        __syncthreads();
        float4 g = rv[0];
        float2 gr = rr[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) {
          const float4 o = rv[w];
          if (better(ff{o.x, o.y}, __float_as_int(o.z), ff{g.x, g.y}, __float_as_int(g.z))) {
            g = o;
            gr = rr[w];
          }
        }
        int ui = __float_as_int(g.z);
        if (ui < 0 || ui >= T * T) ui = 0;  // no comparable value (cannot happen for finite data)
        const int u1 = ui / T, u2 = ui - u1 * T;
        // ---- coefficient (Eq. 5, Eq. 14) ----
        float s1n, s2n;
        const int f1 = dct_fold<T>(2 * u1, s1n) * S, f2 = dct_fold<T>(2 * u2, s2n);
        const float2 n0 = ct[0], n1 = ct[f1], n2 = ct[f2], n3 = ct[f1 + f2];
        ff nrm = ff_add(ff_add(ff{n0.x, n0.y}, ff_sign(ff{n1.x, n1.y}, s1n)),
                        ff_add(ff_sign(ff{n2.x, n2.y}, s2n), ff_sign(ff{n3.x, n3.y}, s1n * s2n)));
        nrm = ff_scale(nrm, 0.25f);
        const ff cff = nrm.h > 0.f ? ff_div(ff_mul(gam, ff{gr.x, gr.y}), nrm) : ff{0.f, 0.f};
        if (tid == 0) {
          trU[it] = (short)ui;
          trC[it] = make_float2(cff.h, cff.l);
        }
        // ---- R[k] -= c/4 sum C[|k1 +- u1|, |k2 +- u2|], and the next best ----
        const ff c4 = ff_scale(cff, 0.25f);
        float sgc;
        const int cp = dct_fold<T>(k2 + u2, sgc), cm = abs(k2 - u2);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const int k1 = r0 + j * RS;
          float sgr;
          const int rp = dct_fold<T>(k1 + u1, sgr) * S, rm = abs(k1 - u1) * S;
          const float2 ap = ct[rp + cp], bp = ct[rp + cm], cp2 = ct[rm + cp];
          const float sa = sgr * sgc, sb = sgr;
          const float2 a = make_float2(ap.x * sa, ap.y * sa), bq = make_float2(bp.x * sb, bp.y * sb);
          const float2 cq = make_float2(cp2.x * sgc, cp2.y * sgc), d = ct[rm + cm];
          // four-term float-float sum: exact sums of the high parts, low parts added
          const ff s1 = ff_two_sum(a.x, bq.x), s2 = ff_two_sum(cq.x, d.x), s = ff_two_sum(s1.h, s2.h);
          const float lo = ((a.y + bq.y) + (cq.y + d.y)) + (s1.l + s2.l) + s.l;
          // R - c4 t with one product and one compensated subtraction
          const ff pr = ff_two_prod(c4.h, s.h);
          const float pe = __fmaf_rn(c4.h, lo, __fmaf_rn(c4.l, s.h, pr.l));
          const ff dd = ff_two_sum(R[j].h, -pr.h);
          R[j] = ff_fast_two_sum(dd.h, dd.l + (R[j].l - pe));
        }
        thread_best();
      }
    }
  }
  __syncthreads();

  // ---- synthesis of B (Eq. 1) from the trace; outputs ----------------------
  const int nIt = st == FOFSE_BLK_OK ? iters : 0;
  // the terms: one per iteration, or (FP32 loop) one per distinct index
  const short* syY = trU;
  const float2* syC = trC;
  int nSyn = nIt;
  if constexpr (FILT) {
    syY = reinterpret_cast<const short*>(chunk + G::r0x_bytes);
    syC = reinterpret_cast<const float2*>(chunk + G::r0x_bytes + ((2 * (size_t)iters + 15) & ~size_t(15)));
    nSyn = st == FOFSE_BLK_OK ? *reinterpret_cast<const int*>(dsm + G::ndx_off) : 0;
  }
  const int ld = args.out_ld;
  for (int pidx = tid; pidx < ld * ld; pidx += NT) {
    const int bm = pidx / ld, bn = pidx - bm * ld;
    float v = 0.f;
    if (bm < b && bn < b) {
      const int m = br + bm, n = br + bn;
      ff acc = {0.f, 0.f};
      for (int i = 0; i < nSyn; ++i) {
        const int yy = syY[i];
        const int a1 = yy / T, a2 = yy - a1 * T;
        const float2 c = syC[i];
        ff_mac(acc, ff{c.x, c.y}, ff_mul(cosv(a1, m), cosv(a2, n)));
      }
      acc = ff_norm(acc);
      v = acc.h + acc.l;
      if (args.out_frame) {
        const int fy = bd.y + bm, fx = bd.x + bn;
        if (fy >= 0 && fy < args.height && fx >= 0 && fx < args.width)
          args.out_frame[(size_t)fy * args.pitch + fx] = v;
      }
    }
    if (args.out_blocks) args.out_blocks[(size_t)blk * args.out_stride + pidx] = v;
  }
  if (args.trace) {  // (the FP32 loop wrote its iterations' entries as they ran)
    for (int i = (FILT ? done_it : 0) + tid; i < args.trace_stride; i += NT) {
      fofse_trace_entry e;
      if (!FILT && i < nIt) {
        const int yy = trU[i];
        e.u1 = (int16_t)(yy / T);
        e.u2 = (int16_t)(yy - (yy / T) * T);
        e.dc_re = trC[i].x;
      } else {
        e.u1 = e.u2 = 0;
        e.dc_re = 0.f;
      }
      e.dc_im = 0.f;
      args.trace[(size_t)blk * args.trace_stride + i] = e;
    }
  }
  if (args.gamma_out) {
    for (int i = tid; i < args.trace_stride; i += NT)
      args.gamma_out[(size_t)blk * args.trace_stride + i] =
          make_float2(i < nIt ? IO::gamma(P).h : 0.f, 0.f);
  }
  if (tid == 0) {
    if (args.w0) args.w0[blk] = st == FOFSE_BLK_OK ? W0.h + W0.l : 0.f;
    if (args.status) args.status[blk] = st;
  }
  __syncthreads();
}

template <int T, int NT, bool FILT>
__global__ void __launch_bounds__(NT) fofse_forward_dct_kernel(const __grid_constant__ FwdArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];  // 16-byte slots, no TMA
  unsigned char* dsm = smem_raw;
  __shared__ int s_item;
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
    forward_block_dct<T, NT, FILT>(args, item, dsm);
  }
}

// The table C of the complete support of plan P (every sample of L in the
// support shape and outside B usable): C[a1][a2] = sum_m cos(a1, m) zc[m][a2],
// zc[m][a2] = sum_n w[m][n] cos(a2, n), in float-float.  A CTA owns DCT_TAB_A
// columns a2 of C: it sums zc for its columns over every row m of L, then its
// columns of C over m (renormalised every 16 rows), for a1, a2 in [0, T];
// the padding column a2 = T + 1 is written as 0.  The same kernel builds the plan's table and the
// per-call table of a call with device-side (rho, gamma), so both hold the
// same values for the same rho, bit for bit.
constexpr int DCT_TAB_A = 4;
constexpr int DCT_TAB_NT = 256;
template <int T> __host__ __device__ constexpr size_t dct_table_smem() {
  return sizeof(float2) * ((size_t)T * T + 4 * T + (size_t)T * DCT_TAB_A);
}
template <int T>
__global__ void __launch_bounds__(DCT_TAB_NT) fofse_dct_table_kernel(const PlanDev P, float2* out) {
  constexpr int TC = T + 1, S = T + 2, A = DCT_TAB_A, NT = DCT_TAB_NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];  // 8-byte slots, no TMA
  float2* wsm = reinterpret_cast<float2*>(smem_raw);  // [Ls][Ls] masked w
  float2* cosT = wsm + T * T;                         // [4T]
  float2* zc = cosT + 4 * T;                          // [Ls][A]
  const int tid = threadIdx.x, b = P.block, br = P.border, Ls = P.Ls;
  const int c0 = blockIdx.x * A;
  auto cosv = [&](int a, int m) -> ff {
    const float2 v = cosT[(a * (2 * m + 1)) & (4 * T - 1)];
    return {v.x, v.y};
  };
  for (int e = tid; e < 4 * T; e += NT) cosT[e] = P.tab.dct_cos_ff[e];
  for (int e = tid; e < Ls * Ls; e += NT) {
    const int m = e / Ls, n = e - m * Ls;
    wsm[e] = dct_in_support(P.support, m, n, b, br) ? P.tab.w_ff[e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int e = tid; e < Ls * A; e += NT) {
    const int m = e / A, a2 = min(c0 + e % A, TC - 1);
    zc[e] = dct_row_sum<T>(wsm + m * Ls, a2, Ls, cosv);
  }
  __syncthreads();
  for (int e = tid; e < TC * A; e += NT) {
    const int a1 = e / A, j = e - a1 * A, a2 = c0 + j;
    if (a2 >= S) continue;
    float2 c = make_float2(0.f, 0.f);
    if (a2 < TC) {
      ff acc = {0.f, 0.f};
      for (int m0 = 0; m0 < Ls; m0 += 16) {
        for (int m = m0; m < min(m0 + 16, Ls); ++m) {
          const float2 v = zc[m * A + j];
          ff_mac(acc, cosv(a1, m), ff{v.x, v.y});
        }
        acc = ff_norm(acc);
      }
      c = make_float2(acc.h, acc.l);
    }
    out[(size_t)a1 * S + a2] = c;
  }
}

template <int T> cudaError_t build_dct_table_T(const PlanDev& p, float2* out, cudaStream_t s) {
  constexpr size_t sm = dct_table_smem<T>();
  static_assert(sm <= 48 * 1024, "table kernel shared memory");
  constexpr int grid = (T + 2 + DCT_TAB_A - 1) / DCT_TAB_A;  // the S columns of the table
  fofse_dct_table_kernel<T><<<grid, DCT_TAB_NT, sm, s>>>(p, out);
  return cudaGetLastError();
}

template <int T, int NT, bool FILT> struct VariantDct {
  static cudaError_t launch(const FwdArgs& a, cudaStream_t s) {
    const size_t sm = Dct<T, NT>::bytes(a.plan.iters, FILT);
    int grid = 0;
    const cudaError_t e = prepare_kernel(fofse_forward_dct_kernel<T, NT, FILT>, NT, sm, &grid);
    if (e != cudaSuccess) return e;
    if (grid > a.n_blocks) grid = a.n_blocks;
    if (grid < 1) return cudaSuccess;
    fofse_forward_dct_kernel<T, NT, FILT><<<grid, NT, sm, s>>>(a);
    return cudaGetLastError();
  }
};

// ---------------------------------------------------------------------------
// Backward (adjoint along the frozen path) with the DCT basis.  With
// c_i = gamma p_i / N_i, p_i = sum_A w (f - g_{i-1}) phi_i, N_i = sum_A w phi_i^2
// and B_hat = sum_i c_i phi_i on B, for the loss gradient e on B, in reverse
// order of the iterations:
//   cbar_i = sum_L gbar phi_i            (gbar starts as e on B)
//   gammabar += cbar_i c_i / gamma
//   pbar = gamma cbar_i / N_i, Nbar = -cbar_i c_i / N_i
//   on A:  fbar += w pbar phi_i,  gbar -= w pbar phi_i,
//          wbar += (f - g_{i-1}) pbar phi_i + Nbar phi_i^2
// with g_{i-1} = g_i - c_i phi_i un-built from the final model; then
// rhobar = sum_A wbar w dist / rho (Eq. 15).  One block per CTA; each thread
// keeps its samples of L in registers; FP32, FP64 for the rho sums.
// ---------------------------------------------------------------------------
template <int T, int NT> struct DctBwd {
  static constexpr int KS = T * T / NT;  // samples of L per thread (Ls <= T)
  static constexpr int NW = NT / 32;
  static constexpr int CHI = 32;         // iterations per reduction batch
};

template <int T, int NT>
__global__ void __launch_bounds__(NT, 2) fofse_backward_dct_kernel(const __grid_constant__ BwdArgs a) {
  using G = DctBwd<T, NT>;
  constexpr int KS = G::KS, NW = G::NW, CHI = G::CHI;
  extern __shared__ unsigned char smem_raw[];
  float* cosT = reinterpret_cast<float*>(smem_raw);                // [4T]
  float* part = cosT + 4 * T;                                      // [NW][CHI] warp partials
  float* nrm = part + NW * CHI;                                    // [iters]
  float* cco = nrm + a.plan.iters;                                 // [iters] coefficients
  int* uu = reinterpret_cast<int*>(cco + a.plan.iters);            // [iters] packed u1 | u2 << 16
  double* dred = reinterpret_cast<double*>(uu + a.plan.iters + (a.plan.iters & 1));  // [3][NW]
  const PlanDev& P = a.plan;
  const int blk = blockIdx.x;
  const fofse_block bd = a.blocks[blk];
  if (bd.plan != a.plan_index) return;
  const float w0 = a.w0[blk];
  if (!(w0 > 0.f)) return;  // the block had no valid extrapolation
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int iters = P.iters, b = P.block, br = P.border, Ls = P.Ls;
  const float gamma = P.rho_gamma_dev ? P.rho_gamma_dev[1] : (float)P.gamma;
  const double rho = P.rho_gamma_dev ? (double)P.rho_gamma_dev[0] : (double)P.rho;
  for (int e = tid; e < 4 * T; e += NT) cosT[e] = P.tab.dct_cos_ff[e].x;
  for (int i = tid; i < iters; i += NT) {
    const fofse_trace_entry t = a.trace[(size_t)blk * a.trace_stride + i];
    cco[i] = t.dc_re;
    uu[i] = (t.u1 & (T - 1)) | ((t.u2 & (T - 1)) << 16);
  }
  // this thread's samples of L: weight, value, model, adjoints.  Thread t
  // holds column n = t mod Ls in rows t / Ls + k RB (RB = NT / Ls row groups;
  // RB KS >= T >= Ls, so every sample of L has a thread): the threads of a
  // warp share each row's cosine (a broadcast load) and each thread loads its
  // column's cosine once per iteration.
  float wv[KS], fv[KS], gv[KS], gb[KS], fb[KS], wb[KS];
  int mm[KS];
  const int RB = NT / Ls, cn = tid % Ls, rb = tid / Ls;
  const int pn = 2 * cn + 1;  // the column's phase step
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const int m = rb + k * RB, n = cn;
    const bool on = rb < RB && m < Ls;
    mm[k] = on ? m : 0;
    wv[k] = fv[k] = gv[k] = gb[k] = fb[k] = wb[k] = 0.f;
    if (!on) continue;
    const bool inB = m >= br && m < br + b && n >= br && n < br + b;
    bool inS = true;
    if (P.support == FOFSE_SUPPORT_CAUSAL_L) inS = (m < br) ? (n < br + b) : (m < br + b ? n < br : false);
    const int fy = bd.y - br + m, fx = bd.x - br + n;
    const bool in = fy >= 0 && fy < a.height && fx >= 0 && fx < a.width;
    if (in && !inB && inS && a.avail[(size_t)fy * a.pitch + fx]) {
      wv[k] = P.tab.w_f32[m * Ls + n];
      fv[k] = a.frame[(size_t)fy * a.pitch + fx];
    }
    if (inB) gb[k] = a.grad_blocks[(size_t)blk * a.grad_stride + (m - br) * a.grad_ld + (n - br)];
  }
  __syncthreads();
  // phi_u at sample k: the row's cosine times the column's (cc)
  auto colcos = [&](int u) -> float { return cosT[((u >> 16) * pn) & (4 * T - 1)]; };
  auto phi = [&](int u, int k, float cc) -> float {
    return cosT[((u & 0xffff) * (2 * mm[k] + 1)) & (4 * T - 1)] * cc;
  };
  // ---- weighted norms N_i, and the final model g_I = sum_i c_i phi_i ----
  for (int i0 = 0; i0 < iters; i0 += CHI) {
    const int ni = min(CHI, iters - i0);
    for (int j = 0; j < ni; ++j) {
      const int u = uu[i0 + j];
      const float c = cco[i0 + j], cc = colcos(u);
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const float ph = phi(u, k, cc);
        s = __fmaf_rn(wv[k] * ph, ph, s);
        gv[k] = __fmaf_rn(c, ph, gv[k]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFullMask, s, o);
      if (lane == 0) part[warp * CHI + j] = s;
    }
    __syncthreads();
    for (int j = tid; j < ni; j += NT) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) s += part[w * CHI + j];
      nrm[i0 + j] = s;
    }
    __syncthreads();
  }
  // ---- reverse pass ----
  float gam_acc = 0.f;
  for (int i = iters - 1; i >= 0; --i) {
    const int u = uu[i];
    const float c = cco[i], cc = colcos(u);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < KS; ++k) s = __fmaf_rn(gb[k], phi(u, k, cc), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFullMask, s, o);
    float* pw = part + (i & 1) * NW;  // double-buffered warp partials
    if (lane == 0) pw[warp] = s;
    __syncthreads();
    float cbar = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) cbar += pw[w];
    const float N = nrm[i];
    if (!(N > 0.f)) continue;
    gam_acc += cbar * c;
    const float pbar = gamma * cbar / N, nbar = -cbar * c / N;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const float ph = phi(u, k, cc);
      gv[k] = __fmaf_rn(-c, ph, gv[k]);  // g_{i-1}
      if (wv[k] != 0.f) {
        const float q = pbar * ph;
        fb[k] = __fmaf_rn(wv[k], q, fb[k]);
        gb[k] = __fmaf_rn(-wv[k], q, gb[k]);
        wb[k] = __fmaf_rn(fv[k] - gv[k], q, __fmaf_rn(nbar * ph, ph, wb[k]));
      }
    }
  }
  // ---- outputs: frame gradient, d/dgamma, d/drho ----
  double s_a = 0.0, s_b = 0.0, s_w = 0.0, s_wd = 0.0;
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    if (wv[k] == 0.f) continue;
    const int m = mm[k], n = cn;
    if (a.grad_frame) {
      const int fy = bd.y - br + m, fx = bd.x - br + n;
      atomicAdd(&a.grad_frame[(size_t)fy * a.pitch + fx], fb[k]);
    }
    const double d = P.tab.dist[m * Ls + n];
    const double ww = (double)wb[k] * (double)wv[k];
    s_a += ww * d;
    s_b += ww;
    s_w += (double)wv[k];
    s_wd += (double)wv[k] * d;
  }
  if (a.grad_rho_gamma) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s_a += __shfl_xor_sync(kFullMask, s_a, o);
      s_b += __shfl_xor_sync(kFullMask, s_b, o);
      s_w += __shfl_xor_sync(kFullMask, s_w, o);
      s_wd += __shfl_xor_sync(kFullMask, s_wd, o);
    }
    __syncthreads();
    if (lane == 0) {
      dred[warp] = s_a;
      dred[NW + warp] = s_b;
      dred[2 * NW + warp] = s_wd;
      part[warp] = (float)s_w;  // the weights' sum (for the mean distance)
    }
    __syncthreads();
    if (tid == 0) {
      double A = 0.0, Bs = 0.0, W = 0.0, WD = 0.0;
      for (int w = 0; w < NW; ++w) {
        A += dred[w];
        Bs += dred[NW + w];
        WD += dred[2 * NW + w];
        W += (double)part[w];
      }
      // sum_A wbar w = 0 up to rounding (B_hat does not change when w is scaled):
      // subtract it at the mean distance to keep the cancellation small
      const double dbar = W > 0.0 ? WD / W : 0.0;
      atomicAdd(&a.grad_rho_gamma[0], (float)((A - dbar * Bs) / rho));
      atomicAdd(&a.grad_rho_gamma[1], gam_acc / gamma);
    }
  }
}

template <int T, int NT> cudaError_t launch_bwd_dct(const BwdArgs& a, cudaStream_t s) {
  const int iters = a.plan.iters;
  const size_t sm = sizeof(float) * (4 * T + DctBwd<T, NT>::NW * DctBwd<T, NT>::CHI) +
                    (sizeof(float) * 2 + sizeof(int)) * (size_t)iters + 16 +
                    sizeof(double) * 3 * DctBwd<T, NT>::NW;
  int grid = 0;
  const cudaError_t e = prepare_kernel(fofse_backward_dct_kernel<T, NT>, NT, sm, &grid);
  if (e != cudaSuccess) return e;
  if (a.n_blocks < 1) return cudaSuccess;
  fofse_backward_dct_kernel<T, NT><<<a.n_blocks, NT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward_dct(const BwdArgs& a, cudaStream_t s) {
  if (a.plan.T == 32) return launch_bwd_dct<32, 128>(a, s);
  // 256 threads at two blocks per SM (16 samples of L per thread) overlap two
  // blocks' reductions: 0.92 ms on the 1080p batch against 1.15 ms with 512
  // threads and one block per SM
  if (a.plan.T == 64) return launch_bwd_dct<64, 256>(a, s);
  return cudaErrorNotSupported;
}

// FOFSE_FP32: the FP32 working spectrum with exact decisions (variant 0) or
// every bin in float-float (variant 1); FOFSE_FP32_FULLFF: every bin in
// float-float.
cudaError_t launch_forward_dct(const FwdArgs& a, cudaStream_t s) {
  const bool ff = a.plan.variant == 1 || a.plan.precision == FOFSE_FP32_FULLFF;
  if (a.plan.T == 32) return ff ? VariantDct<32, 128, false>::launch(a, s) : VariantDct<32, 128, true>::launch(a, s);
  if (a.plan.T == 64) return ff ? VariantDct<64, 256, false>::launch(a, s) : VariantDct<64, 256, true>::launch(a, s);
  return cudaErrorNotSupported;
}

int forward_dct_variant_count(const PlanDev& p) { return (p.T == 32 || p.T == 64) ? 2 : 1; }

size_t dct_table_elems(int T) { return (size_t)(T + 1) * (T + 2); }

cudaError_t build_dct_table(const PlanDev& p, float2* out, cudaStream_t s) {
  if (p.T == 32) return build_dct_table_T<32>(p, out, s);
  if (p.T == 64) return build_dct_table_T<64>(p, out, s);
  return cudaErrorNotSupported;
}

}  // namespace fofse
