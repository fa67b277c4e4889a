// In-place radix-2 decimation-in-time 2-D FFT of a T x T complex grid held in
// shared memory in the two-plane layout (element (r, c): part 0 at r*2T + c,
// part 1 at r*2T + T + c).  The input must sit at bit-reversed positions
// (element (m, n) of the signal at (brev(m), brev(n))); the output is in
// natural order.  Textbook iterative Cooley-Tukey: stage h pairs indices
// (i, i + h) with twiddle exp(-+ j 2 pi (i mod h) / (2h)).
//
//  rows_with_data  the row pass only transforms storage rows brev(r),
//                  r < rows_with_data (the other rows are zero);
//  cols_needed     the column pass only produces columns c < cols_needed;
//  tw              exp(-j 2 pi e / T), e < T/2 (conjugated for INVERSE, which
//                  gives the unnormalised inverse DFT).
#pragma once
#include "fofse_arith.cuh"

namespace fofse {

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

template <class A, int T, int NT, bool INVERSE>
__device__ __forceinline__ void fft2d_dit(typename A::E* Z, const typename A::C* tw,
                                          int rows_with_data, int cols_needed) {
  using C = typename A::C;
  constexpr int LOGT = ilog2c(T), T2 = 2 * T;
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int lh = 0; lh < LOGT; ++lh) {
    const int h = 1 << lh;
    for (int it = tid; it < rows_with_data * (T / 2); it += NT) {
      const int rr = it >> (LOGT - 1), q = it & (T / 2 - 1);
      const int row = __brev(rr) >> (32 - LOGT);
      const int i = ((q >> lh) << (lh + 1)) | (q & (h - 1));
      const int ex = (q & (h - 1)) << (LOGT - 1 - lh);
      const int ia = row * T2 + i, ib = ia + h;
      const C a = A::load(Z, ia, T), bb = A::load(Z, ib, T);
      const C w = INVERSE ? A::conj(tw[ex]) : tw[ex];
      const C wb = A::mul_norm(w, bb);
      A::store(Z, ia, T, A::add(a, wb));
      A::store(Z, ib, T, A::sub(a, wb));
    }
    __syncthreads();
  }
#pragma unroll 1
  for (int lh = 0; lh < LOGT; ++lh) {
    const int h = 1 << lh;
    for (int it = tid; it < cols_needed * (T / 2); it += NT) {
      const int c = it % cols_needed, q = it / cols_needed;
      const int i = ((q >> lh) << (lh + 1)) | (q & (h - 1));
      const int ex = (q & (h - 1)) << (LOGT - 1 - lh);
      const int ia = i * T2 + c, ib = ia + h * T2;
      const C a = A::load(Z, ia, T), bb = A::load(Z, ib, T);
      const C w = INVERSE ? A::conj(tw[ex]) : tw[ex];
      const C wb = A::mul_norm(w, bb);
      A::store(Z, ia, T, A::add(a, wb));
      A::store(Z, ib, T, A::sub(a, wb));
    }
    __syncthreads();
  }
}

}  // namespace fofse
