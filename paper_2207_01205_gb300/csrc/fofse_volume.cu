// FOFSE over video volumes (Sec. 1: the method carried over to
// three-dimensional sets; Sec. 2's transform-domain recursion on a 3-D grid).
//
// Per lost block the volume L holds Lt = 2 depth + 1 frames (B's frame at its
// centre) of Ls x Ls samples, Ls = block + 2 border.  With the 3-D DFT on a
// T x T x Tt grid (L at the origin):
//   W = DFT(w), R = DFT(w f), w = rho^d on A (d: distance to the centre of B
//   in B's frame, a frame counting as one sample; A = the usable samples of L
//   outside B in B's own frame);
//   iters times: u = argmax |R[k]| over one index per conjugate pair
//   (lin(k) = (k1 T + k2) Tt + k3 <= lin(-k), ties to the smallest lin);
//   c = gamma R[u] / W[0] (real for the self-conjugate u);
//   R[k] -= c W[k - u] + s(u) conj(c) W[k + u];
//   B_hat += (1 + s(u)) Re(c exp(+j 2 pi (u1 m / T + u2 n / T + u3 depth / Tt))).
//
// One CTA per block, everything in FP64 in shared memory: R and W (T^2 Tt
// complex each, at most 4096 bins = 64 KB each), a stage buffer for the
// separable DFTs that build them, and the twiddle tables.  Each iteration is
// one pass over the canonical half of the bins (a compact index list built
// once per CTA) that applies the update and evaluates the next selection's
// energies, then a block-wide argmax (two barriers per iteration).  The
// output samples of B accumulate in registers as the iterations run.  The
// kernel is bound by the FP64 pipe: the energy compares run on 64-bit integer
// keys, and the per-iteration products of c are formed once per CTA.
#include <math.h>

#include <cstring>
#include <new>
#include <vector>

#include "fofse_volume32.cuh"

struct fofse_volume_plan_s {
  int block, border, depth, T, Tt, Ls, Lt, iters;
  float rho, gamma;
  int precision;     // FOFSE_FP32 (the product) or FOFSE_FP64_VALIDATE
  int variant;       // launch shape of the FP32 kernel
  int device;        // the device current at creation, which owns the tables
  double* wtab;      // device: rho^d over the Lt x Ls x Ls volume (tau, m, n)
  float2* wff;       // device: the same as float pairs (hi, lo)
  float4* tw_ff;     // device: exp(-j 2 pi e / T), e < T/2, float pairs
  float4* twt_ff;    // device: exp(-j 2 pi p / Tt), p < Tt, float pairs
  float2* syn;       // device: (cos, sin)(2 pi p / (T Tt)), p < T Tt
  void* mem;         // the allocation holding wtab and the tables
};

namespace fofse {
namespace {

struct VolArgs {
  int block, border, depth, Ls, Lt, iters;
  double gamma;
  const double* wtab;
  const fofse_volume_block* blocks;
  const float* video;
  const uint8_t* avail;
  int frames, height, width, pitch;
  float* out;       // n x block x block
  int32_t* path;    // n x iters x 3, nullable
  double* coef;     // n x iters x 2, nullable
  double* w0;       // n, nullable
  int32_t* status;  // n, nullable
};

template <int T, int TT> struct VolGeom {
  static constexpr int K = T * T * TT;                  // bins
  static constexpr int NT = K >= 2048 ? 512 : 256;      // threads
  static constexpr int NW = NT / 32;
  static constexpr int BPT = K / NT;                    // bins per thread
  static constexpr int LOGT = ilog2(T);
  static constexpr int LOGTT = ilog2(TT);
  static constexpr int PPT = 2;                         // samples of B per thread
  static_assert(K % NT == 0 && BPT >= 1, "bins must tile the threads");
  static_assert((1 << LOGT) == T && (1 << LOGTT) == TT, "power-of-two grid");
};

// Dynamic shared memory: R, W, then the stage buffer (Lt T^2 complex, which
// also holds the 2 Lt Ls^2 input doubles at first).
__host__ __device__ inline size_t vol_smem_bytes(int T, int TT, int Lt) {
  return sizeof(double2) * ((size_t)2 * T * T * TT + (size_t)Lt * T * T);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Energies |R[k]|^2 >= 0 are compared through their bit patterns as signed
// 64-bit integers, which order non-negative doubles as their values do (and
// keep the compares off the FP64 pipe); -1 is below every energy.
__device__ __forceinline__ long long energy_key(double2 r) {
  return __double_as_longlong(fma(r.x, r.x, r.y * r.y));
}

// (key, lin) pairs: the larger energy wins, equal energies go to the smaller lin.
__device__ __forceinline__ void better(long long& e, int& l, long long oe, int ol) {
  if (oe > e || (oe == e && ol < l)) {
    e = oe;
    l = ol;
  }
}

__device__ __forceinline__ void warp_argmax(long long& e, int& l) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const long long oe = __shfl_xor_sync(0xffffffffu, e, o);
    const int ol = __shfl_xor_sync(0xffffffffu, l, o);
    better(e, l, oe, ol);
  }
}

// Stage 1 (along n): z[(tau Ls + m) T + k2] = sum_n x[(tau Ls + m) Ls + n] e^{-j 2 pi k2 n / T}.
template <int T, int NT>
__device__ void dft_rows(const double* x, double2* z, int Lt, int Ls, const double2* tw) {
  constexpr int LOGT = ilog2(T);
  const int nq = Lt * Ls * T;
  for (int q = threadIdx.x; q < nq; q += NT) {
    const int row = q >> LOGT, k2 = q & (T - 1);
    const double* xr = x + row * Ls;
    double re = 0.0, im = 0.0;
    for (int n = 0; n < Ls; ++n) {
      const double v = xr[n];
      const double2 t = tw[(k2 * n) & (T - 1)];
      re = fma(v, t.x, re);
      im = fma(v, t.y, im);
    }
    z[q] = make_double2(re, im);
  }
}

// Stage 2 (along m): z2[(tau T + k1) T + k2] = sum_m z1[(tau Ls + m) T + k2] e^{-j 2 pi k1 m / T}.
template <int T, int NT>
__device__ void dft_cols(const double2* z1, double2* z2, int Lt, int Ls, const double2* tw) {
  constexpr int LOGT = ilog2(T);
  const int nq = Lt * T * T;
  for (int q = threadIdx.x; q < nq; q += NT) {
    const int k2 = q & (T - 1), k1 = (q >> LOGT) & (T - 1), tau = q >> (2 * LOGT);
    const double2* zc = z1 + tau * Ls * T + k2;
    double re = 0.0, im = 0.0;
    for (int m = 0; m < Ls; ++m) {
      const double2 v = zc[m * T];
      const double2 t = tw[(k1 * m) & (T - 1)];
      re = fma(v.x, t.x, re);
      re = fma(-v.y, t.y, re);
      im = fma(v.x, t.y, im);
      im = fma(v.y, t.x, im);
    }
    z2[q] = make_double2(re, im);
  }
}

// Stage 3 (along tau), column c = k1 T + k2: out[k3 T^2 + c] =
// sum_tau in[tau T^2 + c] e^{-j 2 pi k3 tau / Tt}.  A thread reads its whole
// column before writing it, so `in` may equal `out`.
template <int T, int TT, int NT>
__device__ void dft_time(const double2* in, double2* out, int Lt, const double2* twt) {
  for (int c = threadIdx.x; c < T * T; c += NT) {
    double2 v[TT];
#pragma unroll
    for (int tau = 0; tau < TT; ++tau) v[tau] = tau < Lt ? in[tau * T * T + c] : make_double2(0.0, 0.0);
#pragma unroll
    for (int k3 = 0; k3 < TT; ++k3) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int tau = 0; tau < TT; ++tau) {
        const double2 t = twt[(k3 * tau) & (TT - 1)];
        re = fma(v[tau].x, t.x, re);
        re = fma(-v[tau].y, t.y, re);
        im = fma(v[tau].x, t.y, im);
        im = fma(v[tau].y, t.x, im);
      }
      out[k3 * T * T + c] = make_double2(re, im);
    }
  }
}

template <int T, int TT>
__global__ void __launch_bounds__(VolGeom<T, TT>::NT, 1)
    fofse_volume_kernel(const __grid_constant__ VolArgs a) {
  using G = VolGeom<T, TT>;
  constexpr int K = G::K, NT = G::NT, NW = G::NW, BPT = G::BPT, LOGT = G::LOGT,
                LOGTT = G::LOGTT, PPT = G::PPT;
  extern __shared__ __align__(16) unsigned char vol_smem[];
  double2* R = reinterpret_cast<double2*>(vol_smem);
  double2* W = R + K;
  double2* X = W + K;
  __shared__ double2 twT[T], twTT[TT], syn[T * TT];
  __shared__ double red_e[NW];
  __shared__ long long red_k[NW];
  __shared__ int red_l[NW];
  __shared__ double bc[5];  // cr, ci, s cr, (1 + s) cr, (1 + s) ci
  __shared__ int bc_u[3];
  // the canonical set H as a list of layout indices: only H's bins are
  // updated and searched (the others hold the conjugates of H's and are
  // never read); |H| = (K + number of self-conjugate k) / 2 <= K / 2 + 4
  constexpr int NCMAX = K / 2 + 4;
  constexpr int RC = (NCMAX + NT - 1) / NT;  // list entries per thread
  __shared__ int hidx[NCMAX];
  __shared__ int wcnt[NW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bi = blockIdx.x;
  const fofse_volume_block blk = a.blocks[bi];
  const int Ls = a.Ls, Lt = a.Lt, b = a.block, e = a.border, D = a.depth;
  const int NS = Lt * Ls * Ls;

  for (int p = tid; p < T; p += NT) {
    double s, c;
    sincospi(2.0 * p / T, &s, &c);
    twT[p] = make_double2(c, -s);
  }
  for (int p = tid; p < TT; p += NT) {
    double s, c;
    sincospi(2.0 * p / TT, &s, &c);
    twTT[p] = make_double2(c, -s);
  }
  for (int p = tid; p < T * TT; p += NT) {
    double s, c;
    sincospi(2.0 * p / (T * TT), &s, &c);
    syn[p] = make_double2(c, s);
  }

  // ---- H in increasing layout order: per-thread chunks of BPT bins, block scan ----
  {
    unsigned mask = 0;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      const int i = tid * BPT + j;
      const int k2 = i & (T - 1), k1 = (i >> LOGT) & (T - 1), k3 = i >> (2 * LOGT);
      const int lin = ((k1 << LOGT) + k2) * TT + k3;
      const int nlin = ((((-k1) & (T - 1)) << LOGT) + ((-k2) & (T - 1))) * TT + ((-k3) & (TT - 1));
      if (lin <= nlin) {
        mask |= 1u << j;
        ++cnt;
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wcnt[warp] = incl;
    __syncthreads();
    int off = incl - cnt;
    for (int w = 0; w < warp; ++w) off += wcnt[w];
#pragma unroll
    for (int j = 0; j < BPT; ++j)
      if ((mask >> j) & 1u) hidx[off++] = tid * BPT + j;
  }
  int nc = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) nc += wcnt[w];

  // ---- weighted volume (Eq. 3, Eq. 4, Eq. 15 over three coordinates) ----
  double* xw = reinterpret_cast<double*>(X);
  double* xr = xw + NS;
  double wsum = 0.0;
  int bad = 0;
  for (int s = tid; s < NS; s += NT) {
    const int tau = s / (Ls * Ls), r = s - tau * Ls * Ls, m = r / Ls, n = r - m * Ls;
    const int ft = blk.t - D + tau, fy = blk.y - e + m, fx = blk.x - e + n;
    const bool inB = tau == D && m >= e && m < e + b && n >= e && n < e + b;
    double w = 0.0, wf = 0.0;
    if (!inB && ft >= 0 && ft < a.frames && fy >= 0 && fy < a.height && fx >= 0 && fx < a.width) {
      const long long o = ((long long)ft * a.height + fy) * a.pitch + fx;
      if (a.avail[o]) {
        w = a.wtab[s];
        const float f = a.video[o];
        if (w != 0.0) {
          if (isfinite(f))
            wf = w * (double)f;
          else
            bad = 1;
        }
      }
    }
    xw[s] = w;
    xr[s] = wf;
    wsum += w;
  }
  wsum = warp_sum(wsum);
  if (lane == 0) red_e[warp] = wsum;
  const int any_bad = __syncthreads_or(bad);
  double W0 = 0.0;
#pragma unroll
  for (int i = 0; i < NW; ++i) W0 += red_e[i];
  const int st = !(W0 > 0.0) ? FOFSE_BLK_NO_SUPPORT : any_bad ? FOFSE_BLK_NONFINITE : FOFSE_BLK_OK;
  if (tid == 0) {
    if (a.w0) a.w0[bi] = W0;
    if (a.status) a.status[bi] = st;
  }
  if (st != FOFSE_BLK_OK) {
    for (int p = tid; p < b * b; p += NT) a.out[(size_t)bi * b * b + p] = 0.0f;
    for (int p = tid; p < a.iters; p += NT) {
      const size_t o = (size_t)bi * a.iters + p;
      if (a.path) a.path[3 * o] = a.path[3 * o + 1] = a.path[3 * o + 2] = 0;
      if (a.coef) a.coef[2 * o] = a.coef[2 * o + 1] = 0.0;
    }
    return;
  }

  // ---- W = DFT(w) into W, then R = DFT(w f) into R (Eq. 8 on the 3-D grid) ----
  dft_rows<T, NT>(xw, R, Lt, Ls, twT);
  __syncthreads();
  dft_cols<T, NT>(R, W, Lt, Ls, twT);
  __syncthreads();
  dft_time<T, TT, NT>(W, W, Lt, twTT);
  __syncthreads();
  dft_rows<T, NT>(xr, R, Lt, Ls, twT);
  __syncthreads();
  dft_cols<T, NT>(R, X, Lt, Ls, twT);
  __syncthreads();
  dft_time<T, TT, NT>(X, R, Lt, twTT);
  __syncthreads();

  // ---- this thread's entries of H: layout index and lin (-1: none) ----
  int hi[RC], hl[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) {
    const int j = tid + r * NT;
    hi[r] = -1;
    hl[r] = 0x7fffffff;
    if (j < nc) {
      const int i = hidx[j];
      const int k2 = i & (T - 1), k1 = (i >> LOGT) & (T - 1), k3 = i >> (2 * LOGT);
      hi[r] = i;
      hl[r] = ((k1 << LOGT) + k2) * TT + k3;
    }
  }
  long long bk = -1;
  int bl = 0x7fffffff;
#pragma unroll
  for (int r = 0; r < RC; ++r)
    if (hi[r] >= 0) better(bk, bl, energy_key(R[hi[r]]), hl[r]);

  double g[PPT];
  int gm[PPT], gn[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int p = tid + q * NT;
    g[q] = 0.0;
    gm[q] = e + (p < b * b ? p / b : 0);
    gn[q] = e + (p < b * b ? p % b : 0);
  }

  const double gamma = a.gamma;
  for (int it = 0; it < a.iters; ++it) {
    // ---- Eq. 9: block-wide argmax over the canonical set ----
    warp_argmax(bk, bl);
    if (lane == 0) {
      red_k[warp] = bk;
      red_l[warp] = bl;
    }
    __syncthreads();
    if (warp == 0) {
      long long k2_ = lane < NW ? red_k[lane] : -1;
      int l2 = lane < NW ? red_l[lane] : 0x7fffffff;
      warp_argmax(k2_, l2);
      // no entry at all would leave the sentinel: take k = 0 so that the
      // index below stays inside R
      if (l2 == 0x7fffffff) l2 = 0;
      if (lane == 0) {
        const int u3 = l2 & (TT - 1), u2 = (l2 >> LOGTT) & (T - 1), u1 = l2 >> (LOGTT + LOGT);
        const double2 ru = R[(u3 << (2 * LOGT)) | (u1 << LOGT) | u2];
        const int s = (((2 * u1) & (T - 1)) == 0 && ((2 * u2) & (T - 1)) == 0 &&
                       ((2 * u3) & (TT - 1)) == 0)
                          ? 0
                          : 1;
        // Eq. 5 (p_u = R[u] / W0) and Eq. 14 (c = gamma p_u)
        const double cr = gamma * ru.x / W0;
        const double ci = s ? gamma * ru.y / W0 : 0.0;
        const double mult = s ? 2.0 : 1.0;
        bc[0] = cr;
        bc[1] = ci;
        bc[2] = s ? cr : 0.0;  // ci is 0 when s is
        bc[3] = mult * cr;
        bc[4] = mult * ci;
        bc_u[0] = u1;
        bc_u[1] = u2;
        bc_u[2] = u3;
        const size_t o = (size_t)bi * a.iters + it;
        if (a.path) {
          a.path[3 * o] = u1;
          a.path[3 * o + 1] = u2;
          a.path[3 * o + 2] = u3;
        }
        if (a.coef) {
          a.coef[2 * o] = cr;
          a.coef[2 * o + 1] = ci;
        }
      }
    }
    __syncthreads();
    const double cr = bc[0], ci = bc[1], crs = bc[2], mcr = bc[3], mci = bc[4];
    const int u1 = bc_u[0], u2 = bc_u[1], u3 = bc_u[2];

    // ---- Eq. 1-2: B_hat += (1 + s) Re(c phi_u) at B (frame tau = depth) ----
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      if (tid + q * NT < b * b) {
        const int ph = ((((u1 * gm[q] + u2 * gn[q]) & (T - 1)) * TT) + ((u3 * D) & (TT - 1)) * T) &
                       (T * TT - 1);
        const double2 y = syn[ph];
        g[q] = fma(mcr, y.x, g[q]);
        g[q] = fma(-mci, y.y, g[q]);
      }
    }

    // ---- R[k] -= c W[k - u] + s conj(c) W[k + u] on H; energies of the next pick ----
    bk = -1;
    bl = 0x7fffffff;
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      const int i = hi[r];
      if (i < 0) continue;
      const int k2 = i & (T - 1), k1 = (i >> LOGT) & (T - 1), k3 = i >> (2 * LOGT);
      const int im_ = (((k3 - u3) & (TT - 1)) << (2 * LOGT)) | (((k1 - u1) & (T - 1)) << LOGT) |
                      ((k2 - u2) & (T - 1));
      const int ip_ = (((k3 + u3) & (TT - 1)) << (2 * LOGT)) | (((k1 + u1) & (T - 1)) << LOGT) |
                      ((k2 + u2) & (T - 1));
      const double2 wa = W[im_], wb = W[ip_];
      // c W[k-u] = (cr wa.x - ci wa.y) + j (cr wa.y + ci wa.x)
      // conj(c) W[k+u] = (cr wb.x + ci wb.y) + j (cr wb.y - ci wb.x)
      double2 rr = R[i];
      rr.x = fma(-cr, wa.x, rr.x);
      rr.x = fma(ci, wa.y, rr.x);
      rr.x = fma(-crs, wb.x, rr.x);
      rr.x = fma(-ci, wb.y, rr.x);
      rr.y = fma(-cr, wa.y, rr.y);
      rr.y = fma(-ci, wa.x, rr.y);
      rr.y = fma(-crs, wb.y, rr.y);
      rr.y = fma(ci, wb.x, rr.y);
      R[i] = rr;
      better(bk, bl, energy_key(rr), hl[r]);
    }
  }

#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int p = tid + q * NT;
    if (p < b * b) a.out[(size_t)bi * b * b + p] = (float)g[q];
  }
}

// rho^d over the volume, d the distance to the centre of B in frame tau =
// depth (FP64, and split into float pairs).
__global__ void fofse_volume_weights_kernel(double* wtab, float2* wff, int block, int border,
                                            int depth, double rho) {
  const int Ls = block + 2 * border, Lt = 2 * depth + 1;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Lt * Ls * Ls) return;
  const int tau = s / (Ls * Ls), r = s - tau * Ls * Ls, m = r / Ls, n = r - m * Ls;
  const double c = border + (block - 1) / 2.0;
  const double dt = tau - depth, dm = m - c, dn = n - c;
  const double w = pow(rho, sqrt(dt * dt + dm * dm + dn * dn));
  wtab[s] = w;
  const float hi = (float)w;
  wff[s] = make_float2(hi, (float)(w - (double)hi));
}

template <int T, int TT>
cudaError_t launch_volume_T(const VolArgs& a, int n_blocks, cudaStream_t stream) {
  using G = VolGeom<T, TT>;
  const size_t smem = vol_smem_bytes(T, TT, a.Lt);
  cudaError_t e = cudaFuncSetAttribute(fofse_volume_kernel<T, TT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fofse_volume_kernel<T, TT><<<n_blocks, G::NT, smem, stream>>>(a);
  return cudaGetLastError();
}

// Grids of the FP64 kernel: T in {16, 32}, Tt in {1, 2, 4, 8}, T^2 Tt <= 4096.
bool volume_grid_supported(int T, int Tt) {
  if (T == 16) return Tt == 1 || Tt == 2 || Tt == 4 || Tt == 8;
  if (T == 32) return Tt == 1 || Tt == 2 || Tt == 4;
  return false;
}

cudaError_t launch_volume(int T, int Tt, const VolArgs& a, int n_blocks, cudaStream_t s) {
  switch (T * 100 + Tt) {
    case 1601: return launch_volume_T<16, 1>(a, n_blocks, s);
    case 1602: return launch_volume_T<16, 2>(a, n_blocks, s);
    case 1604: return launch_volume_T<16, 4>(a, n_blocks, s);
    case 1608: return launch_volume_T<16, 8>(a, n_blocks, s);
    case 3201: return launch_volume_T<32, 1>(a, n_blocks, s);
    case 3202: return launch_volume_T<32, 2>(a, n_blocks, s);
    case 3204: return launch_volume_T<32, 4>(a, n_blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

// Grids of the FP32 kernel: T in {16, 32, 64}, Tt in {1, 2, 4, 8}, T^2 Tt <= 16384.
bool volume32_grid_supported(int T, int Tt) {
  if (T == 16 || T == 32) return Tt == 1 || Tt == 2 || Tt == 4 || Tt == 8;
  if (T == 64) return Tt == 1 || Tt == 2 || Tt == 4;
  return false;
}

// The valid launch shapes of a grid, in the order of their variant numbers.
template <int T, int TT, class F> cudaError_t volume32_shape(int variant, F&& f) {
  static_assert(V3Shape<T, TT, 0>::valid, "shape 0 exists on every grid");
  int v = 0;
  if (variant == v++) return f(VariantV3<T, TT, 0>());
  if constexpr (V3Shape<T, TT, 1>::valid)
    if (variant == v++) return f(VariantV3<T, TT, 1>());
  if constexpr (V3Shape<T, TT, 2>::valid)
    if (variant == v++) return f(VariantV3<T, TT, 2>());
  return cudaErrorInvalidValue;
}
template <int T, int TT> constexpr int volume32_shapes() {
  return 1 + (V3Shape<T, TT, 1>::valid ? 1 : 0) + (V3Shape<T, TT, 2>::valid ? 1 : 0);
}

template <class F> cudaError_t volume32_dispatch(int T, int Tt, int variant, F&& f) {
  switch (T * 100 + Tt) {
    case 1601: return volume32_shape<16, 1>(variant, f);
    case 1602: return volume32_shape<16, 2>(variant, f);
    case 1604: return volume32_shape<16, 4>(variant, f);
    case 1608: return volume32_shape<16, 8>(variant, f);
    case 3201: return volume32_shape<32, 1>(variant, f);
    case 3202: return volume32_shape<32, 2>(variant, f);
    case 3204: return volume32_shape<32, 4>(variant, f);
    case 3208: return volume32_shape<32, 8>(variant, f);
    case 6401: return volume32_shape<64, 1>(variant, f);
    case 6402: return volume32_shape<64, 2>(variant, f);
    case 6404: return volume32_shape<64, 4>(variant, f);
    default: return cudaErrorInvalidValue;
  }
}

int volume32_variant_count(int T, int Tt) {
  switch (T * 100 + Tt) {
    case 1601: return volume32_shapes<16, 1>();
    case 1602: return volume32_shapes<16, 2>();
    case 1604: return volume32_shapes<16, 4>();
    case 1608: return volume32_shapes<16, 8>();
    case 3201: return volume32_shapes<32, 1>();
    case 3202: return volume32_shapes<32, 2>();
    case 3204: return volume32_shapes<32, 4>();
    case 3208: return volume32_shapes<32, 8>();
    case 6401: return volume32_shapes<64, 1>();
    case 6402: return volume32_shapes<64, 2>();
    case 6404: return volume32_shapes<64, 4>();
    default: return 1;
  }
}

constexpr size_t kVolCounterBytes = 256;

int volume_threads(int T, int Tt) { return T * T * Tt >= 2048 ? 512 : 256; }


// ---------------------------------------------------------------------------
// Backward over video volumes: the adjoint of the recursion along the frozen
// selection path, in the transform domain (as for images).  With phi_i =
// exp(+j 2 pi (u1 m / T + u2 n / T + u3 tau / Tt)), mult_i = 1 + s(u_i),
// c_i = gamma p_i / W0, p_i = sum_A w r_{i-1} conj(phi_i) and W[k] = sum w
// conj(phi_k), the reverse sweep of the spatial recursion (gbar_{i-1} =
// gbar_i - w Re(pbar_i phi_i) on A, gbar_I = dl/dB_hat on B) only needs, per
// iteration, acc_i = sum gbar_i conj(phi_i), and acc_j for j < i changes by
//   -1/2 (pbar_i conj(W[u_i - u_j]) + conj(pbar_i) W[u_i + u_j]),
// a triangular solve on W's values at the path's sums and differences:
//   acc_j = sum_B e conj(phi_j) (the DFT of e = dl/dB_hat at u_j)
//   for i = I..1: cbar_i = mult_i acc_i (imaginary part 0 if s = 0),
//     gammabar += Re(conj(cbar_i) c_i) / gamma, W0bar -= Re(conj(cbar_i) c_i) / W0,
//     pbar_i = gamma cbar_i / W0, then acc_j for j < i as above.
// A sample pass then goes over the trace per sample of A with the residual
// rebuilt along it (r_0 = f, r_i = r_{i-1} - mult_i Re(c_i phi_i)):
//   q_i = Re(pbar_i phi_i),  fbar = w sum_i q_i,  wbar = sum_i r_{i-1} q_i + W0bar,
// and rhobar = sum_A wbar w d / rho (d the distance to the centre of B, summed
// in FP64 with the mean distance subtracted: sum_A wbar w vanishes, since
// B_hat does not change when w is scaled).  Kernel 1 (one CTA per block):
// W in FP32 by separable DFTs of w (rows, columns, then the frames), the
// solve; kernel 2 (CTAs over chunks of each block's samples): the sample
// pass.  FP32, FP64 for the rho sums.
// ---------------------------------------------------------------------------
struct VolBwdArgs {
  int block, border, depth, Ls, Lt, T, Tt, iters;
  float gamma, rho;
  const float2* wff;
  const float2* syn;
  const fofse_volume_block* blocks;
  const float* video;
  const uint8_t* avail;
  int frames, height, width, pitch;
  const int32_t* path;
  const double* coef;
  const double* w0;
  const int32_t* status;
  const float* grad_blocks;
  float* grad_video;
  float* grad_rho_gamma;
  float2* pbar;       // workspace: n x iters
  double* scal;       // workspace: n x 2 (W0bar, mean distance over A)
  size_t off_y, off_ws, off_it, off_tw;  // solve kernel: byte offsets of Y, w, the per-iteration
                                         // arrays and the twiddle table
  int chunks;         // sample kernel: CTAs per block
};

constexpr int kVolBwdThreads = 256;

struct VolBwdLayout {  // shared memory of the solve kernel
  size_t off_y, off_ws, off_it, off_tw, bytes;
};
VolBwdLayout vol_bwd_layout(int T, int Tt, int Ls, int Lt, int iters) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  VolBwdLayout L;
  const size_t wb = (size_t)8 * T * T * Tt;            // W [k3][k1][k2] float2
  const size_t yb = (size_t)8 * Lt * Ls * T;           // row transforms [tau][m][k2]
  const size_t wsb = (size_t)4 * Lt * Ls * Ls;         // w of the volume
  const size_t itb = (size_t)28 * iters;               // acc, pbar, c (float2), packed u
  L.off_y = wb;
  // w sits in W's frames beyond Lt (free until the DFT over the frames) when it fits
  const bool w_in_W = Lt < Tt && (size_t)8 * (Tt - Lt) * T * T >= wsb;
  L.off_ws = w_in_W ? (size_t)8 * Lt * T * T : al(wb + (yb > itb ? yb : itb));
  L.off_it = wb;  // the per-iteration arrays reuse Y's region after the DFTs
  L.off_tw = w_in_W ? al(wb + (yb > itb ? yb : itb)) : al(L.off_ws + wsb);  // (cos, -sin), T Tt
  L.bytes = L.off_tw + (size_t)8 * T * Tt;
  return L;
}

__device__ __forceinline__ double vb_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// w of a volume sample: the plan's weight where the sample is usable (in the
// video, available, not in B), else 0
__device__ __forceinline__ float vb_weight(const VolBwdArgs& a, const fofse_volume_block& bd, int tau,
                                           int m, int n) {
  const int b = a.block, br = a.border, D = a.depth, Ls = a.Ls;
  const bool inB = tau == D && m >= br && m < br + b && n >= br && n < br + b;
  const int ft = bd.t - D + tau, fy = bd.y - br + m, fx = bd.x - br + n;
  if (inB || ft < 0 || ft >= a.frames || fy < 0 || fy >= a.height || fx < 0 || fx >= a.width) return 0.f;
  if (!a.avail[((size_t)ft * a.height + fy) * a.pitch + fx]) return 0.f;
  const float2 w = a.wff[(tau * Ls + m) * Ls + n];
  return w.x + w.y;
}

__device__ __forceinline__ bool vb_block_ok(const VolBwdArgs& a, int blk) {
  if (a.status && a.status[blk] != FOFSE_BLK_OK) return false;
  const double W0 = a.w0[blk];
  return W0 > 0.0 && isfinite(W0);
}

__global__ void __launch_bounds__(kVolBwdThreads) fofse_volume_bwd_solve_kernel(const __grid_constant__ VolBwdArgs a) {
  constexpr int NT = kVolBwdThreads;
  extern __shared__ __align__(16) unsigned char vb_smem[];
  __shared__ double redd[NT / 32];
  const int blk = blockIdx.x;
  if (!vb_block_ok(a, blk)) return;
  const int T = a.T, Tt = a.Tt, Ls = a.Ls, Lt = a.Lt, M = T * Tt, iters = a.iters;
  const int b = a.block, br = a.border, D = a.depth;
  const int tid = threadIdx.x;
  const fofse_volume_block bd = a.blocks[blk];
  float2* Wb = reinterpret_cast<float2*>(vb_smem);                 // [k3][k1][k2]
  float2* Y = reinterpret_cast<float2*>(vb_smem + a.off_y);        // [tau][m][k2]
  float* ws = reinterpret_cast<float*>(vb_smem + a.off_ws);        // [tau][m][n]
  float2* tw = reinterpret_cast<float2*>(vb_smem + a.off_tw);      // e^{-j 2 pi p / M}
  const int LT = __ffs(T) - 1;  // T and Tt are powers of two
  for (int p = tid; p < M; p += NT) {
    const float2 v = a.syn[p];
    tw[p] = make_float2(v.x, -v.y);
  }
  auto twd = [&](int p) -> float2 { return tw[p & (M - 1)]; };
  // w of the volume, and the mean distance over A (for the rho sums of the
  // sample pass)
  double sd = 0.0, na = 0.0;
  const double cen = br + (b - 1) / 2.0;
  for (int x = tid; x < Lt * Ls * Ls; x += NT) {
    const int tau = x / (Ls * Ls), rm = x - tau * Ls * Ls, m = rm / Ls, n = rm - m * Ls;
    const float w = vb_weight(a, bd, tau, m, n);
    ws[x] = w;
    if (w != 0.f) {
      const double dt = tau - D, dmm = m - cen, dn = n - cen;
      sd += sqrt(dt * dt + dmm * dmm + dn * dn);
      na += 1.0;
    }
  }
  const double nA = vb_block_sum(na, redd), sdA = vb_block_sum(sd, redd);  // (barriers)
  // rows: Y[tau][m][k2] = sum_n w e^{-j 2 pi k2 n / T}
  for (int e = tid; e < Lt * Ls * T; e += NT) {
    const int k2 = e & (T - 1), tm = e >> LT;
    const float* wr = ws + (size_t)tm * Ls;
    float2 acc = make_float2(0.f, 0.f);
    for (int n = 0; n < Ls; ++n) {
      const float2 t = twd(((k2 * n) & (T - 1)) * Tt);
      acc.x += wr[n] * t.x;
      acc.y += wr[n] * t.y;
    }
    Y[e] = acc;
  }
  __syncthreads();
  // columns: Z[tau][k1][k2] = sum_m Y[tau][m][k2] e^{-j 2 pi k1 m / T}, into W's frames tau < Lt
  for (int e = tid; e < Lt * T * T; e += NT) {
    const int k2 = e & (T - 1), k1 = (e >> LT) & (T - 1), tau = e >> (2 * LT);
    const float2* yc = Y + (size_t)tau * Ls * T + k2;
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 0; m < Ls; ++m) {
      const float2 y = yc[(size_t)m * T], t = twd(((k1 * m) & (T - 1)) * Tt);
      acc.x += y.x * t.x - y.y * t.y;
      acc.y += y.x * t.y + y.y * t.x;
    }
    Wb[e] = acc;
  }
  __syncthreads();
  // frames: W[k3][k1][k2] = sum_tau Z[tau][k1][k2] e^{-j 2 pi k3 tau / Tt}, in place per column
  for (int c = tid; c < T * T; c += NT) {
    float2 z[8];
#pragma unroll
    for (int tau = 0; tau < 8; ++tau) z[tau] = tau < Lt ? Wb[(size_t)tau * T * T + c] : make_float2(0.f, 0.f);
    for (int k3 = 0; k3 < Tt; ++k3) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int tau = 0; tau < 8; ++tau) {
        if (tau >= Lt) break;
        const float2 t = twd(((k3 * tau) & (Tt - 1)) * T);
        acc.x += z[tau].x * t.x - z[tau].y * t.y;
        acc.y += z[tau].x * t.y + z[tau].y * t.x;
      }
      Wb[(size_t)k3 * T * T + c] = acc;
    }
  }
  __syncthreads();
  // per-iteration arrays (Y's region is free now)
  float2* acc = reinterpret_cast<float2*>(vb_smem + a.off_it);
  float2* pbs = acc + iters;
  float2* cs = pbs + iters;
  int* up = reinterpret_cast<int*>(cs + iters);
  const int32_t* path = a.path + (size_t)blk * iters * 3;
  const double* coef = a.coef + (size_t)blk * iters * 2;
  // acc_i = sum_B e conj(phi_i) (phases of frame `depth`)
  for (int i = tid; i < iters; i += NT) {
    const int u1 = path[3 * i], u2 = path[3 * i + 1], u3 = path[3 * i + 2];
    up[i] = u1 | (u2 << 8) | (u3 << 16);
    cs[i] = make_float2((float)coef[2 * i], (float)coef[2 * i + 1]);
    const int p3 = ((u3 * D) & (Tt - 1)) * T;
    const float* e = a.grad_blocks + (size_t)blk * b * b;
    float2 s = make_float2(0.f, 0.f);
    for (int bm = 0; bm < b; ++bm)
      for (int bn = 0; bn < b; ++bn) {
        const int m = br + bm, n = br + bn;
        const float2 t = twd(((u1 * m + u2 * n) & (T - 1)) * Tt + p3);  // conj(phi)
        const float ev = e[bm * b + bn];
        s.x += ev * t.x;
        s.y += ev * t.y;
      }
    acc[i] = s;
  }
  __syncthreads();
  const float W0 = (float)a.w0[blk], gamma = a.gamma;
  const float iW0 = 1.f / W0, ig = 1.f / gamma, gW0 = gamma / W0;
  float gam = 0.f, w0bar = 0.f;
  for (int i = iters - 1; i >= 0; --i) {
    const int ui = up[i], u1 = ui & 255, u2 = (ui >> 8) & 255, u3 = ui >> 16;
    const bool sc = (u1 & (T / 2 - 1)) == 0 && (u2 & (T / 2 - 1)) == 0 && (Tt == 1 || (u3 & (Tt / 2 - 1)) == 0);
    const float mu = sc ? 1.f : 2.f;
    const float2 ai = acc[i], ci = cs[i];
    const float cbr = mu * ai.x, cbi = sc ? 0.f : mu * ai.y;
    const float cc = cbr * ci.x + cbi * ci.y;  // Re(conj(cbar) c)
    gam += cc * ig;
    w0bar -= cc * iW0;
    const float pr = gW0 * cbr, pi = gW0 * cbi;
    if (tid == 0) pbs[i] = make_float2(pr, pi);
    for (int j = tid; j < i; j += NT) {
      const int uj = up[j], v1 = uj & 255, v2 = (uj >> 8) & 255, v3 = uj >> 16;
      const int dm = ((((u3 - v3) & (Tt - 1)) * T + ((u1 - v1) & (T - 1))) * T) + ((u2 - v2) & (T - 1));
      const int dp = ((((u3 + v3) & (Tt - 1)) * T + ((u1 + v1) & (T - 1))) * T) + ((u2 + v2) & (T - 1));
      const float2 wm = Wb[dm], wp = Wb[dp];
      // pbar conj(wm) + conj(pbar) wp
      const float tr = pr * wm.x + pi * wm.y + pr * wp.x + pi * wp.y;
      const float ti = pi * wm.x - pr * wm.y + pr * wp.y - pi * wp.x;
      float2 v = acc[j];
      v.x -= 0.5f * tr;
      v.y -= 0.5f * ti;
      acc[j] = v;
    }
    __syncthreads();
  }
  for (int i = tid; i < iters; i += NT) a.pbar[(size_t)blk * iters + i] = pbs[i];
  if (tid == 0) {
    a.scal[2 * blk] = (double)w0bar;
    a.scal[2 * blk + 1] = nA > 0.0 ? sdA / nA : 0.0;
    if (a.grad_rho_gamma) atomicAdd(&a.grad_rho_gamma[1], gam);
  }
}

__global__ void __launch_bounds__(kVolBwdThreads) fofse_volume_bwd_samples_kernel(const __grid_constant__ VolBwdArgs a) {
  constexpr int NT = kVolBwdThreads;
  extern __shared__ __align__(16) unsigned char vb_smem[];
  __shared__ double redd[NT / 32];
  const int blk = blockIdx.x;  // blockIdx.y: the chunk of the block's samples
  if (!vb_block_ok(a, blk)) return;
  const int T = a.T, Tt = a.Tt, Ls = a.Ls, Lt = a.Lt, M = T * Tt, iters = a.iters;
  const int b = a.block, br = a.border, D = a.depth;
  const int tid = threadIdx.x;
  const fofse_volume_block bd = a.blocks[blk];
  // per iteration: (pbar, c) and the packed index with its weight
  float4* pc = reinterpret_cast<float4*>(vb_smem);
  int* up = reinterpret_cast<int*>(pc + iters);
  const int32_t* path = a.path + (size_t)blk * iters * 3;
  const double* coef = a.coef + (size_t)blk * iters * 2;
  for (int i = tid; i < iters; i += NT) {
    const float2 pb = a.pbar[(size_t)blk * iters + i];
    pc[i] = make_float4(pb.x, pb.y, (float)coef[2 * i], (float)coef[2 * i + 1]);
    const int u1 = path[3 * i], u2 = path[3 * i + 1], u3 = path[3 * i + 2];
    const bool sc = (u1 & (T / 2 - 1)) == 0 && (u2 & (T / 2 - 1)) == 0 && (Tt == 1 || (u3 & (Tt / 2 - 1)) == 0);
    up[i] = u1 | (u2 << 8) | (u3 << 16) | (sc ? 0 : 1 << 24);
  }
  __syncthreads();
  const int N = Lt * Ls * Ls;
  // two samples per thread share each iteration's decode
  int xs[2], ms[2], ns[2], ts[2];
  float wv[2], r[2], xb[2], wbar[2];
  size_t os[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = blockIdx.y * (2 * NT) + k * NT + tid;
    xs[k] = x;
    wv[k] = 0.f;
    ts[k] = ms[k] = ns[k] = 0;
    os[k] = 0;
    r[k] = xb[k] = wbar[k] = 0.f;
    if (x < N) {
      const int tau = x / (Ls * Ls), rm = x - tau * Ls * Ls, m = rm / Ls, n = rm - m * Ls;
      ts[k] = tau;
      ms[k] = m;
      ns[k] = n;
      wv[k] = vb_weight(a, bd, tau, m, n);
      if (wv[k] != 0.f) {
        os[k] = ((size_t)(bd.t - D + tau) * a.height + (bd.y - br + m)) * a.pitch + (bd.x - br + n);
        r[k] = a.video[os[k]];
      }
    }
  }
  if (wv[0] != 0.f || wv[1] != 0.f) {
    for (int i = 0; i < iters; ++i) {
      const int ui = up[i], u1 = ui & 255, u2 = (ui >> 8) & 255, u3 = (ui >> 16) & 255;
      const float mu = (ui >> 24) ? 2.f : 1.f;
      const float4 v = pc[i];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float2 t = __ldg(&a.syn[(((u1 * ms[k] + u2 * ns[k]) & (T - 1)) * Tt +
                                       ((u3 * ts[k]) & (Tt - 1)) * T) & (M - 1)]);
        const float q = v.x * t.x - v.y * t.y;
        xb[k] += q;
        wbar[k] += r[k] * q;
        r[k] -= mu * (v.z * t.x - v.w * t.y);
      }
    }
  }
  double s1 = 0.0;
  const double cen = br + (b - 1) / 2.0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (wv[k] == 0.f) continue;
    if (a.grad_video) atomicAdd(&a.grad_video[os[k]], wv[k] * xb[k]);
    const double dt = ts[k] - D, dm = ms[k] - cen, dn = ns[k] - cen;
    const double d = sqrt(dt * dt + dm * dm + dn * dn);
    s1 += ((double)wbar[k] + a.scal[2 * blk]) * (double)wv[k] * (d - a.scal[2 * blk + 1]);
  }
  (void)xs;
  if (!a.grad_rho_gamma) return;
  const double s = vb_block_sum(s1, redd);
  if (tid == 0 && s != 0.0) atomicAdd(&a.grad_rho_gamma[0], (float)(s / (double)a.rho));
}

}  // namespace
}  // namespace fofse

using namespace fofse;

extern "C" {

fofse_status fofse_volume_plan_create(int block, int border, int depth, int fft_size, int fft_time,
                                      float rho, float gamma, int iters, fofse_volume_plan* out) {
  if (!out || block < 1 || border < 0 || depth < 0 || fft_size < 1 || fft_time < 1) return FOFSE_E_ARG;
  if (!(rho > 0.0f && rho <= 1.0f) || !(gamma > 0.0f && gamma <= 1.0f)) return FOFSE_E_ARG;
  if (iters < 1 || iters > 4096) return FOFSE_E_ARG;
  const int Ls = block + 2 * border, Lt = 2 * depth + 1;
  if (Ls > fft_size || Lt > fft_time) return FOFSE_E_ARG;
  if (!volume32_grid_supported(fft_size, fft_time)) return FOFSE_E_UNSUPPORTED;
  fofse_volume_plan_s* p = new (std::nothrow) fofse_volume_plan_s();
  if (!p) return FOFSE_E_NOMEM;
  p->block = block;
  p->border = border;
  p->depth = depth;
  p->T = fft_size;
  p->Tt = fft_time;
  p->Ls = Ls;
  p->Lt = Lt;
  p->iters = iters;
  p->rho = rho;
  p->gamma = gamma;
  p->precision = FOFSE_FP32;
  p->variant = 0;
  const int T = fft_size, Tt = fft_time;
  const int ns = Lt * Ls * Ls;
  // host tables from integer phases in FP64, split into float pairs
  constexpr double kTwoPi = 6.283185307179586476925286766559;
  std::vector<float4> tw(T / 2), twt(Tt);
  std::vector<float2> syn((size_t)T * Tt);
  auto pair4 = [](double c, double s) {
    const float ch = (float)c, sh = (float)s;
    return make_float4(ch, sh, (float)(c - ch), (float)(s - sh));
  };
  for (int e = 0; e < T / 2; ++e) tw[e] = pair4(std::cos(kTwoPi * e / T), -std::sin(kTwoPi * e / T));
  for (int q = 0; q < Tt; ++q) twt[q] = pair4(std::cos(kTwoPi * q / Tt), -std::sin(kTwoPi * q / Tt));
  for (int q = 0; q < T * Tt; ++q)
    syn[q] = make_float2((float)std::cos(kTwoPi * q / (T * Tt)), (float)std::sin(kTwoPi * q / (T * Tt)));
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_w = 0, o_wff = al(sizeof(double) * ns), o_tw = o_wff + al(sizeof(float2) * ns),
               o_twt = o_tw + al(sizeof(float4) * (T / 2)), o_syn = o_twt + al(sizeof(float4) * Tt),
               total = o_syn + al(sizeof(float2) * T * Tt);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return record_cuda_error(e);
  }
  e = cudaMalloc(&p->mem, total);
  if (e != cudaSuccess) {
    delete p;
    return e == cudaErrorMemoryAllocation ? FOFSE_E_NOMEM : record_cuda_error(e);
  }
  unsigned char* base = static_cast<unsigned char*>(p->mem);
  p->wtab = reinterpret_cast<double*>(base + o_w);
  p->wff = reinterpret_cast<float2*>(base + o_wff);
  p->tw_ff = reinterpret_cast<float4*>(base + o_tw);
  p->twt_ff = reinterpret_cast<float4*>(base + o_twt);
  p->syn = reinterpret_cast<float2*>(base + o_syn);
  if ((e = cudaMemcpy(p->tw_ff, tw.data(), sizeof(float4) * (T / 2), cudaMemcpyHostToDevice)) == cudaSuccess &&
      (e = cudaMemcpy(p->twt_ff, twt.data(), sizeof(float4) * Tt, cudaMemcpyHostToDevice)) == cudaSuccess &&
      (e = cudaMemcpy(p->syn, syn.data(), sizeof(float2) * T * Tt, cudaMemcpyHostToDevice)) == cudaSuccess) {
    fofse_volume_weights_kernel<<<(ns + 255) / 256, 256>>>(p->wtab, p->wff, block, border, depth,
                                                            (double)rho);
    if ((e = cudaGetLastError()) == cudaSuccess) e = cudaStreamSynchronize(0);
  }
  if (e != cudaSuccess) {
    cudaFree(p->mem);
    delete p;
    return record_cuda_error(e);
  }
  *out = p;
  return FOFSE_OK;
}

fofse_status fofse_volume_plan_set_precision(fofse_volume_plan plan, int precision) {
  if (!plan || (precision != FOFSE_FP32 && precision != FOFSE_FP64_VALIDATE)) return FOFSE_E_ARG;
  if (precision == FOFSE_FP64_VALIDATE &&
      (!volume_grid_supported(plan->T, plan->Tt) ||
       plan->block * plan->block > 2 * volume_threads(plan->T, plan->Tt)))
    return FOFSE_E_UNSUPPORTED;
  plan->precision = precision;
  return FOFSE_OK;
}

size_t fofse_volume_workspace_bytes(fofse_volume_plan plan, int n_blocks) {
  if (!plan || n_blocks < 0) return 0;
  if (plan->precision != FOFSE_FP32) return 0;
  // the largest over the launch shapes, so that a workspace sized once serves
  // every variant
  size_t most = 0;
  for (int v = 0; v < volume32_variant_count(plan->T, plan->Tt); ++v) {
    size_t b = 0;
    const cudaError_t e = volume32_dispatch(plan->T, plan->Tt, v, [&](auto x) {
      return decltype(x)::scratch(plan->iters, &b);
    });
    if (e != cudaSuccess) return 0;
    most = b > most ? b : most;
  }
  return kVolCounterBytes + most;
}

int fofse_volume_plan_variant_count(fofse_volume_plan plan) {
  return plan ? volume32_variant_count(plan->T, plan->Tt) : 0;
}

fofse_status fofse_volume_plan_set_variant(fofse_volume_plan plan, int variant) {
  if (!plan || variant < 0 || variant >= volume32_variant_count(plan->T, plan->Tt)) return FOFSE_E_ARG;
  plan->variant = variant;
  return FOFSE_OK;
}

void fofse_volume_plan_destroy(fofse_volume_plan plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  cudaFree(plan->mem);
  delete plan;
}

fofse_status fofse_extrapolate_volume_batch(fofse_volume_plan plan,
                                            const fofse_volume_block* d_blocks, int n_blocks,
                                            const float* d_video, const uint8_t* d_avail,
                                            int frames, int height, int width, int pitch,
                                            float* d_out_blocks, int32_t* d_path, double* d_coef,
                                            double* d_w0, int32_t* d_block_status,
                                            void* d_workspace, void* stream) {
  if (!plan || n_blocks < 0 || frames < 1 || height < 1 || width < 1 || pitch < width)
    return FOFSE_E_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return FOFSE_E_ARG;
  if (plan->precision == FOFSE_FP32 && !d_workspace) return FOFSE_E_ARG;
  if (n_blocks == 0) return FOFSE_OK;
  if (!d_blocks || !d_video || !d_avail || !d_out_blocks) return FOFSE_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (plan->precision == FOFSE_FP32) {
    VolArgs32 a;
    std::memset(&a, 0, sizeof(a));
    a.block = plan->block;
    a.border = plan->border;
    a.depth = plan->depth;
    a.Ls = plan->Ls;
    a.Lt = plan->Lt;
    a.iters = plan->iters;
    a.gamma_h = plan->gamma;
    a.gamma_l = 0.f;
    a.w_ff = plan->wff;
    a.tab.tw_ff = plan->tw_ff;
    a.twt_ff = plan->twt_ff;
    a.syn = plan->syn;
    a.blocks = d_blocks;
    a.n_blocks = n_blocks;
    a.video = d_video;
    a.avail = d_avail;
    a.frames = frames;
    a.height = height;
    a.width = width;
    a.pitch = pitch;
    a.out = d_out_blocks;
    a.path = d_path;
    a.coef = d_coef;
    a.w0 = d_w0;
    a.status = d_block_status;
    unsigned char* ws = static_cast<unsigned char*>(d_workspace);
    a.queue = reinterpret_cast<int*>(ws);
    a.scratch = ws + kVolCounterBytes;
    a.scratch_bytes = fofse_volume_workspace_bytes(plan, n_blocks) - kVolCounterBytes;
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), s);
    if (e == cudaSuccess)
      e = volume32_dispatch(plan->T, plan->Tt, plan->variant,
                            [&](auto v) { return decltype(v)::launch(a, s); });
    return e == cudaSuccess ? FOFSE_OK : record_cuda_error(e);
  }
  VolArgs a;
  a.block = plan->block;
  a.border = plan->border;
  a.depth = plan->depth;
  a.Ls = plan->Ls;
  a.Lt = plan->Lt;
  a.iters = plan->iters;
  a.gamma = (double)plan->gamma;
  a.wtab = plan->wtab;
  a.blocks = d_blocks;
  a.video = d_video;
  a.avail = d_avail;
  a.frames = frames;
  a.height = height;
  a.width = width;
  a.pitch = pitch;
  a.out = d_out_blocks;
  a.path = d_path;
  a.coef = d_coef;
  a.w0 = d_w0;
  a.status = d_block_status;
  const cudaError_t e = launch_volume(plan->T, plan->Tt, a, n_blocks, s);
  return e == cudaSuccess ? FOFSE_OK : record_cuda_error(e);
}

size_t fofse_volume_backward_workspace_bytes(fofse_volume_plan plan, int n_blocks) {
  if (!plan || n_blocks < 0) return 0;
  return (((size_t)8 * plan->iters * n_blocks + 255) & ~size_t(255)) + (size_t)16 * n_blocks;
}

fofse_status fofse_volume_backward(fofse_volume_plan plan, const fofse_volume_block* d_blocks,
                                   int n_blocks, const float* d_video, const uint8_t* d_avail,
                                   int frames, int height, int width, int pitch,
                                   const int32_t* d_path, const double* d_coef, const double* d_w0,
                                   const int32_t* d_block_status, const float* d_grad_blocks,
                                   float* d_grad_video, float* d_grad_rho_gamma, void* d_workspace,
                                   void* stream) {
  if (!plan || n_blocks < 0 || frames < 1 || height < 1 || width < 1 || pitch < width)
    return FOFSE_E_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return FOFSE_E_ARG;
  const VolBwdLayout L = vol_bwd_layout(plan->T, plan->Tt, plan->Ls, plan->Lt, plan->iters);
  const size_t sm2 = (size_t)20 * plan->iters;
  if (L.bytes > 227 * 1024 || sm2 > 227 * 1024) return FOFSE_E_UNSUPPORTED;
  if (n_blocks == 0) return FOFSE_OK;
  if (!d_blocks || !d_video || !d_avail || !d_path || !d_coef || !d_w0 || !d_grad_blocks ||
      !d_workspace)
    return FOFSE_E_ARG;
  VolBwdArgs a;
  a.block = plan->block;
  a.border = plan->border;
  a.depth = plan->depth;
  a.Ls = plan->Ls;
  a.Lt = plan->Lt;
  a.T = plan->T;
  a.Tt = plan->Tt;
  a.iters = plan->iters;
  a.gamma = plan->gamma;
  a.rho = plan->rho;
  a.wff = plan->wff;
  a.syn = plan->syn;
  a.blocks = d_blocks;
  a.video = d_video;
  a.avail = d_avail;
  a.frames = frames;
  a.height = height;
  a.width = width;
  a.pitch = pitch;
  a.path = d_path;
  a.coef = d_coef;
  a.w0 = d_w0;
  a.status = d_block_status;
  a.grad_blocks = d_grad_blocks;
  a.grad_video = d_grad_video;
  a.grad_rho_gamma = d_grad_rho_gamma;
  unsigned char* ws = static_cast<unsigned char*>(d_workspace);
  a.pbar = reinterpret_cast<float2*>(ws);
  a.scal = reinterpret_cast<double*>(ws + (((size_t)8 * plan->iters * n_blocks + 255) & ~size_t(255)));
  a.off_y = L.off_y;
  a.off_ws = L.off_ws;
  a.off_it = L.off_it;
  a.off_tw = L.off_tw;
  const int N = plan->Lt * plan->Ls * plan->Ls;
  a.chunks = (N + 2 * kVolBwdThreads - 1) / (2 * kVolBwdThreads);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaFuncSetAttribute(fofse_volume_bwd_solve_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fofse_volume_bwd_samples_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e == cudaSuccess) {
    fofse_volume_bwd_solve_kernel<<<n_blocks, kVolBwdThreads, L.bytes, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    fofse_volume_bwd_samples_kernel<<<dim3(n_blocks, a.chunks), kVolBwdThreads, sm2, s>>>(a);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? FOFSE_OK : record_cuda_error(e);
}

}  // extern "C"
