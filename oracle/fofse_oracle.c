/*
 * FP64 CPU oracle for fast orthogonality deficiency compensated frequency
 * selective extrapolation (FOFSE; Seiler & Kaup, arXiv 2207.01205).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * The oracle follows the algorithm in the paper's order, in the spatial
 * domain, re-projecting the weighted residual onto every 2-D DFT basis
 * function in every iteration (as the original OFSE does), which is slow and
 * obviously tied to the equations:
 *
 *   Sec. 2, Eq. 1-2   model g = sum c_k phi_k, built one basis pair per iteration
 *   Sec. 2, Eq. 3     residual r = f - g on the support area A, 0 on B
 *   Sec. 2, Eq. 4     weighting w = rho[m,n] on A, 0 on B
 *   Sec. 4, Eq. 15    isotropic rho[m,n] = rho_hat ^ distance to the B centre
 *   Sec. 2, Eq. 5     projection coefficient p_k = <r w, phi_k> / <w phi_k, phi_k>
 *   Sec. 2, Eq. 7-9   selection u = argmax_k |T{r w}[k]|
 *   Sec. 2, Eq. 14    constant compensation c_u = gamma * p_u
 *
 * Readings of points the paper leaves open:
 *  - basis phi_k[m,n] = exp(+j 2 pi (k1 m + k2 n) / T) over a T x T grid with
 *    the area L at its origin; the projection uses the conjugate basis, so
 *    p_k = P[k] / W0 with P = unnormalised forward DFT of r*w and W0 = sum w
 *    (|phi_k| = 1, so the Eq. 5 denominator is W0 for every k);
 *  - a real model needs conjugate pairs: one iteration adds c_u phi_u and
 *    conj(c_u) phi_{-u}, i.e. g += (1 + s(u)) Re(c_u phi_u), s(u) = 0 for the
 *    four self-conjugate indices (2u = 0 mod T), whose coefficient is real;
 *  - the argmax runs over the canonical set H = {k : k1 T + k2 <= (-k)1 T + (-k)2}
 *    (one index per conjugate pair); exact ties go to the smallest k1 T + k2;
 *  - the weighting centre is the centre of B; samples outside the frame,
 *    in other lost blocks, or outside the chosen support shape get w = 0.
 *
 * Frozen-path companions (the selection sequence fixed, so the output is
 * linear in f): a replay, a reverse-mode adjoint of the spatial recursion,
 * and a forward-mode tangent in rho and gamma.
 *
 * Beside the DFT basis with the constant compensation:
 *  - the transform-domain form of the same method (Sec. 2, closing remark),
 *    the like-for-like CPU program and a second check of the re-projection;
 *  - OFSE's compensation (Sec. 3, Eq. 10-13) with Q[u] = sum_l P[l] W[u - l]
 *    summed directly, and its factors gamma_u;
 *  - the 2-D DCT-II basis (Sec. 2 names it as the other transform-domain
 *    basis), with its replay and adjoint;
 *  - the squared error over B after every iteration count (Fig. 4, Fig. 5);
 *  - a threaded batch driver over a frame and its lost blocks;
 *  - video volumes (Sec. 1: the method carried over to three-dimensional
 *    sets), with the readings listed at the head of that section, and their
 *    frozen-path replay and adjoint.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NO_SUPPORT 1
#define ORC_NONFINITE 2

typedef struct {
    int block;     /* lost block side b                         */
    int border;    /* support border width                      */
    int fft_size;  /* T                                         */
    int iters;     /* I                                         */
    int support;   /* 0 = full frame around B, 1 = causal L     */
    double rho;    /* rho_hat of Eq. 15                         */
    double gamma;  /* constant compensation factor of Eq. 14    */
    int compensation; /* 0 = constant gamma (Eq. 14), 1 = OFSE's compensation (Eq. 10-12) */
    int basis;        /* 0 = 2-D DFT, 1 = 2-D DCT-II (Sec. 2, transform-domain remark) */
} oracle_plan;

static const double TWO_PI = 6.283185307179586476925286766559;

/* s(u) = 0 for self-conjugate u (2u = 0 mod T in both coordinates), else 1. */
static int pair_weight_s(int u1, int u2, int T) {
    return ((2 * u1) % T == 0 && (2 * u2) % T == 0) ? 0 : 1;
}

/* k is in the canonical set H when its row-major index does not exceed its mirror's. */
static int in_canonical_set(int k1, int k2, int T) {
    int mk1 = (T - k1) % T, mk2 = (T - k2) % T;
    return k1 * T + k2 <= mk1 * T + mk2;
}

static void twiddles(int T, double* c, double* s) {
    for (int p = 0; p < T; ++p) {
        c[p] = cos(TWO_PI * (double)p / (double)T);
        s[p] = sin(TWO_PI * (double)p / (double)T);
    }
}

/* -------------------------------------------------------------------------- */
/* Geometry and weighting (Eq. 4, Eq. 15)                                      */
/* -------------------------------------------------------------------------- */

/* Distance of every sample of L to the centre of B (the centre of L when B is
 * central).  L is Ls x Ls with B at rows/cols [border, border+block). */
void oracle_distance(int block, int border, double* dist) {
    int Ls = block + 2 * border;
    double c = border + (block - 1) / 2.0;
    for (int m = 0; m < Ls; ++m)
        for (int n = 0; n < Ls; ++n)
            dist[m * Ls + n] = sqrt((m - c) * (m - c) + (n - c) * (n - c));
}

/* Membership of (m, n) in the support shape (excluding B itself). */
static int in_support_shape(int block, int border, int support, int m, int n) {
    int inB = m >= border && m < border + block && n >= border && n < border + block;
    if (inB) return 0;
    if (support == 0) return 1;
    /* causal L: everything above B's rows up to B's right edge, and left of B in B's rows */
    if (m < border) return n < border + block;
    if (m < border + block) return n < border;
    return 0;
}

/* w[m,n] = rho_hat^dist on A, 0 elsewhere.  availL: 1 for usable samples of L. */
void oracle_weights(int block, int border, int support, double rho, const unsigned char* availL,
                    double* w) {
    int Ls = block + 2 * border;
    double* dist = (double*)malloc(sizeof(double) * Ls * Ls);
    oracle_distance(block, border, dist);
    for (int m = 0; m < Ls; ++m)
        for (int n = 0; n < Ls; ++n) {
            int i = m * Ls + n;
            int inA = availL[i] && in_support_shape(block, border, support, m, n);
            w[i] = inA ? pow(rho, dist[i]) : 0.0;
        }
    free(dist);
}

/* Cut the area L of a block out of the frame; samples outside the frame are
 * unavailable (and read as 0). */
void oracle_cut_area(const float* frame, const unsigned char* avail, int height, int width,
                     int pitch, int y, int x, int block, int border, double* fL,
                     unsigned char* aL) {
    int Ls = block + 2 * border;
    for (int m = 0; m < Ls; ++m)
        for (int n = 0; n < Ls; ++n) {
            int fy = y - border + m, fx = x - border + n;
            int in = fy >= 0 && fy < height && fx >= 0 && fx < width;
            fL[m * Ls + n] = in ? (double)frame[(size_t)fy * pitch + fx] : 0.0;
            aL[m * Ls + n] = in ? avail[(size_t)fy * pitch + fx] : 0;
        }
}

/* -------------------------------------------------------------------------- */
/* Transform operator T of Eq. 8: all T^2 weighted projections                 */
/* -------------------------------------------------------------------------- */

/* P[k1,k2] = sum_{m,n in L} rw[m,n] exp(-j 2 pi (k1 m + k2 n) / T), computed
 * separably (first along n, then along m) with twiddles from integer phases. */
void oracle_project(int Ls, int T, const double* rw, double* P_re, double* P_im) {
    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* Y_re = (double*)malloc(sizeof(double) * Ls * T);
    double* Y_im = (double*)malloc(sizeof(double) * Ls * T);
    twiddles(T, c, s);
    for (int m = 0; m < Ls; ++m)
        for (int k2 = 0; k2 < T; ++k2) {
            double re = 0.0, im = 0.0;
            for (int n = 0; n < Ls; ++n) {
                int p = (k2 * n) % T;
                re += rw[m * Ls + n] * c[p];
                im -= rw[m * Ls + n] * s[p];
            }
            Y_re[m * T + k2] = re;
            Y_im[m * T + k2] = im;
        }
    for (int k1 = 0; k1 < T; ++k1)
        for (int k2 = 0; k2 < T; ++k2) {
            double re = 0.0, im = 0.0;
            for (int m = 0; m < Ls; ++m) {
                int p = (k1 * m) % T;
                double yr = Y_re[m * T + k2], yi = Y_im[m * T + k2];
                /* (yr + j yi)(c - j s) */
                re += yr * c[p] + yi * s[p];
                im += yi * c[p] - yr * s[p];
            }
            P_re[k1 * T + k2] = re;
            P_im[k1 * T + k2] = im;
        }
    free(c); free(s); free(Y_re); free(Y_im);
}

/* Selection of Eq. 9 over the canonical set H; returns the relative gap
 * (best - runner-up) / best of |P|^2 over H through *gap. */
void oracle_select(int T, const double* P_re, const double* P_im, int* u1, int* u2, double* gap) {
    double best = -1.0, second = -1.0;
    int bi = 0;
    for (int k1 = 0; k1 < T; ++k1)
        for (int k2 = 0; k2 < T; ++k2) {
            if (!in_canonical_set(k1, k2, T)) continue;
            int i = k1 * T + k2;
            double v = P_re[i] * P_re[i] + P_im[i] * P_im[i];
            if (v > best) {
                second = best;
                best = v;
                bi = i;
            } else if (v > second) {
                second = v;
            }
        }
    *u1 = bi / T;
    *u2 = bi % T;
    if (gap) *gap = best > 0.0 ? (best - (second < 0.0 ? 0.0 : second)) / best : 0.0;
}

/* g += (1 + s(u)) Re(c phi_u) over L (Eq. 2 with the conjugate partner). */
static void add_basis_pair(int Ls, int T, const double* c, const double* s, int u1, int u2,
                           double c_re, double c_im, double* g) {
    double mult = 1.0 + pair_weight_s(u1, u2, T);
    for (int m = 0; m < Ls; ++m)
        for (int n = 0; n < Ls; ++n) {
            int p = (u1 * m + u2 * n) % T;
            g[m * Ls + n] += mult * (c_re * c[p] - c_im * s[p]);
        }
}

/* -------------------------------------------------------------------------- */
/* Extrapolation of one area (Sec. 2, Eq. 1-9, Eq. 14)                         */
/* -------------------------------------------------------------------------- */

/*
 * fL, wL: Ls x Ls samples and weights of L (w = 0 outside A).  Returns the
 * status; on ORC_OK fills g (final model over L), the selection path, the
 * coefficients c_u (dc) and the per-iteration relative gap.  Any of the path
 * outputs may be NULL.
 */
int oracle_extrapolate_area(int Ls, int T, const double* fL, const double* wL, double gamma,
                            int iters, double* g, int* path_u1, int* path_u2, double* dc_re,
                            double* dc_im, double* gap, double* w0_out) {
    int N = Ls * Ls;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    if (w0_out) *w0_out = W0;
    for (int i = 0; i < N; ++i) g[i] = 0.0;            /* g^(0) = 0 */
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    for (int i = 0; i < N; ++i)
        if (wL[i] != 0.0 && !isfinite(fL[i])) return ORC_NONFINITE;

    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* rw = (double*)malloc(sizeof(double) * N);
    double* P_re = (double*)malloc(sizeof(double) * T * T);
    double* P_im = (double*)malloc(sizeof(double) * T * T);
    twiddles(T, c, s);
    for (int it = 0; it < iters; ++it) {
        /* Eq. 3 and Eq. 7: weighted residual, zero outside A */
        for (int i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * (fL[i] - g[i]) : 0.0;
        /* Eq. 8: decomposition onto every basis function */
        oracle_project(Ls, T, rw, P_re, P_im);
        /* Eq. 9 */
        int u1, u2;
        double gp;
        oracle_select(T, P_re, P_im, &u1, &u2, &gp);
        /* Eq. 5 (p_u = P[u] / W0) and Eq. 14 (c_u = gamma p_u) */
        int ui = u1 * T + u2;
        double cr = gamma * P_re[ui] / W0;
        double ci = pair_weight_s(u1, u2, T) ? gamma * P_im[ui] / W0 : 0.0;
        /* Eq. 2 */
        add_basis_pair(Ls, T, c, s, u1, u2, cr, ci, g);
        if (path_u1) path_u1[it] = u1;
        if (path_u2) path_u2[it] = u2;
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
        if (gap) gap[it] = gp;
    }
    free(c); free(s); free(rw); free(P_re); free(P_im);
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* The 2-D DCT basis (Sec. 2: the DCT admits the transform-domain form too)     */
/* -------------------------------------------------------------------------- */

/*
 * FOFSE with the real basis of the 2-D DCT-II on the T x T grid, L at the
 * origin: phi_k[m,n] = cos(pi k1 (2m+1) / (2T)) cos(pi k2 (2n+1) / (2T)).
 * Every iteration (spatial re-projection, FP64):
 *   P[k] = sum w r phi_k                                (Eq. 8, unnormalised)
 *   u    = argmax_k (a_k1 a_k2 P[k])^2                   (Eq. 9; a_0 = sqrt(1/T),
 *          a_k = sqrt(2/T): the orthonormal DCT, so that the magnitude is the
 *          energy of the basis function's portion; ties: smallest k1 T + k2)
 *   c    = gamma P[u] / sum w phi_u^2                    (Eq. 5, Eq. 14)
 *   g   += c phi_u                                       (Eq. 2; real basis, no pairs)
 * path/dc/gap as for the DFT (dc real); the energies drop the common 1/T^2
 * (factors 1, 2 or 4).
 */
int oracle_extrapolate_area_dct(int Ls, int T, const double* fL, const double* wL, double gamma,
                                int iters, double* g, int* path_u1, int* path_u2, double* dc,
                                double* gap, double* w0_out) {
    int N = Ls * Ls;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    if (w0_out) *w0_out = W0;
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    for (int i = 0; i < N; ++i)
        if (wL[i] != 0.0 && !isfinite(fL[i])) return ORC_NONFINITE;

    /* cs[a * Ls + m] = cos(pi a (2m+1) / (2T)) from the integer phase a(2m+1) mod 4T */
    double* cs = (double*)malloc(sizeof(double) * T * Ls);
    for (int a = 0; a < T; ++a)
        for (int m = 0; m < Ls; ++m) {
            int p = (a * (2 * m + 1)) % (4 * T);
            cs[a * Ls + m] = cos(TWO_PI * (double)p / (double)(4 * T));
        }
    double* rw = (double*)malloc(sizeof(double) * N);
    double* Y = (double*)malloc(sizeof(double) * Ls * T);
    double* P = (double*)malloc(sizeof(double) * T * T);
    for (int it = 0; it < iters; ++it) {
        for (int i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * (fL[i] - g[i]) : 0.0;
        for (int m = 0; m < Ls; ++m)
            for (int k2 = 0; k2 < T; ++k2) {
                double acc = 0.0;
                for (int n = 0; n < Ls; ++n) acc += rw[m * Ls + n] * cs[k2 * Ls + n];
                Y[m * T + k2] = acc;
            }
        for (int k1 = 0; k1 < T; ++k1)
            for (int k2 = 0; k2 < T; ++k2) {
                double acc = 0.0;
                for (int m = 0; m < Ls; ++m) acc += cs[k1 * Ls + m] * Y[m * T + k2];
                P[k1 * T + k2] = acc;
            }
        double best = -1.0, second = -1.0;
        int bi = 0;
        for (int k1 = 0; k1 < T; ++k1)
            for (int k2 = 0; k2 < T; ++k2) {
                int i = k1 * T + k2;
                double e = P[i] * P[i] * (k1 ? 2.0 : 1.0) * (k2 ? 2.0 : 1.0);
                if (e > best) {
                    second = best;
                    best = e;
                    bi = i;
                } else if (e > second) {
                    second = e;
                }
            }
        int u1 = bi / T, u2 = bi % T;
        double nrm = 0.0;
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                double ph = cs[u1 * Ls + m] * cs[u2 * Ls + n];
                nrm += wL[m * Ls + n] * ph * ph;
            }
        double c = nrm > 0.0 ? gamma * P[bi] / nrm : 0.0;
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) g[m * Ls + n] += c * cs[u1 * Ls + m] * cs[u2 * Ls + n];
        if (path_u1) path_u1[it] = u1;
        if (path_u2) path_u2[it] = u2;
        if (dc) dc[it] = c;
        if (gap) gap[it] = best > 0.0 ? (best - (second < 0.0 ? 0.0 : second)) / best : 0.0;
    }
    free(cs); free(rw); free(Y); free(P);
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* Error over the iterations (the PSNR-over-iterations curves, Fig. 4, Fig. 5) */
/* -------------------------------------------------------------------------- */

/*
 * The model of Eq. 1 rebuilt iteration by iteration from a selection path and
 * its coefficients; after the nu-th iteration sse[nu - 1] = sum over B of
 * (clip(g, 0, 255) - truth)^2, truthB the block x block reference samples of
 * B (row-major), B at (border, border) inside L.
 */
void oracle_error_curve(int Ls, int T, int block, int border, const int* path_u1,
                        const int* path_u2, const double* dc_re, const double* dc_im, int iters,
                        const double* truthB, double* sse, int basis) {
    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* g = (double*)calloc((size_t)Ls * Ls, sizeof(double));
    twiddles(T, c, s);
    for (int it = 0; it < iters; ++it) {
        if (basis == 1) {  /* DCT-II: g += c cos(pi u1 (2m+1)/(2T)) cos(pi u2 (2n+1)/(2T)) */
            for (int m = 0; m < Ls; ++m)
                for (int n = 0; n < Ls; ++n) {
                    int p1 = (path_u1[it] * (2 * m + 1)) % (4 * T);
                    int p2 = (path_u2[it] * (2 * n + 1)) % (4 * T);
                    g[m * Ls + n] += dc_re[it] * cos(TWO_PI * (double)p1 / (4.0 * T)) *
                                     cos(TWO_PI * (double)p2 / (4.0 * T));
                }
        } else {
            add_basis_pair(Ls, T, c, s, path_u1[it], path_u2[it], dc_re[it], dc_im[it], g);
        }
        double e = 0.0;
        for (int bm = 0; bm < block; ++bm)
            for (int bn = 0; bn < block; ++bn) {
                double v = g[(border + bm) * Ls + border + bn];
                v = v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v);
                double d = v - truthB[bm * block + bn];
                e += d * d;
            }
        sse[it] = e;
    }
    free(c); free(s); free(g);
}

/* -------------------------------------------------------------------------- */
/* OFSE's orthogonality deficiency compensation (Sec. 3, Eq. 10-12)            */
/* -------------------------------------------------------------------------- */

/*
 * The spatial re-projection with the compensation FOFSE replaces: every
 * iteration all projections P[l] of the weighted residual are formed (Eq. 8)
 * and the coefficient of the selected u is
 *     c_u = p_u / sum_l (p_l / p_u) Khat[u, l]                          (Eq. 10)
 * with Khat = diag(K)^-1 K (Eq. 11) and K the matrix of weighted scalar
 * products of the basis functions (Eq. 12).  For the DFT basis K[u, l] =
 * sum w phi_l conj(phi_u) = W[u - l] with W = DFT(w), diag(K) = W0, so
 *     sum_l p_l Khat[u, l] = Q[u] / W0^2,  Q[u] = sum_l P[l] W[u - l],
 *     c_u = P[u]^2 / Q[u],   gamma_u = c_u / p_u = P[u] W0 / Q[u]      (Eq. 13)
 * (p_l = P[l] / W0).  Q[u] is summed directly over all T^2 bins l.  The
 * conjugate partner gets conj(c_u), as with the constant compensation; for
 * the four self-conjugate u both P[u] and Q[u] are real.  gamma_u (complex for
 * the complex basis) is returned per iteration for the distribution of Fig. 2.
 */
int oracle_extrapolate_area_ofse(int Ls, int T, const double* fL, const double* wL, int iters,
                                 double* g, int* path_u1, int* path_u2, double* dc_re,
                                 double* dc_im, double* gamma_re, double* gamma_im, double* gap,
                                 double* w0_out) {
    int N = Ls * Ls, TT = T * T;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    if (w0_out) *w0_out = W0;
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    for (int i = 0; i < N; ++i)
        if (wL[i] != 0.0 && !isfinite(fL[i])) return ORC_NONFINITE;

    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* rw = (double*)malloc(sizeof(double) * N);
    double* P_re = (double*)malloc(sizeof(double) * TT);
    double* P_im = (double*)malloc(sizeof(double) * TT);
    double* W_re = (double*)malloc(sizeof(double) * TT);
    double* W_im = (double*)malloc(sizeof(double) * TT);
    twiddles(T, c, s);
    oracle_project(Ls, T, wL, W_re, W_im);             /* K[u, l] = W[u - l] */
    for (int it = 0; it < iters; ++it) {
        for (int i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * (fL[i] - g[i]) : 0.0;
        oracle_project(Ls, T, rw, P_re, P_im);
        int u1, u2;
        double gp;
        oracle_select(T, P_re, P_im, &u1, &u2, &gp);
        /* Q[u] = sum_l P[l] W[u - l] */
        double q_re = 0.0, q_im = 0.0;
        for (int l1 = 0; l1 < T; ++l1)
            for (int l2 = 0; l2 < T; ++l2) {
                int a = ((u1 - l1 + T) % T) * T + (u2 - l2 + T) % T;
                double pr = P_re[l1 * T + l2], pi = P_im[l1 * T + l2];
                q_re += pr * W_re[a] - pi * W_im[a];
                q_im += pr * W_im[a] + pi * W_re[a];
            }
        int ui = u1 * T + u2, pair = pair_weight_s(u1, u2, T);
        double pr = P_re[ui], pi = pair ? P_im[ui] : 0.0;
        if (!pair) q_im = 0.0;
        /* c = P^2 / Q,  gamma = P W0 / Q */
        double den = q_re * q_re + q_im * q_im;
        double sq_re = pr * pr - pi * pi, sq_im = 2.0 * pr * pi;
        double cr = 0.0, ci = 0.0, gr = 0.0, gi = 0.0;
        if (den > 0.0) {
            cr = (sq_re * q_re + sq_im * q_im) / den;
            ci = (sq_im * q_re - sq_re * q_im) / den;
            gr = W0 * (pr * q_re + pi * q_im) / den;
            gi = W0 * (pi * q_re - pr * q_im) / den;
        }
        add_basis_pair(Ls, T, c, s, u1, u2, cr, ci, g);
        if (path_u1) path_u1[it] = u1;
        if (path_u2) path_u2[it] = u2;
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
        if (gamma_re) gamma_re[it] = gr;
        if (gamma_im) gamma_im[it] = gi;
        if (gap) gap[it] = gp;
    }
    free(c); free(s); free(rw); free(P_re); free(P_im); free(W_re); free(W_im);
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* The transform-domain form (Sec. 2, closing remark)                          */
/* -------------------------------------------------------------------------- */

/*
 * The same extrapolation in the paper's complete transform-domain
 * formulation: R_w = DFT(w f) and W = DFT(w) are formed once; each iteration
 * takes the argmax of Eq. 9 over the canonical set, c = gamma R_w[u] / W0
 * (Eq. 5, Eq. 14), and subtracts the spectrum of the added pair from every
 * bin: R_w[k] -= c W[k - u] + s(u) conj(c) W[k + u] (Eq. 2, Eq. 3, Eq. 7 in
 * the DFT domain).  O(I T^2) per block instead of O(I T^2 Ls).  It is the
 * CPU program the GPU path is timed against for a like-for-like ratio, and a
 * second, independently written check of the spatial re-projection above
 * (same interface and outputs as oracle_extrapolate_area).
 */
int oracle_extrapolate_area_fd(int Ls, int T, const double* fL, const double* wL, double gamma,
                               int iters, double* g, int* path_u1, int* path_u2, double* dc_re,
                               double* dc_im, double* gap, double* w0_out) {
    int N = Ls * Ls, TT = T * T;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    if (w0_out) *w0_out = W0;
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    for (int i = 0; i < N; ++i)
        if (wL[i] != 0.0 && !isfinite(fL[i])) return ORC_NONFINITE;

    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* rw = (double*)malloc(sizeof(double) * N);
    double* R_re = (double*)malloc(sizeof(double) * TT);
    double* R_im = (double*)malloc(sizeof(double) * TT);
    double* W_re = (double*)malloc(sizeof(double) * TT);
    double* W_im = (double*)malloc(sizeof(double) * TT);
    twiddles(T, c, s);
    for (int i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * fL[i] : 0.0;
    oracle_project(Ls, T, rw, R_re, R_im);            /* R_w = DFT(w f) */
    oracle_project(Ls, T, wL, W_re, W_im);            /* W = DFT(w)     */
    for (int it = 0; it < iters; ++it) {
        int u1, u2;
        double gp;
        oracle_select(T, R_re, R_im, &u1, &u2, &gp);
        int ui = u1 * T + u2, pair = pair_weight_s(u1, u2, T);
        double cr = gamma * R_re[ui] / W0;
        double ci = pair ? gamma * R_im[ui] / W0 : 0.0;
        for (int k1 = 0; k1 < T; ++k1)
            for (int k2 = 0; k2 < T; ++k2) {
                int a = ((k1 - u1 + T) % T) * T + (k2 - u2 + T) % T;  /* k - u */
                int b = ((k1 + u1) % T) * T + (k2 + u2) % T;          /* k + u */
                /* c W[k - u] + s conj(c) W[k + u] */
                double tr = cr * W_re[a] - ci * W_im[a];
                double ti = cr * W_im[a] + ci * W_re[a];
                if (pair) {
                    tr += cr * W_re[b] + ci * W_im[b];
                    ti += cr * W_im[b] - ci * W_re[b];
                }
                R_re[k1 * T + k2] -= tr;
                R_im[k1 * T + k2] -= ti;
            }
        add_basis_pair(Ls, T, c, s, u1, u2, cr, ci, g);   /* Eq. 2, for the output */
        if (path_u1) path_u1[it] = u1;
        if (path_u2) path_u2[it] = u2;
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
        if (gap) gap[it] = gp;
    }
    free(c); free(s); free(rw); free(R_re); free(R_im); free(W_re); free(W_im);
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* Frozen-path companions                                                      */
/* -------------------------------------------------------------------------- */

/* The coefficient of iteration i along a fixed path: c = gamma * P[u] / W0 with
 * P[u] the weighted projection of the current residual onto phi_u. */
static void project_one(int Ls, int T, const double* c, const double* s, const double* rw, int u1,
                        int u2, double* p_re, double* p_im) {
    double re = 0.0, im = 0.0;
    for (int m = 0; m < Ls; ++m)
        for (int n = 0; n < Ls; ++n) {
            int p = (u1 * m + u2 * n) % T;
            re += rw[m * Ls + n] * c[p];
            im -= rw[m * Ls + n] * s[p];
        }
    *p_re = re;
    *p_im = im;
}

/* Forward pass along a given path (no selection).  g_hist, if non-NULL,
 * receives g^(0..iters-1) (the model before each iteration), iters * Ls^2. */
int oracle_replay_area(int Ls, int T, const double* fL, const double* wL, double gamma, int iters,
                       const int* u1, const int* u2, double* g, double* dc_re, double* dc_im,
                       double* g_hist) {
    int N = Ls * Ls;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* rw = (double*)malloc(sizeof(double) * N);
    twiddles(T, c, s);
    for (int it = 0; it < iters; ++it) {
        if (g_hist) memcpy(g_hist + (size_t)it * N, g, sizeof(double) * N);
        for (int i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * (fL[i] - g[i]) : 0.0;
        double pr, pi;
        project_one(Ls, T, c, s, rw, u1[it], u2[it], &pr, &pi);
        double cr = gamma * pr / W0;
        double ci = pair_weight_s(u1[it], u2[it], T) ? gamma * pi / W0 : 0.0;
        add_basis_pair(Ls, T, c, s, u1[it], u2[it], cr, ci, g);
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
    }
    free(c); free(s); free(rw);
    return ORC_OK;
}

/*
 * Reverse-mode adjoint of the spatial recursion along a fixed path.
 *   gbar_out: adjoint of the final model g^(I) over L (Ls x Ls), e.g. dloss/dB on B, 0 elsewhere.
 * Outputs: fbar (Ls x Ls, nonzero only on A), wbar (Ls x Ls, on A), gammabar.
 * rho enters only through w; the caller chains wbar to rho (rhobar below).
 */
int oracle_adjoint_area(int Ls, int T, const double* fL, const double* wL, double gamma,
                        int iters, const int* u1, const int* u2, const double* gbar_out,
                        double* fbar, double* wbar, double* gammabar) {
    int N = Ls * Ls;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    for (int i = 0; i < N; ++i) fbar[i] = wbar[i] = 0.0;
    *gammabar = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* g = (double*)malloc(sizeof(double) * N);
    double* gh = (double*)malloc(sizeof(double) * (size_t)iters * N);
    double* dcr = (double*)malloc(sizeof(double) * iters);
    double* dci = (double*)malloc(sizeof(double) * iters);
    double* gbar = (double*)malloc(sizeof(double) * N);
    double* q = (double*)malloc(sizeof(double) * N);
    twiddles(T, c, s);
    oracle_replay_area(Ls, T, fL, wL, gamma, iters, u1, u2, g, dcr, dci, gh);
    memcpy(gbar, gbar_out, sizeof(double) * N);
    double W0bar = 0.0;
    for (int it = iters - 1; it >= 0; --it) {
        int a1 = u1[it], a2 = u2[it];
        int sp = pair_weight_s(a1, a2, T);
        double mult = 1.0 + sp;
        const double* gprev = gh + (size_t)it * N;
        /* g_it = g_prev + mult (c_re cos - c_im sin): adjoint of the coefficient */
        double cbar_re = 0.0, cbar_im = 0.0;
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                int p = (a1 * m + a2 * n) % T;
                cbar_re += mult * gbar[m * Ls + n] * c[p];
                cbar_im -= mult * gbar[m * Ls + n] * s[p];
            }
        if (!sp) cbar_im = 0.0;               /* the self-conjugate coefficient is real */
        /* c = gamma p / W0 */
        double p_re = dcr[it] * W0 / gamma, p_im = dci[it] * W0 / gamma;
        *gammabar += (cbar_re * p_re + cbar_im * p_im) / W0;
        W0bar -= (cbar_re * dcr[it] + cbar_im * dci[it]) / W0;
        double pbar_re = gamma / W0 * cbar_re, pbar_im = gamma / W0 * cbar_im;
        /* p_re = sum rw cos, p_im = -sum rw sin, rw = w (f - g_prev) on A */
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                int p = (a1 * m + a2 * n) % T;
                q[m * Ls + n] = pbar_re * c[p] - pbar_im * s[p];
            }
        for (int i = 0; i < N; ++i) {
            if (wL[i] == 0.0) continue;
            fbar[i] += wL[i] * q[i];
            gbar[i] -= wL[i] * q[i];
            wbar[i] += (fL[i] - gprev[i]) * q[i];
        }
    }
    for (int i = 0; i < N; ++i)
        if (wL[i] != 0.0) wbar[i] += W0bar;    /* W0 = sum of w over A */
    free(c); free(s); free(g); free(gh); free(dcr); free(dci); free(gbar); free(q);
    return ORC_OK;
}

/* phi_u over L for the DCT-II basis: cos(pi u1 (2m+1)/(2T)) cos(pi u2 (2n+1)/(2T)) */
static void dct_basis(int Ls, int T, int u1, int u2, double* phi) {
    for (int m = 0; m < Ls; ++m)
        for (int n = 0; n < Ls; ++n) {
            int p1 = (u1 * (2 * m + 1)) % (4 * T), p2 = (u2 * (2 * n + 1)) % (4 * T);
            phi[m * Ls + n] = cos(TWO_PI * (double)p1 / (4.0 * T)) * cos(TWO_PI * (double)p2 / (4.0 * T));
        }
}

/* DCT-II basis: forward along a fixed path (c = gamma sum w r phi / sum w phi^2,
 * Eq. 5, 14); g over L, coefficients, and (nullable) the model before each
 * iteration. */
int oracle_replay_area_dct(int Ls, int T, const double* fL, const double* wL, double gamma,
                           int iters, const int* u1, const int* u2, double* g, double* dc,
                           double* g_hist) {
    int N = Ls * Ls;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* phi = (double*)malloc(sizeof(double) * N);
    for (int it = 0; it < iters; ++it) {
        if (g_hist) memcpy(g_hist + (size_t)it * N, g, sizeof(double) * N);
        dct_basis(Ls, T, u1[it], u2[it], phi);
        double p = 0.0, nrm = 0.0;
        for (int i = 0; i < N; ++i) {
            if (wL[i] == 0.0) continue;
            p += wL[i] * (fL[i] - g[i]) * phi[i];
            nrm += wL[i] * phi[i] * phi[i];
        }
        double c = nrm > 0.0 ? gamma * p / nrm : 0.0;
        for (int i = 0; i < N; ++i) g[i] += c * phi[i];
        if (dc) dc[it] = c;
    }
    free(phi);
    return ORC_OK;
}

/*
 * DCT-II basis: reverse-mode adjoint along a fixed path (as oracle_adjoint_area).
 * Per iteration, reverse order: cbar = <gbar, phi>; gammabar += cbar c / gamma;
 * pbar = gamma cbar / N, Nbar = -cbar c / N with p = sum_A w (f - g_prev) phi and
 * N = sum_A w phi^2; then fbar += w pbar phi, gbar -= w pbar phi,
 * wbar += (f - g_prev) pbar phi + Nbar phi^2.
 */
int oracle_adjoint_area_dct(int Ls, int T, const double* fL, const double* wL, double gamma,
                            int iters, const int* u1, const int* u2, const double* gbar_out,
                            double* fbar, double* wbar, double* gammabar) {
    int N = Ls * Ls;
    double W0 = 0.0;
    for (int i = 0; i < N; ++i) W0 += wL[i];
    for (int i = 0; i < N; ++i) fbar[i] = wbar[i] = 0.0;
    *gammabar = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* g = (double*)malloc(sizeof(double) * N);
    double* gh = (double*)malloc(sizeof(double) * (size_t)iters * N);
    double* dc = (double*)malloc(sizeof(double) * iters);
    double* gbar = (double*)malloc(sizeof(double) * N);
    double* phi = (double*)malloc(sizeof(double) * N);
    oracle_replay_area_dct(Ls, T, fL, wL, gamma, iters, u1, u2, g, dc, gh);
    memcpy(gbar, gbar_out, sizeof(double) * N);
    for (int it = iters - 1; it >= 0; --it) {
        dct_basis(Ls, T, u1[it], u2[it], phi);
        const double* gprev = gh + (size_t)it * N;
        double cbar = 0.0, nrm = 0.0;
        for (int i = 0; i < N; ++i) {
            cbar += gbar[i] * phi[i];
            if (wL[i] != 0.0) nrm += wL[i] * phi[i] * phi[i];
        }
        if (!(nrm > 0.0)) continue;
        *gammabar += cbar * dc[it] / gamma;
        double pbar = gamma * cbar / nrm, nbar = -cbar * dc[it] / nrm;
        for (int i = 0; i < N; ++i) {
            if (wL[i] == 0.0) continue;
            double q = pbar * phi[i];
            fbar[i] += wL[i] * q;
            gbar[i] -= wL[i] * q;
            wbar[i] += (fL[i] - gprev[i]) * q + nbar * phi[i] * phi[i];
        }
    }
    free(g); free(gh); free(dc); free(gbar); free(phi);
    return ORC_OK;
}

/* rho_bar = sum_A wbar * d/d rho (rho^dist) = sum_A wbar * dist * rho^(dist - 1). */
double oracle_rho_chain(int N, const double* wL, const double* dist, double rho, const double* wbar) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i)
        if (wL[i] != 0.0) acc += wbar[i] * dist[i] * pow(rho, dist[i] - 1.0);
    return acc;
}

/*
 * Forward-mode tangent along a fixed path: derivative of the final model over
 * L with respect to a perturbation (w_dot, gamma_dot); w_dot = dist rho^(dist-1)
 * on A for d/d rho.
 */
int oracle_tangent_area(int Ls, int T, const double* fL, const double* wL, const double* wdot,
                        double gamma, double gamma_dot, int iters, const int* u1, const int* u2,
                        double* gdot) {
    int N = Ls * Ls;
    double W0 = 0.0, W0dot = 0.0;
    for (int i = 0; i < N; ++i) {
        W0 += wL[i];
        if (wL[i] != 0.0) W0dot += wdot[i];
    }
    for (int i = 0; i < N; ++i) gdot[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* c = (double*)malloc(sizeof(double) * T);
    double* s = (double*)malloc(sizeof(double) * T);
    double* g = (double*)calloc(N, sizeof(double));
    double* rw = (double*)malloc(sizeof(double) * N);
    double* rwdot = (double*)malloc(sizeof(double) * N);
    twiddles(T, c, s);
    for (int it = 0; it < iters; ++it) {
        for (int i = 0; i < N; ++i) {
            if (wL[i] == 0.0) {
                rw[i] = rwdot[i] = 0.0;
            } else {
                rw[i] = wL[i] * (fL[i] - g[i]);
                rwdot[i] = wdot[i] * (fL[i] - g[i]) - wL[i] * gdot[i];
            }
        }
        double pr, pi, pdr, pdi;
        project_one(Ls, T, c, s, rw, u1[it], u2[it], &pr, &pi);
        project_one(Ls, T, c, s, rwdot, u1[it], u2[it], &pdr, &pdi);
        int sp = pair_weight_s(u1[it], u2[it], T);
        double cr = gamma * pr / W0, ci = sp ? gamma * pi / W0 : 0.0;
        double cdr = gamma_dot * pr / W0 + gamma * pdr / W0 - gamma * pr * W0dot / (W0 * W0);
        double cdi = sp ? gamma_dot * pi / W0 + gamma * pdi / W0 - gamma * pi * W0dot / (W0 * W0) : 0.0;
        add_basis_pair(Ls, T, c, s, u1[it], u2[it], cr, ci, g);
        add_basis_pair(Ls, T, c, s, u1[it], u2[it], cdr, cdi, gdot);
    }
    free(c); free(s); free(g); free(rw); free(rwdot);
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* Whole batches of lost blocks (independent; threads over blocks)            */
/* -------------------------------------------------------------------------- */

typedef struct {
    const float* frame;
    const unsigned char* avail;
    int height, width, pitch;
    const int* blocks;          /* n x 3: y, x, plan */
    const oracle_plan* plans;
    int n_blocks;
    int out_stride;             /* floats per block in out_blocks */
    int trace_stride;           /* entries per block in the path arrays */
    double* out_blocks;         /* n x out_stride, B row-major b x b */
    int* status;                /* n */
    double* w0;                 /* n */
    int* path_u1;               /* n x trace_stride (nullable) */
    int* path_u2;
    double* dc_re;
    double* dc_im;
    double* gap;
    double* gamma_re;           /* OFSE compensation factors (nullable) */
    double* gamma_im;
    int transform_domain;       /* 0: spatial re-projection, 1: transform-domain form */
    int next;                   /* work counter */
    pthread_mutex_t lock;
} batch_job;

static void run_one(batch_job* J, int bi) {
    const int* bd = J->blocks + 3 * bi;
    const oracle_plan* P = J->plans + bd[2];
    int Ls = P->block + 2 * P->border, N = Ls * Ls;
    double* fL = (double*)malloc(sizeof(double) * N);
    double* wL = (double*)malloc(sizeof(double) * N);
    double* g = (double*)malloc(sizeof(double) * N);
    unsigned char* aL = (unsigned char*)malloc(N);
    oracle_cut_area(J->frame, J->avail, J->height, J->width, J->pitch, bd[0], bd[1], P->block,
                    P->border, fL, aL);
    oracle_weights(P->block, P->border, P->support, P->rho, aL, wL);
    size_t to = (size_t)bi * J->trace_stride;
    int st;
    if (P->basis == 1) {
        st = oracle_extrapolate_area_dct(Ls, P->fft_size, fL, wL, P->gamma, P->iters, g,
                                         J->path_u1 ? J->path_u1 + to : NULL,
                                         J->path_u2 ? J->path_u2 + to : NULL,
                                         J->dc_re ? J->dc_re + to : NULL,
                                         J->gap ? J->gap + to : NULL, J->w0 ? J->w0 + bi : NULL);
        if (J->dc_im)
            for (int i = 0; i < P->iters; ++i) J->dc_im[to + i] = 0.0;
    } else if (P->compensation == 1)
        st = oracle_extrapolate_area_ofse(
            Ls, P->fft_size, fL, wL, P->iters, g, J->path_u1 ? J->path_u1 + to : NULL,
            J->path_u2 ? J->path_u2 + to : NULL, J->dc_re ? J->dc_re + to : NULL,
            J->dc_im ? J->dc_im + to : NULL, J->gamma_re ? J->gamma_re + to : NULL,
            J->gamma_im ? J->gamma_im + to : NULL, J->gap ? J->gap + to : NULL,
            J->w0 ? J->w0 + bi : NULL);
    else
        st = (J->transform_domain ? oracle_extrapolate_area_fd : oracle_extrapolate_area)(
            Ls, P->fft_size, fL, wL, P->gamma, P->iters, g, J->path_u1 ? J->path_u1 + to : NULL,
            J->path_u2 ? J->path_u2 + to : NULL, J->dc_re ? J->dc_re + to : NULL,
            J->dc_im ? J->dc_im + to : NULL, J->gap ? J->gap + to : NULL, J->w0 ? J->w0 + bi : NULL);
    J->status[bi] = st;
    double* ob = J->out_blocks + (size_t)bi * J->out_stride;
    for (int m = 0; m < P->block; ++m)
        for (int n = 0; n < P->block; ++n)
            ob[m * P->block + n] = g[(m + P->border) * Ls + (n + P->border)];
    free(fL); free(wL); free(g); free(aL);
}

static void* batch_worker(void* arg) {
    batch_job* J = (batch_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int bi = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (bi >= J->n_blocks) break;
        run_one(J, bi);
    }
    return NULL;
}

/* Extrapolate every listed block of a frame; returns the number of threads used.
 * transform_domain selects oracle_extrapolate_area_fd instead of the spatial
 * re-projection. */
int oracle_batch_mode(const float* frame, const unsigned char* avail, int height, int width,
                      int pitch, const int* blocks, int n_blocks, const oracle_plan* plans,
                      int out_stride, int trace_stride, double* out_blocks, int* status, double* w0,
                      int* path_u1, int* path_u2, double* dc_re, double* dc_im, double* gap,
                      int n_threads, int transform_domain, double* gamma_re, double* gamma_im) {
    batch_job J;
    J.transform_domain = transform_domain;
    J.gamma_re = gamma_re;
    J.gamma_im = gamma_im;
    J.frame = frame; J.avail = avail; J.height = height; J.width = width; J.pitch = pitch;
    J.blocks = blocks; J.plans = plans; J.n_blocks = n_blocks; J.out_stride = out_stride;
    J.trace_stride = trace_stride; J.out_blocks = out_blocks; J.status = status; J.w0 = w0;
    J.path_u1 = path_u1; J.path_u2 = path_u2; J.dc_re = dc_re; J.dc_im = dc_im; J.gap = gap;
    J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_blocks) n_threads = n_blocks > 0 ? n_blocks : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, batch_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return n_threads;
}

int oracle_batch(const float* frame, const unsigned char* avail, int height, int width, int pitch,
                 const int* blocks, int n_blocks, const oracle_plan* plans, int out_stride,
                 int trace_stride, double* out_blocks, int* status, double* w0, int* path_u1,
                 int* path_u2, double* dc_re, double* dc_im, double* gap, int n_threads) {
    return oracle_batch_mode(frame, avail, height, width, pitch, blocks, n_blocks, plans,
                             out_stride, trace_stride, out_blocks, status, w0, path_u1, path_u2,
                             dc_re, dc_im, gap, n_threads, 0, NULL, NULL);
}

/* -------------------------------------------------------------------------- */
/* Adjoint of a whole batch along given paths                                  */
/* -------------------------------------------------------------------------- */

typedef struct {
    const float* frame;
    const unsigned char* avail;
    int height, width, pitch;
    const int* blocks;
    const oracle_plan* plans;
    int n_blocks;
    const int* path_u1;         /* n x trace_stride */
    const int* path_u2;
    int trace_stride;
    const double* e_blocks;     /* n x e_stride: dloss/dB, b x b row-major */
    int e_stride;
    int n_plans;
    double** grad_frame_t;      /* per thread: height x width accumulators */
    double** grad_rg_t;         /* per thread: n_plans x 2 */
    int next;
    pthread_mutex_t lock;
} adj_job;

typedef struct { adj_job* J; int t; } adj_arg;

static void adj_one(adj_job* J, int bi, double* gf, double* grg) {
    const int* bd = J->blocks + 3 * bi;
    const oracle_plan* P = J->plans + bd[2];
    int b = P->block, br = P->border, Ls = b + 2 * br, N = Ls * Ls;
    double* fL = (double*)malloc(sizeof(double) * N);
    double* wL = (double*)malloc(sizeof(double) * N);
    double* dist = (double*)malloc(sizeof(double) * N);
    double* gbar = (double*)calloc(N, sizeof(double));
    double* fbar = (double*)malloc(sizeof(double) * N);
    double* wbar = (double*)malloc(sizeof(double) * N);
    unsigned char* aL = (unsigned char*)malloc(N);
    oracle_cut_area(J->frame, J->avail, J->height, J->width, J->pitch, bd[0], bd[1], b, br, fL, aL);
    oracle_weights(b, br, P->support, P->rho, aL, wL);
    oracle_distance(b, br, dist);
    const double* e = J->e_blocks + (size_t)bi * J->e_stride;
    for (int m = 0; m < b; ++m)
        for (int n = 0; n < b; ++n) gbar[(m + br) * Ls + (n + br)] = e[m * b + n];
    double gam = 0.0;
    size_t to = (size_t)bi * J->trace_stride;
    int st = (P->basis == 1 ? oracle_adjoint_area_dct : oracle_adjoint_area)(
        Ls, P->fft_size, fL, wL, P->gamma, P->iters, J->path_u1 + to, J->path_u2 + to, gbar, fbar,
        wbar, &gam);
    if (st == ORC_OK) {
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                int i = m * Ls + n;
                if (wL[i] == 0.0) continue;
                int fy = bd[0] - br + m, fx = bd[1] - br + n;
                gf[(size_t)fy * J->width + fx] += fbar[i];
            }
        grg[2 * bd[2]] += oracle_rho_chain(N, wL, dist, P->rho, wbar);
        grg[2 * bd[2] + 1] += gam;
    }
    free(fL); free(wL); free(dist); free(gbar); free(fbar); free(wbar); free(aL);
}

static void* adj_worker(void* arg) {
    adj_arg* a = (adj_arg*)arg;
    adj_job* J = a->J;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int bi = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (bi >= J->n_blocks) break;
        adj_one(J, bi, J->grad_frame_t[a->t], J->grad_rg_t[a->t]);
    }
    return NULL;
}

/* Gradients of sum_blocks <e_block, B_hat_block> with every path frozen: adds
 * dloss/dframe into grad_frame (height x width, row-major, unit pitch) and
 * dloss/drho, dloss/dgamma into grad_rg (n_plans x 2).  Per-thread
 * accumulators are summed in thread order, so the result is deterministic for
 * a given thread count. */
int oracle_batch_adjoint(const float* frame, const unsigned char* avail, int height, int width,
                         int pitch, const int* blocks, int n_blocks, const oracle_plan* plans,
                         int n_plans, const int* path_u1, const int* path_u2, int trace_stride,
                         const double* e_blocks, int e_stride, double* grad_frame,
                         double* grad_rg, int n_threads) {
    adj_job J;
    J.frame = frame; J.avail = avail; J.height = height; J.width = width; J.pitch = pitch;
    J.blocks = blocks; J.plans = plans; J.n_blocks = n_blocks; J.path_u1 = path_u1;
    J.path_u2 = path_u2; J.trace_stride = trace_stride; J.e_blocks = e_blocks;
    J.e_stride = e_stride; J.n_plans = n_plans; J.next = 0;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_blocks) n_threads = n_blocks > 0 ? n_blocks : 1;
    size_t HW = (size_t)height * width;
    J.grad_frame_t = (double**)malloc(sizeof(double*) * n_threads);
    J.grad_rg_t = (double**)malloc(sizeof(double*) * n_threads);
    for (int t = 0; t < n_threads; ++t) {
        J.grad_frame_t[t] = (double*)calloc(HW, sizeof(double));
        J.grad_rg_t[t] = (double*)calloc(2 * n_plans, sizeof(double));
    }
    pthread_mutex_init(&J.lock, NULL);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
    adj_arg* args = (adj_arg*)malloc(sizeof(adj_arg) * n_threads);
    for (int t = 0; t < n_threads; ++t) {
        args[t].J = &J;
        args[t].t = t;
        pthread_create(&th[t], NULL, adj_worker, &args[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < n_threads; ++t) {
        for (size_t i = 0; i < HW; ++i) grad_frame[i] += J.grad_frame_t[t][i];
        for (int i = 0; i < 2 * n_plans; ++i) grad_rg[i] += J.grad_rg_t[t][i];
        free(J.grad_frame_t[t]);
        free(J.grad_rg_t[t]);
    }
    free(J.grad_frame_t); free(J.grad_rg_t); free(th); free(args);
    pthread_mutex_destroy(&J.lock);
    return n_threads;
}

/* -------------------------------------------------------------------------- */
/* Video volumes (Sec. 1: the method carried over to three-dimensional sets)   */
/* -------------------------------------------------------------------------- */

/*
 * The paper states the algorithm for images only and notes that it carries
 * over to three-dimensional signals; the readings taken here:
 *  - the area L is a volume of Lt = 2 depth + 1 frames (the frame of the lost
 *    block B at its centre, index tau = depth) x Ls x Ls samples, stored
 *    tau-major, tau then m then n;
 *  - A = the usable samples of L outside B in the centre frame; the samples
 *    of B's position in the other frames belong to A when they are usable;
 *  - w[tau,m,n] = rho_hat^d with d the Euclidean distance to the centre of B
 *    in the centre frame, one frame counting as one sample (Eq. 15 over three
 *    coordinates);
 *  - basis phi_k[tau,m,n] = exp(+j 2 pi (k1 m / T + k2 n / T + k3 tau / Tt))
 *    over a T x T x Tt grid with L at its origin (the 3-D DFT), so that
 *    p_k = P[k] / W0 as in two dimensions;
 *  - conjugate pairs and the canonical set as in two dimensions with the
 *    row-major index lin(k) = (k1 T + k2) Tt + k3: k is canonical when
 *    lin(k) <= lin(-k), exact ties of the selection go to the smallest lin(k),
 *    and s(u) = 0 for the self-conjugate indices (2u = 0 mod (T, T, Tt));
 *  - constant compensation c_u = gamma p_u (Eq. 14).
 * With depth 0 and Tt = 1 every step reduces to the two-dimensional oracle.
 */

typedef struct {
    int block;     /* lost block side b                               */
    int border;    /* spatial support border width                    */
    int depth;     /* frames on each side of B's frame (Lt = 2 depth + 1) */
    int fft_size;  /* T (both spatial axes)                           */
    int fft_time;  /* Tt (time axis), Tt >= Lt                        */
    int iters;     /* I                                               */
    double rho;    /* rho_hat of Eq. 15                               */
    double gamma;  /* constant compensation factor of Eq. 14          */
} oracle_vplan;

static int pair_weight_s3(int u1, int u2, int u3, int T, int Tt) {
    return ((2 * u1) % T == 0 && (2 * u2) % T == 0 && (2 * u3) % Tt == 0) ? 0 : 1;
}

static long lin3(int k1, int k2, int k3, int T, int Tt) {
    return ((long)k1 * T + k2) * Tt + k3;
}

static int in_canonical_set3(int k1, int k2, int k3, int T, int Tt) {
    return lin3(k1, k2, k3, T, Tt) <= lin3((T - k1) % T, (T - k2) % T, (Tt - k3) % Tt, T, Tt);
}

/* Distance of every sample of the volume to the centre of B in frame tau = depth. */
void oracle_distance3(int block, int border, int depth, double* dist) {
    int Ls = block + 2 * border, Lt = 2 * depth + 1;
    double c = border + (block - 1) / 2.0;
    for (int t = 0; t < Lt; ++t)
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                double dt = t - depth, dm = m - c, dn = n - c;
                dist[((size_t)t * Ls + m) * Ls + n] = sqrt(dt * dt + dm * dm + dn * dn);
            }
}

/* w = rho_hat^d on A (usable, and not B of the centre frame), 0 elsewhere. */
void oracle_weights3(int block, int border, int depth, double rho, const unsigned char* availL,
                     double* w) {
    int Ls = block + 2 * border, Lt = 2 * depth + 1;
    size_t N = (size_t)Lt * Ls * Ls;
    double* dist = (double*)malloc(sizeof(double) * N);
    oracle_distance3(block, border, depth, dist);
    for (int t = 0; t < Lt; ++t)
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                size_t i = ((size_t)t * Ls + m) * Ls + n;
                int inB = t == depth && m >= border && m < border + block && n >= border &&
                          n < border + block;
                w[i] = (availL[i] && !inB) ? pow(rho, dist[i]) : 0.0;
            }
    free(dist);
}

/* Cut the volume of a block (B's top-left corner (y, x) in frame t) out of a
 * video of `frames` frames, each height x width with `pitch` elements per row
 * and frames back to back; samples outside the video are unusable (0). */
void oracle_cut_volume(const float* video, const unsigned char* avail, int frames, int height,
                       int width, int pitch, int t, int y, int x, int block, int border, int depth,
                       double* fL, unsigned char* aL) {
    int Ls = block + 2 * border, Lt = 2 * depth + 1;
    for (int tau = 0; tau < Lt; ++tau)
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                int ft = t - depth + tau, fy = y - border + m, fx = x - border + n;
                int in = ft >= 0 && ft < frames && fy >= 0 && fy < height && fx >= 0 && fx < width;
                size_t i = ((size_t)tau * Ls + m) * Ls + n;
                size_t s = ((size_t)ft * height + fy) * pitch + fx;
                fL[i] = in ? (double)video[s] : 0.0;
                aL[i] = in ? avail[s] : 0;
            }
}

/* P[k] = sum over the volume of rw exp(-j 2 pi (k1 m / T + k2 n / T + k3 tau / Tt)),
 * P stored at lin(k): every frame's 2-D projection, then the sum over tau. */
void oracle_project3(int Lt, int Ls, int T, int Tt, const double* rw, double* P_re,
                     double* P_im) {
    size_t plane = (size_t)T * T;
    double* Y_re = (double*)malloc(sizeof(double) * Lt * plane);
    double* Y_im = (double*)malloc(sizeof(double) * Lt * plane);
    double* ct = (double*)malloc(sizeof(double) * Tt);
    double* st = (double*)malloc(sizeof(double) * Tt);
    twiddles(Tt, ct, st);
    for (int tau = 0; tau < Lt; ++tau)
        oracle_project(Ls, T, rw + (size_t)tau * Ls * Ls, Y_re + tau * plane, Y_im + tau * plane);
    for (int k1 = 0; k1 < T; ++k1)
        for (int k2 = 0; k2 < T; ++k2)
            for (int k3 = 0; k3 < Tt; ++k3) {
                double re = 0.0, im = 0.0;
                for (int tau = 0; tau < Lt; ++tau) {
                    int p = (k3 * tau) % Tt;
                    double yr = Y_re[tau * plane + k1 * T + k2], yi = Y_im[tau * plane + k1 * T + k2];
                    re += yr * ct[p] + yi * st[p];  /* (yr + j yi)(ct - j st) */
                    im += yi * ct[p] - yr * st[p];
                }
                P_re[lin3(k1, k2, k3, T, Tt)] = re;
                P_im[lin3(k1, k2, k3, T, Tt)] = im;
            }
    free(Y_re); free(Y_im); free(ct); free(st);
}

/* Eq. 9 over the canonical set of the 3-D grid; u[3]; gap as oracle_select. */
void oracle_select3(int T, int Tt, const double* P_re, const double* P_im, int* u, double* gap) {
    double top = -1.0, second = -1.0;
    long bi = 0;
    for (int k1 = 0; k1 < T; ++k1)
        for (int k2 = 0; k2 < T; ++k2)
            for (int k3 = 0; k3 < Tt; ++k3) {
                if (!in_canonical_set3(k1, k2, k3, T, Tt)) continue;
                long i = lin3(k1, k2, k3, T, Tt);
                double e = P_re[i] * P_re[i] + P_im[i] * P_im[i];
                if (e > top) {
                    second = top;
                    top = e;
                    bi = i;
                } else if (e > second) {
                    second = e;
                }
            }
    u[0] = (int)(bi / Tt / T);
    u[1] = (int)(bi / Tt % T);
    u[2] = (int)(bi % Tt);
    if (gap) *gap = top > 0.0 ? (top - (second < 0.0 ? 0.0 : second)) / top : 0.0;
}

/* g += (1 + s(u)) Re(c phi_u) over the volume, phases as integers mod T Tt. */
static void add_basis_pair3(int Lt, int Ls, int T, int Tt, const int* u, double c_re, double c_im,
                            double* g) {
    int M = T * Tt;
    double mult = 1.0 + pair_weight_s3(u[0], u[1], u[2], T, Tt);
    for (int tau = 0; tau < Lt; ++tau)
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                long p = (((long)u[0] * m + (long)u[1] * n) * Tt + (long)u[2] * tau * T) % M;
                double th = TWO_PI * (double)p / (double)M;
                g[((size_t)tau * Ls + m) * Ls + n] += mult * (c_re * cos(th) - c_im * sin(th));
            }
}

/*
 * FOFSE over one volume, spatial re-projection in every iteration: fL, wL
 * Lt x Ls x Ls; g the final model over the volume; path (iters x 3), dc,
 * gap, w0 as oracle_extrapolate_area (any may be NULL).
 */
int oracle_extrapolate_volume(int Lt, int Ls, int T, int Tt, const double* fL, const double* wL,
                              double gamma, int iters, double* g, int* path, double* dc_re,
                              double* dc_im, double* gap, double* w0_out) {
    size_t N = (size_t)Lt * Ls * Ls, K = (size_t)T * T * Tt;
    double W0 = 0.0;
    for (size_t i = 0; i < N; ++i) W0 += wL[i];
    if (w0_out) *w0_out = W0;
    for (size_t i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    for (size_t i = 0; i < N; ++i)
        if (wL[i] != 0.0 && !isfinite(fL[i])) return ORC_NONFINITE;
    double* rw = (double*)malloc(sizeof(double) * N);
    double* P_re = (double*)malloc(sizeof(double) * K);
    double* P_im = (double*)malloc(sizeof(double) * K);
    for (int it = 0; it < iters; ++it) {
        for (size_t i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * (fL[i] - g[i]) : 0.0;
        oracle_project3(Lt, Ls, T, Tt, rw, P_re, P_im);
        int u[3];
        double gp;
        oracle_select3(T, Tt, P_re, P_im, u, &gp);
        long ui = lin3(u[0], u[1], u[2], T, Tt);
        double cr = gamma * P_re[ui] / W0;
        double ci = pair_weight_s3(u[0], u[1], u[2], T, Tt) ? gamma * P_im[ui] / W0 : 0.0;
        add_basis_pair3(Lt, Ls, T, Tt, u, cr, ci, g);
        if (path) {
            path[3 * it] = u[0];
            path[3 * it + 1] = u[1];
            path[3 * it + 2] = u[2];
        }
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
        if (gap) gap[it] = gp;
    }
    free(rw); free(P_re); free(P_im);
    return ORC_OK;
}

/*
 * The same method on the volume in the paper's transform-domain form (the
 * closing remark of Sec. 2 on a 3-D grid): R = DFT(w f) and W = DFT(w) once
 * (oracle_project3), then per iteration the pick over the canonical set, c =
 * gamma R[u] / W0 and R[k] -= c W[k - u] + s(u) conj(c) W[k + u] over every
 * bin, FP64.  The like-for-like CPU program for the GPU/CPU ratio, and a
 * second, independently written check of the re-projection.  Arguments and
 * outputs as oracle_extrapolate_volume.
 */
int oracle_extrapolate_volume_fd(int Lt, int Ls, int T, int Tt, const double* fL,
                                 const double* wL, double gamma, int iters, double* g, int* path,
                                 double* dc_re, double* dc_im, double* gap, double* w0_out) {
    size_t N = (size_t)Lt * Ls * Ls, K = (size_t)T * T * Tt;
    double W0 = 0.0;
    for (size_t i = 0; i < N; ++i) W0 += wL[i];
    if (w0_out) *w0_out = W0;
    for (size_t i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    for (size_t i = 0; i < N; ++i)
        if (wL[i] != 0.0 && !isfinite(fL[i])) return ORC_NONFINITE;
    double* x = (double*)malloc(sizeof(double) * N);
    double* R_re = (double*)malloc(sizeof(double) * K);
    double* R_im = (double*)malloc(sizeof(double) * K);
    double* W_re = (double*)malloc(sizeof(double) * K);
    double* W_im = (double*)malloc(sizeof(double) * K);
    for (size_t i = 0; i < N; ++i) x[i] = wL[i] != 0.0 ? wL[i] * fL[i] : 0.0;
    oracle_project3(Lt, Ls, T, Tt, x, R_re, R_im);
    oracle_project3(Lt, Ls, T, Tt, wL, W_re, W_im);
    for (int it = 0; it < iters; ++it) {
        int u[3];
        double gp;
        oracle_select3(T, Tt, R_re, R_im, u, &gp);
        long ui = lin3(u[0], u[1], u[2], T, Tt);
        int sp = pair_weight_s3(u[0], u[1], u[2], T, Tt);
        double cr = gamma * R_re[ui] / W0;
        double ci = sp ? gamma * R_im[ui] / W0 : 0.0;
        for (int k1 = 0; k1 < T; ++k1)
            for (int k2 = 0; k2 < T; ++k2)
                for (int k3 = 0; k3 < Tt; ++k3) {
                    long k = lin3(k1, k2, k3, T, Tt);
                    long a = lin3((k1 - u[0] + T) % T, (k2 - u[1] + T) % T, (k3 - u[2] + Tt) % Tt, T, Tt);
                    long b = lin3((k1 + u[0]) % T, (k2 + u[1]) % T, (k3 + u[2]) % Tt, T, Tt);
                    /* c W[a] */
                    double tr = cr * W_re[a] - ci * W_im[a];
                    double ti = cr * W_im[a] + ci * W_re[a];
                    if (sp) {  /* + conj(c) W[b] */
                        tr += cr * W_re[b] + ci * W_im[b];
                        ti += cr * W_im[b] - ci * W_re[b];
                    }
                    R_re[k] -= tr;
                    R_im[k] -= ti;
                }
        add_basis_pair3(Lt, Ls, T, Tt, u, cr, ci, g);
        if (path) {
            path[3 * it] = u[0];
            path[3 * it + 1] = u[1];
            path[3 * it + 2] = u[2];
        }
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
        if (gap) gap[it] = gp;
    }
    free(x); free(R_re); free(R_im); free(W_re); free(W_im);
    return ORC_OK;
}

typedef struct {
    const float* video;
    const unsigned char* avail;
    int frames, height, width, pitch;
    const int* blocks;          /* n x 3: t, y, x */
    oracle_vplan plan;
    int n_blocks;
    double* out_blocks;         /* n x b x b */
    int* status;
    double* w0;
    int* path;                  /* n x iters x 3 (nullable) */
    double* dc_re;              /* n x iters (nullable) */
    double* dc_im;
    double* gap;
    int transform_domain;       /* 0: spatial re-projection, 1: transform-domain form */
    int next;
    pthread_mutex_t lock;
} vbatch_job;

static void run_one_volume(vbatch_job* J, int bi) {
    const oracle_vplan* P = &J->plan;
    const int* bd = J->blocks + 3 * bi;
    int Ls = P->block + 2 * P->border, Lt = 2 * P->depth + 1;
    size_t N = (size_t)Lt * Ls * Ls, I = (size_t)P->iters;
    double* fL = (double*)malloc(sizeof(double) * N);
    double* wL = (double*)malloc(sizeof(double) * N);
    double* g = (double*)malloc(sizeof(double) * N);
    unsigned char* aL = (unsigned char*)malloc(N);
    oracle_cut_volume(J->video, J->avail, J->frames, J->height, J->width, J->pitch, bd[0], bd[1],
                      bd[2], P->block, P->border, P->depth, fL, aL);
    oracle_weights3(P->block, P->border, P->depth, P->rho, aL, wL);
    J->status[bi] = (J->transform_domain ? oracle_extrapolate_volume_fd : oracle_extrapolate_volume)(
        Lt, Ls, P->fft_size, P->fft_time, fL, wL, P->gamma, P->iters, g,
        J->path ? J->path + 3 * I * bi : NULL, J->dc_re ? J->dc_re + I * bi : NULL,
        J->dc_im ? J->dc_im + I * bi : NULL, J->gap ? J->gap + I * bi : NULL,
        J->w0 ? J->w0 + bi : NULL);
    double* ob = J->out_blocks + (size_t)bi * P->block * P->block;
    for (int m = 0; m < P->block; ++m)
        for (int n = 0; n < P->block; ++n)
            ob[m * P->block + n] = g[((size_t)P->depth * Ls + m + P->border) * Ls + n + P->border];
    free(fL); free(wL); free(g); free(aL);
}

static void* vbatch_worker(void* arg) {
    vbatch_job* J = (vbatch_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int bi = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (bi >= J->n_blocks) break;
        run_one_volume(J, bi);
    }
    return NULL;
}

/* Extrapolate every listed block of a video with one volume plan; returns
 * the number of threads used.  transform_domain selects
 * oracle_extrapolate_volume_fd instead of the spatial re-projection. */
int oracle_batch_volume_mode(const float* video, const unsigned char* avail, int frames,
                             int height, int width, int pitch, const int* blocks, int n_blocks,
                             const oracle_vplan* plan, double* out_blocks, int* status, double* w0,
                             int* path, double* dc_re, double* dc_im, double* gap, int n_threads,
                             int transform_domain) {
    vbatch_job J;
    J.transform_domain = transform_domain;
    J.video = video; J.avail = avail; J.frames = frames; J.height = height; J.width = width;
    J.pitch = pitch; J.blocks = blocks; J.plan = *plan; J.n_blocks = n_blocks;
    J.out_blocks = out_blocks; J.status = status; J.w0 = w0; J.path = path; J.dc_re = dc_re;
    J.dc_im = dc_im; J.gap = gap; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_blocks) n_threads = n_blocks > 0 ? n_blocks : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, vbatch_worker, &J);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return n_threads;
}

/* -------------------------------------------------------------------------- */
/* Video volumes along a frozen path: replay and reverse-mode adjoint          */
/* -------------------------------------------------------------------------- */

/* Phase index of phi_u at (tau, m, n) over the common denominator T Tt. */
static long phase3(const int* u, int tau, int m, int n, int T, int Tt) {
    return ((((long)u[0] * m + (long)u[1] * n) * Tt) + (long)u[2] * tau * T) % ((long)T * Tt);
}

/* p_u = sum over the volume of rw exp(-j theta_u): the one projection the path needs. */
static void project_one3(int Lt, int Ls, int T, int Tt, const double* rw, const int* u,
                         double* pr, double* pi) {
    double M = (double)T * Tt, re = 0.0, im = 0.0;
    for (int tau = 0; tau < Lt; ++tau)
        for (int m = 0; m < Ls; ++m)
            for (int n = 0; n < Ls; ++n) {
                double th = TWO_PI * (double)phase3(u, tau, m, n, T, Tt) / M;
                double v = rw[((size_t)tau * Ls + m) * Ls + n];
                re += v * cos(th);
                im -= v * sin(th);
            }
    *pr = re;
    *pi = im;
}

/* The recursion of oracle_extrapolate_volume with the selection replaced by
 * the given path (iters x 3); g, coefficients, and optionally the model
 * before every iteration (g_hist, iters x Lt Ls Ls). */
int oracle_replay_volume(int Lt, int Ls, int T, int Tt, const double* fL, const double* wL,
                         double gamma, int iters, const int* path, double* g, double* dc_re,
                         double* dc_im, double* g_hist) {
    size_t N = (size_t)Lt * Ls * Ls;
    double W0 = 0.0;
    for (size_t i = 0; i < N; ++i) W0 += wL[i];
    for (size_t i = 0; i < N; ++i) g[i] = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* rw = (double*)malloc(sizeof(double) * N);
    for (int it = 0; it < iters; ++it) {
        const int* u = path + 3 * it;
        if (g_hist) memcpy(g_hist + (size_t)it * N, g, sizeof(double) * N);
        for (size_t i = 0; i < N; ++i) rw[i] = wL[i] != 0.0 ? wL[i] * (fL[i] - g[i]) : 0.0;
        double pr, pi;
        project_one3(Lt, Ls, T, Tt, rw, u, &pr, &pi);
        double cr = gamma * pr / W0;
        double ci = pair_weight_s3(u[0], u[1], u[2], T, Tt) ? gamma * pi / W0 : 0.0;
        add_basis_pair3(Lt, Ls, T, Tt, u, cr, ci, g);
        if (dc_re) dc_re[it] = cr;
        if (dc_im) dc_im[it] = ci;
    }
    free(rw);
    return ORC_OK;
}

/*
 * Reverse-mode adjoint of the volume recursion along a fixed path.
 *   gbar_out: adjoint of the final model over the volume (Lt x Ls x Ls),
 *   e.g. dloss/dB on B in the centre frame and 0 elsewhere.
 * Outputs fbar and wbar (nonzero only on A) and gammabar; rho enters only
 * through w (oracle_rho_chain with the volume's distances chains wbar to rho).
 */
int oracle_adjoint_volume(int Lt, int Ls, int T, int Tt, const double* fL, const double* wL,
                          double gamma, int iters, const int* path, const double* gbar_out,
                          double* fbar, double* wbar, double* gammabar) {
    size_t N = (size_t)Lt * Ls * Ls;
    double W0 = 0.0, M = (double)T * Tt;
    for (size_t i = 0; i < N; ++i) W0 += wL[i];
    for (size_t i = 0; i < N; ++i) fbar[i] = wbar[i] = 0.0;
    *gammabar = 0.0;
    if (!(W0 > 0.0)) return ORC_NO_SUPPORT;
    double* g = (double*)malloc(sizeof(double) * N);
    double* gh = (double*)malloc(sizeof(double) * (size_t)iters * N);
    double* dcr = (double*)malloc(sizeof(double) * iters);
    double* dci = (double*)malloc(sizeof(double) * iters);
    double* gbar = (double*)malloc(sizeof(double) * N);
    double* cs = (double*)malloc(sizeof(double) * N);
    double* sn = (double*)malloc(sizeof(double) * N);
    oracle_replay_volume(Lt, Ls, T, Tt, fL, wL, gamma, iters, path, g, dcr, dci, gh);
    memcpy(gbar, gbar_out, sizeof(double) * N);
    double W0bar = 0.0;
    for (int it = iters - 1; it >= 0; --it) {
        const int* u = path + 3 * it;
        int sp = pair_weight_s3(u[0], u[1], u[2], T, Tt);
        double mult = 1.0 + sp;
        const double* gprev = gh + (size_t)it * N;
        for (int tau = 0; tau < Lt; ++tau)
            for (int m = 0; m < Ls; ++m)
                for (int n = 0; n < Ls; ++n) {
                    size_t i = ((size_t)tau * Ls + m) * Ls + n;
                    double th = TWO_PI * (double)phase3(u, tau, m, n, T, Tt) / M;
                    cs[i] = cos(th);
                    sn[i] = sin(th);
                }
        /* g_it = g_prev + mult (c_re cos - c_im sin): adjoint of the coefficient */
        double cbar_re = 0.0, cbar_im = 0.0;
        for (size_t i = 0; i < N; ++i) {
            cbar_re += mult * gbar[i] * cs[i];
            cbar_im -= mult * gbar[i] * sn[i];
        }
        if (!sp) cbar_im = 0.0;
        /* c = gamma p / W0 */
        double p_re = dcr[it] * W0 / gamma, p_im = dci[it] * W0 / gamma;
        *gammabar += (cbar_re * p_re + cbar_im * p_im) / W0;
        W0bar -= (cbar_re * dcr[it] + cbar_im * dci[it]) / W0;
        double pbar_re = gamma / W0 * cbar_re, pbar_im = gamma / W0 * cbar_im;
        /* p_re = sum rw cos, p_im = -sum rw sin, rw = w (f - g_prev) on A */
        for (size_t i = 0; i < N; ++i) {
            if (wL[i] == 0.0) continue;
            double qv = pbar_re * cs[i] - pbar_im * sn[i];
            fbar[i] += wL[i] * qv;
            gbar[i] -= wL[i] * qv;
            wbar[i] += (fL[i] - gprev[i]) * qv;
        }
    }
    for (size_t i = 0; i < N; ++i)
        if (wL[i] != 0.0) wbar[i] += W0bar;
    free(g); free(gh); free(dcr); free(dci); free(gbar); free(cs); free(sn);
    return ORC_OK;
}

int oracle_batch_volume(const float* video, const unsigned char* avail, int frames, int height,
                        int width, int pitch, const int* blocks, int n_blocks,
                        const oracle_vplan* plan, double* out_blocks, int* status, double* w0,
                        int* path, double* dc_re, double* dc_im, double* gap, int n_threads) {
    return oracle_batch_volume_mode(video, avail, frames, height, width, pitch, blocks, n_blocks,
                                    plan, out_blocks, status, w0, path, dc_re, dc_im, gap,
                                    n_threads, 0);
}
