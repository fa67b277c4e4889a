/*
 * fofse.h -- C ABI of the GB300 (sm_103a) implementation of fast
 * orthogonality deficiency compensated frequency selective extrapolation
 * (FOFSE; J. Seiler and A. Kaup, arXiv 2207.01205).
 *
 * What the library computes (per lost block; paper Sec. 2 and Sec. 4):
 *   L     the area of the lost b x b block B plus a border of `border`
 *         samples on each side (Fig. 1); A = the usable samples of L outside B.
 *   w     w[m,n] = rho^dist[m,n] on A, 0 elsewhere (Eq. 4 with the isotropic
 *         model of Eq. 15), dist = Euclidean distance to the centre of B.
 *   R_w   = DFT_TxT(w f), W = DFT_TxT(w), L placed at the origin of a T x T
 *         grid (T = fft_size), unnormalised forward DFT (the transform
 *         operator of Eq. 8 for the 2-D DFT basis; "complete formulation in
 *         the transform domain", end of Sec. 2).
 *   loop  iters times: u = argmax |R_w[k]| over one index of every conjugate
 *         pair (Eq. 9); c = gamma * R_w[u] / W[0] (Eq. 5 and Eq. 14);
 *         R_w[k] -= c W[k-u] + s(u) conj(c) W[k+u]  (the spectrum of the
 *         added basis pair, Eq. 2-3 and Eq. 7), s(u) = 0 for the four
 *         self-conjugate indices (2u = 0 mod T), else 1.
 *   out   B_hat[m,n] = sum_i (1 + s(u_i)) Re(c_i exp(+j 2 pi (u_i . (m,n)) / T))
 *         over B (Eq. 1).
 * Readings of points the paper leaves open: the argmax runs over the
 * canonical set H = {k : k1 T + k2 <= (-k)1 T + (-k)2} and exact ties go to
 * the smallest k1 T + k2; the coefficient of a self-conjugate index is real;
 * samples outside the frame, in other lost blocks or outside the chosen
 * support shape are not in A.
 * Variants selected per plan: OFSE's compensation (Sec. 3, Eq. 10-13:
 * c = P[u]^2 / Q[u] with Q[u] = sum_l P[l] W[u - l]) instead of the constant
 * gamma, and the real 2-D DCT-II basis instead of the DFT (fofse_plan_set_
 * compensation, fofse_plan_set_basis).  Besides the forward: the adjoint along
 * the frozen selection path (fofse_backward), the squared error after every
 * iteration count (fofse_error_curve), the compensation factor of every
 * iteration (fofse_extrapolate_batch_gamma), and rho / gamma read from device
 * memory per call (d_rho_gamma).  Video volumes (the method over
 * three-dimensional sets, Sec. 1) have their own plans and batch call
 * (fofse_volume_plan_create, fofse_extrapolate_volume_batch), documented with
 * their readings further down.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are DEVICE memory owned by the caller, on the device
 *    that was current when the plans were created.  Every plan of a call must
 *    have been created on the device that is current at the call: the calls
 *    return FOFSE_E_ARG otherwise (before any launch).  The library never
 *    allocates or frees memory on the launch path (plans allocate their small
 *    constant tables once, in fofse_plan_create, and the DCT basis' table in
 *    fofse_plan_set_basis).
 *  - Frames are row-major float32 with `pitch` elements per row; availability
 *    masks are uint8 (1 = usable sample, 0 = lost) with the same pitch.
 *  - Argument errors are reported synchronously through the return value and
 *    nothing is launched.  Per-block conditions go to d_block_status.  Device
 *    faults the kernels detect themselves (a bounded wait that ran out) set a
 *    device error word read by fofse_check.  No kernel traps.
 *  - All launches go to `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream) and are asynchronous.
 */
#ifndef FOFSE_H_
#define FOFSE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fofse_plan_s* fofse_plan;

typedef enum {
  FOFSE_OK = 0,
  FOFSE_E_ARG = 1,          /* invalid argument (null pointer, size, range)        */
  FOFSE_E_UNSUPPORTED = 2,  /* valid but not implemented (e.g. fft_size 256)       */
  FOFSE_E_NOMEM = 3,        /* plan table allocation failed                        */
  FOFSE_E_CUDA = 4,         /* a CUDA runtime call failed                          */
  FOFSE_E_TIMEOUT = 5,      /* a device-side bounded wait ran out (fofse_check)    */
  FOFSE_E_STATE = 6         /* call out of order                                   */
} fofse_status;

/* support shapes: which part of L may be in A */
enum { FOFSE_SUPPORT_FULL = 0,      /* all of L outside B (concealment)                 */
       FOFSE_SUPPORT_CAUSAL_L = 1 }; /* rows above B up to B's right edge, plus the
                                        samples left of B in B's rows (prediction)      */
/* arithmetic of the kernels (the values 2 and 4 are not used) */
enum { FOFSE_FP32 = 0,           /* the product: exact selection path and coefficients
                                    with FP32 instructions.  With the workspace: FP32
                                    working spectrum with a rigorous error bound, near
                                    ties and every coefficient evaluated exactly (the
                                    register-blocked kernel); without it, as
                                    FOFSE_FP32_FULLFF                                   */
       FOFSE_FP64_VALIDATE = 1,  /* IEEE double; slow on GB300, for validation           */
       FOFSE_FP32_FULLFF = 3 };  /* every bin updated in float-float (pairs of FP32)      */
/* compensation of the projection coefficient */
enum { FOFSE_COMP_CONSTANT = 0,  /* c = gamma p_u with the plan's constant gamma (Eq. 14):
                                    FOFSE, the default                                  */
       FOFSE_COMP_OFSE = 1 };    /* OFSE's compensation (Eq. 10-12): c = p_u / sum_l
                                    (p_l / p_u) Khat[u, l]; with the DFT basis
                                    Khat[u, l] = W[u - l] / W[0], so c = P[u]^2 / Q[u]
                                    with Q[u] = sum_l P[l] W[u - l], gamma unused      */
/* basis functions */
enum { FOFSE_BASIS_DFT = 0,      /* 2-D DFT on the T x T grid (the paper's experiments)   */
       FOFSE_BASIS_DCT = 1 };    /* 2-D DCT-II on the T x T grid, L at its origin: real
                                    phi_k = cos(pi k1 (2m+1)/(2T)) cos(pi k2 (2n+1)/(2T));
                                    selection by the orthonormal DCT magnitude, c =
                                    gamma sum w r phi_u / sum w phi_u^2 (Eq. 5, 14)    */
/* per-block status written to d_block_status */
enum { FOFSE_BLK_OK = 0, FOFSE_BLK_NO_SUPPORT = 1, FOFSE_BLK_NONFINITE = 2 };

/* One lost block: top-left corner of B in the frame and the plan index. */
typedef struct {
  int32_t y, x;
  int32_t plan;
} fofse_block;

/* One iteration of the selection path: canonical index u (0 <= u1, u2 < T)
 * and the coefficient c = gamma R_w[u] / W[0] (OFSE plans: P[u]^2 / Q[u]),
 * rounded to FP32. */
typedef struct {
  int16_t u1, u2;
  float dc_re, dc_im;
} fofse_trace_entry;

/*
 * fofse_plan_create -- parameters of one block class (paper Sec. 4:
 * 16 x 16 blocks, border 16, 64 x 64 FFT, rho 0.8, gamma, iterations).
 *   block     lost block side b, 1 <= b
 *   border    support border width, 0 <= border
 *   fft_size  T in {32, 64, 128}, T >= block + 2 * border
 *   rho       rho_hat of Eq. 15, 0 < rho <= 1
 *   gamma     constant compensation factor of Eq. 14, 0 < gamma <= 1
 *   iters     number of iterations I, 1 <= I <= 4096
 * Builds the plan's constant tables in device memory of the current device:
 * distances to the centre of B and DFT twiddles (from integer phases) on the
 * host in FP64, the weights rho^dist by a kernel (FP64, also split into float
 * pairs and rounded to float), after which it synchronises the legacy default
 * stream (so not while a CUDA graph is being captured).
 * Returns FOFSE_E_ARG for invalid values, FOFSE_E_UNSUPPORTED for a valid but
 * unimplemented fft_size, FOFSE_E_NOMEM / FOFSE_E_CUDA if the tables cannot
 * be allocated.  *out is set only on FOFSE_OK.  Plans are immutable during a
 * launch and may be shared by concurrent launches.
 */
fofse_status fofse_plan_create(int block, int border, int fft_size, float rho, float gamma,
                               int iters, fofse_plan* out);
/* Support shape (FOFSE_SUPPORT_*); default FULL.  FOFSE_E_ARG for other values.
 * For a DCT plan this rebuilds the plan's shared table (fofse_plan_set_basis). */
fofse_status fofse_plan_set_support(fofse_plan plan, int shape);
/* Arithmetic (FOFSE_FP32 default, FOFSE_FP64_VALIDATE, FOFSE_FP32_FULLFF);
 * FOFSE_E_ARG for other values. */
fofse_status fofse_plan_set_precision(fofse_plan plan, int precision);
/* Compensation (FOFSE_COMP_*); default FOFSE_COMP_CONSTANT.  FOFSE_COMP_OFSE
 * runs only with FOFSE_FP32 and a workspace (fofse_extrapolate_batch returns
 * FOFSE_E_UNSUPPORTED otherwise) and has no backward (fofse_backward returns
 * FOFSE_E_UNSUPPORTED: the adjoint of c = P^2 / Q and of Q's recurrence is not
 * built; OFSE serves as the paper's comparison method).  It needs twice the
 * forward scratch of the constant compensation.  FOFSE_E_ARG for other values. */
fofse_status fofse_plan_set_compensation(fofse_plan plan, int compensation);
/* Basis (FOFSE_BASIS_*); default FOFSE_BASIS_DFT.  FOFSE_BASIS_DCT runs its
 * own kernel with exact decisions, for fft_size 32 and 64, precision
 * FOFSE_FP32 or FOFSE_FP32_FULLFF and the constant compensation (the batch
 * calls return FOFSE_E_UNSUPPORTED otherwise): with FOFSE_FP32 an FP32
 * working spectrum with a rigorous bound, near-ties and coefficients resolved
 * exactly (launch-shape variant 0), or every bin in float-float (variant 1,
 * and always with FOFSE_FP32_FULLFF).  It needs no workspace (work-queue
 * counters are used when one is given).  The trace holds u = (k1, k2) in
 * [0, T)^2 and the real coefficient (dc_im = 0); fofse_backward runs the
 * adjoint of this basis' recursion (one block per CTA).  Selecting the DCT
 * basis builds, synchronously on the current device (the plan's), the basis'
 * product table C of the complete support -- every sample of L outside B, and
 * inside the support shape, usable -- for the plan's rho, folded to indices
 * 0..T (C[2T - a] = -C[a]): (T + 1) x (T + 2) float pairs (34 KB at fft_size
 * 64), freed with the plan.  Every block starts
 * from it (C is linear in the weights; a block with missing samples subtracts
 * their part); a call with d_rho_gamma builds the table for its rho in its
 * workspace.  FOFSE_E_ARG for other values or another current device;
 * FOFSE_E_NOMEM / FOFSE_E_CUDA if the table could not be built (the basis is
 * set all the same, and every block then builds C itself). */
fofse_status fofse_plan_set_basis(fofse_plan plan, int basis);
/* Number of launch shapes (threads per block / resident blocks per SM) of the
 * plan's kernel for its current precision; 0 for a NULL plan. */
int fofse_plan_variant_count(fofse_plan plan);
/* Selects launch shape `variant` (0 <= variant < fofse_plan_variant_count;
 * default 0), e.g. from an autotuner.  Every shape computes the same result up
 * to the rounding of float-float sums.  FOFSE_E_ARG otherwise.  Changing the
 * precision resets an out-of-range variant to 0. */
fofse_status fofse_plan_set_variant(fofse_plan plan, int variant);
/* The plan's block side, border, fft_size and iteration count (the values it
 * was created with); each output pointer may be NULL.  Lets a caller size the
 * outputs of a batch (bmax = largest block side, max_iters = largest
 * iteration count over the call's plans).  FOFSE_E_ARG for a NULL plan. */
fofse_status fofse_plan_get_shape(fofse_plan plan, int* block, int* border, int* fft_size,
                                  int* iters);
/* Frees the plan's tables (synchronises the device, so not while a CUDA graph
 * is being captured on it).  NULL is ignored. */
void fofse_plan_destroy(fofse_plan plan);

/*
 * fofse_workspace_bytes -- device scratch for fofse_extrapolate_batch and
 * fofse_backward with these plans and n_blocks blocks on the current device;
 * the weight tables of a call with device-side (rho, gamma) (20 bytes per
 * sample of L per plan), then the larger of the two calls' own needs (the
 * calls never use it at the same time).
 * Forward: 256 bytes of work-queue counters (one per plan, zeroed by every
 * call) plus one slot per resident CTA of the largest plan kernel: the block's
 * FFT buffer, then its exact W, and its exact initial spectrum (FOFSE_FP32:
 * 96 KB per CTA at fft_size 64, about 90 MB on 152 SMs; 384 KB at fft_size
 * 128).  Backward: per block, the adjoint coefficients (8 bytes per iteration)
 * and 44 bytes of sums and counters.  Returns 0 for invalid arguments (more
 * than 64 plans, a NULL plan).
 */
size_t fofse_workspace_bytes(const fofse_plan* plans, int n_plans, int n_blocks);

/*
 * fofse_extrapolate_batch -- extrapolate every block of d_blocks (forward).
 *   plans, n_plans     host array of plans; d_blocks[i].plan indexes it
 *   d_blocks           device array of n_blocks fofse_block; B must lie inside
 *                      the frame (the rest of L may extend beyond it)
 *   d_frame, d_avail   device frame (float32) and availability (uint8),
 *                      height x width, `pitch` elements per row; the values of
 *                      unavailable samples are never read into the arithmetic
 *   d_rho_gamma        nullable; n_plans x 2 floats in device memory, (rho, gamma)
 *                      of each plan for this call in place of the plan's own
 *                      values (tuning loops and CUDA graphs that change them
 *                      without a host round trip).  The weights rho^dist are
 *                      rebuilt on the device at the start of the call (into
 *                      the workspace, which is then required: FOFSE_E_ARG
 *                      without it).  A value out of range (rho or gamma not
 *                      in (0, 1], NaN) gives that plan's blocks status
 *                      FOFSE_BLK_NONFINITE and makes fofse_check return
 *                      FOFSE_E_ARG.
 *   d_out_frame        nullable; B_hat is written into it at each block (other
 *                      samples untouched); may alias d_frame only if no block's
 *                      L overlaps another block's B
 *   d_out_blocks       nullable; n_blocks x bmax x bmax floats, bmax = the
 *                      largest block side over the plans; B_hat fills the
 *                      top-left b x b corner of its bmax x bmax row-major tile,
 *                      the rest is written as zero
 *   d_trace, d_w0      nullable; n_blocks x max_iters entries (max over the plans;
 *                      entries past a block's own iteration count are zero) /
 *                      n_blocks floats (W[0] = sum of w); required for
 *                      fofse_backward
 *   d_block_status     nullable; n_blocks int32 (FOFSE_BLK_*).  Blocks that are
 *                      not OK get B_hat = 0 and an all-zero trace
 *   d_workspace        fofse_workspace_bytes() bytes, caller-owned, 256-byte
 *                      aligned; may be NULL when no plan has fft_size 128 (blocks
 *                      are then dealt to the CTAs round-robin instead of through
 *                      the work queue, and FOFSE_FP32 plans run as
 *                      FOFSE_FP32_FULLFF).  A workspace must not be shared by
 *                      calls that may run concurrently.
 *   stream             cudaStream_t
 * Plans are processed largest first (iters * T^2), each by a persistent kernel
 * whose CTAs take that plan's blocks from a work queue.  All plans of one call
 * must share the precision; at most 64 plans.  Returns FOFSE_OK once the work
 * is queued, FOFSE_E_ARG if a fft_size-128 plan is given no workspace.
 */
fofse_status fofse_extrapolate_batch(const fofse_plan* plans, int n_plans,
                                     const fofse_block* d_blocks, int n_blocks,
                                     const float* d_frame, const uint8_t* d_avail, int height,
                                     int width, int pitch, const float* d_rho_gamma,
                                     float* d_out_frame, float* d_out_blocks,
                                     fofse_trace_entry* d_trace, float* d_w0,
                                     int32_t* d_block_status, void* d_workspace, void* stream);

/*
 * fofse_extrapolate_batch_gamma -- fofse_extrapolate_batch that also writes
 * the compensation factor of every iteration, gamma_u = c_u / p_u (Eq. 13):
 *   d_gamma   nullable; n_blocks x max_iters x 2 floats (re, im), the trace's
 *             layout: the plan's constant gamma (im 0) for FOFSE_COMP_CONSTANT
 *             plans, W[0] P[u] / Q[u] for FOFSE_COMP_OFSE plans (complex with
 *             the complex DFT basis; the canonical member u of the pair).
 *             Entries past a block's iteration count, and all entries of a
 *             block that is not OK, are zero.
 * A non-NULL d_gamma needs FOFSE_FP32 plans and a workspace
 * (FOFSE_E_UNSUPPORTED otherwise).  Other arguments and returns as
 * fofse_extrapolate_batch (which is this call with d_gamma = NULL).
 */
fofse_status fofse_extrapolate_batch_gamma(const fofse_plan* plans, int n_plans,
                                           const fofse_block* d_blocks, int n_blocks,
                                           const float* d_frame, const uint8_t* d_avail,
                                           int height, int width, int pitch,
                                           const float* d_rho_gamma, float* d_out_frame,
                                           float* d_out_blocks, fofse_trace_entry* d_trace,
                                           float* d_w0, int32_t* d_block_status,
                                           float* d_gamma, void* d_workspace, void* stream);

/*
 * fofse_extrapolate_batch_noalloc -- fofse_extrapolate_batch for callers that
 * cannot allocate device memory at all: code running where cudaMalloc is not
 * allowed (for example inside a host callback or under a custom allocator that
 * forbids it), or a host framework that owns every device buffer and passes
 * only its inputs and outputs.  This entry point has no counterpart in the
 * paper; it exists only for those callers.
 *
 * Arguments as in fofse_extrapolate_batch, without d_rho_gamma and
 * d_workspace.  Instead of a workspace it uses one fixed array inside the
 * library: 64 int work-queue counters (256 bytes) that every GPU loading the
 * library holds until the process exits.  It never calls cudaMalloc or
 * cudaFree.  Limits: at most 64 plans (FOFSE_E_ARG beyond), fft_size 32 or 64
 * only (a 128 x 128 FFT needs 256 KB of scratch per SM: FOFSE_E_UNSUPPORTED).
 * Without a workspace there is no per-CTA scratch for the exact spectra, so
 * FOFSE_FP32 plans run the kernel that updates every bin in float-float (the
 * FOFSE_FP32_FULLFF arithmetic: the same exact selection path and
 * coefficients up to float-float rounding, about half the speed of the
 * workspace path) and the plan's launch-shape variant is ignored; DCT and
 * FOFSE_FP64_VALIDATE plans run their usual kernels.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept per device for the life
 *    of the process: after a cudaDeviceReset in the same process it is stale,
 *    so do not call this entry point again after a reset.
 *  - Every call shares the array and clears the counters it uses at its start
 *    (an asynchronous memset on `stream`).  Calls whose work can overlap on the
 *    GPU (different streams, or different host threads) race on it: serialise
 *    them.
 */
fofse_status fofse_extrapolate_batch_noalloc(const fofse_plan* plans, int n_plans,
                                             const fofse_block* d_blocks, int n_blocks,
                                             const float* d_frame, const uint8_t* d_avail,
                                             int height, int width, int pitch,
                                             float* d_out_frame, float* d_out_blocks,
                                             fofse_trace_entry* d_trace, float* d_w0,
                                             int32_t* d_block_status, void* stream);

/*
 * fofse_backward -- adjoint of fofse_extrapolate_batch with the selection path
 * frozen (the map from the support samples to B_hat is then linear).
 *   d_rho_gamma        nullable; as in fofse_extrapolate_batch (the same values
 *                      as the forward call), needs the workspace
 *   d_trace, d_w0      from the forward call with the same inputs
 *   d_grad_blocks      dloss/dB_hat, n_blocks x bmax x bmax (as d_out_blocks)
 *   d_grad_frame       nullable; dloss/df ACCUMULATED (+=) at every sample of A
 *   d_grad_rho_gamma   nullable; n_plans x 2 floats, ACCUMULATED (+=)
 *   d_workspace        nullable; fofse_workspace_bytes() bytes for the same
 *                      plans and n_blocks.  With it the adjoint runs as two
 *                      kernels (a per-block triangular solve, then a sample
 *                      pass spread over several CTAs per block); without it,
 *                      as one kernel per block (slower on large batches).
 *                      Must not be shared with a call that may run at the
 *                      same time.
 * Not implemented for FOFSE_FP64_VALIDATE plans nor for FOFSE_COMP_OFSE plans
 * (FOFSE_E_UNSUPPORTED).
 */
fofse_status fofse_backward(const fofse_plan* plans, int n_plans, const fofse_block* d_blocks,
                            int n_blocks, const float* d_frame, const uint8_t* d_avail,
                            int height, int width, int pitch, const float* d_rho_gamma,
                            const fofse_trace_entry* d_trace, const float* d_w0,
                            const float* d_grad_blocks, float* d_grad_frame,
                            float* d_grad_rho_gamma, void* d_workspace, void* stream);

/*
 * fofse_error_curve -- the squared error of the extrapolation after every
 * iteration count (the PSNR-over-iterations curves of Fig. 4 and Fig. 5):
 *   d_trace       from fofse_extrapolate_batch with the same plans and blocks
 *   d_truth       device float32 reference frame, height x width, `pitch`
 *                 elements per row (the same geometry as the frame)
 *   d_sse         n_blocks x max_iters floats: entry nu - 1 is the sum over B
 *                 of (clip(B_hat_nu, 0, 255) - truth)^2, with B_hat_nu the
 *                 model of Eq. 1 built from the first nu trace entries (in the
 *                 plan's basis); zero
 *                 past a block's iteration count.  PSNR over a set of blocks
 *                 is 10 log10(255^2 N / sum of their entries) for N samples.
 * The model is rebuilt from the trace's FP32 coefficients in FP32.  Blocks
 * with side above 32 are not supported (FOFSE_E_UNSUPPORTED); argument errors
 * as fofse_extrapolate_batch.  Asynchronous on `stream`.
 */
fofse_status fofse_error_curve(const fofse_plan* plans, int n_plans, const fofse_block* d_blocks,
                               int n_blocks, const fofse_trace_entry* d_trace,
                               const float* d_truth, int height, int width, int pitch,
                               float* d_sse, void* stream);

/* Synchronises `stream`, then reads and clears the device error word of the
 * current device: FOFSE_OK, FOFSE_E_TIMEOUT (a bounded wait ran out),
 * FOFSE_E_ARG (a device-side rho / gamma was out of range), or FOFSE_E_CUDA if
 * the stream reported an error. */
fofse_status fofse_check(void* stream);

/* The cudaError_t value behind the most recent FOFSE_E_CUDA returned to the
 * calling thread (0 if there was none), and its static name (e.g.
 * "cudaErrorInvalidValue").  No counterpart in the paper: host-side error
 * reporting of this library. */
int fofse_last_cuda_error(void);
const char* fofse_last_cuda_error_string(void);

/*
 * Video volumes (Sec. 1: the method carried over to three-dimensional sets;
 * the paper gives no formulas for them, so the following are this library's
 * readings).  The area around a lost b x b block B in frame t is a volume of
 * Lt = 2 depth + 1 frames (t - depth .. t + depth) of Ls x Ls samples,
 * Ls = b + 2 border, indexed (tau, m, n) with B's frame at tau = depth.
 *   w     rho^d on A, d = Euclidean distance to the centre of B in frame t,
 *         one frame counting as one sample (Eq. 15 over three coordinates);
 *         A = the usable samples of the volume (inside the video, mask 1)
 *         except B in frame t (B's position in the other frames is in A).
 *   basis the 3-D DFT on a T x T x Tt grid (T = fft_size for m and n,
 *         Tt = fft_time for tau), the volume at its origin:
 *         phi_k = exp(+j 2 pi (k1 m / T + k2 n / T + k3 tau / Tt)).
 *   loop  as for images (Sec. 2, Eq. 1-9, Eq. 14): R = DFT(w f), W = DFT(w);
 *         u = argmax |R[k]| over the canonical set {k : lin(k) <= lin(-k)},
 *         lin(k) = (k1 T + k2) Tt + k3, exact ties to the smallest lin(k);
 *         c = gamma R[u] / W[0] (real for the eight self-conjugate u, 2u = 0
 *         mod (T, T, Tt)); R[k] -= c W[k - u] + s(u) conj(c) W[k + u].
 *   out   B_hat[m,n] = sum_i (1 + s(u_i)) Re(c_i phi_{u_i}[depth, border + m,
 *         border + n]), the model over B in frame t (Eq. 1).
 * Arithmetic (per plan, fofse_volume_plan_set_precision): FOFSE_FP32, the
 * default and the product, runs the design of the two-dimensional FOFSE_FP32
 * kernel on the 3-D grid (FP32 working spectrum with a rigorous error bound,
 * exact float-float decisions and coefficients; float-float transforms; it
 * needs a workspace); FOFSE_FP64_VALIDATE runs the whole recursion in IEEE
 * double (one CTA per block, both spectra in shared memory; grids up to 4096
 * bins).  With depth 0 and fft_time 1 it is the two-dimensional method with
 * the full support shape.
 */
typedef struct fofse_volume_plan_s* fofse_volume_plan;

/* One lost block of a video: frame index and top-left corner of B. */
typedef struct {
  int32_t t, y, x;
} fofse_volume_block;

/*
 * fofse_volume_plan_create -- parameters of extrapolation over volumes.
 *   block     lost block side b, 1 <= b, b * b <= 512 (1024 when
 *             fft_size^2 * fft_time >= 2048)
 *   border    spatial border width, 0 <= border, b + 2 border <= fft_size
 *   depth     frames on each side of B's frame, 0 <= depth, 2 depth + 1 <= fft_time
 *   fft_size  T in {16, 32, 64}
 *   fft_time  Tt in {1, 2, 4, 8}, T^2 Tt <= 16384
 *   rho       rho_hat of Eq. 15, 0 < rho <= 1
 *   gamma     constant compensation factor of Eq. 14, 0 < gamma <= 1
 *   iters     number of iterations I, 1 <= I <= 4096
 * Builds the weight table rho^d (FP64 and float pairs, by a kernel on the
 * current device), the twiddle and synthesis tables, and synchronises the
 * legacy default stream.  The plan starts with FOFSE_FP32.  FOFSE_E_ARG for
 * invalid values, FOFSE_E_UNSUPPORTED for a valid grid without a kernel (other
 * T or Tt, or T^2 Tt > 16384), FOFSE_E_NOMEM / FOFSE_E_CUDA if the tables
 * cannot be built.  *out is set only on FOFSE_OK.
 */
fofse_status fofse_volume_plan_create(int block, int border, int depth, int fft_size, int fft_time,
                                      float rho, float gamma, int iters, fofse_volume_plan* out);

/* Arithmetic of the plan's calls: FOFSE_FP32 (default) or FOFSE_FP64_VALIDATE.
 * FOFSE_E_ARG for a NULL plan or another value; FOFSE_E_UNSUPPORTED for FP64
 * on a grid above 4096 bins or fft_size 64, or a block with b^2 above twice the
 * FP64 kernel's threads (512 or 256 by the grid). */
fofse_status fofse_volume_plan_set_precision(fofse_volume_plan plan, int precision);

/* Launch shapes of the FP32 volume kernel for this plan's grid (threads per
 * CTA and resident CTAs per SM; 0 for a NULL plan).  Every shape computes the
 * same result up to the order of the exact-value sums, which the 64-bit fixed
 * point makes exact: identical paths and outputs.  set_variant selects one
 * (default 0); FOFSE_E_ARG for a NULL plan or a variant out of range.  FP64
 * plans ignore the variant. */
int fofse_volume_plan_variant_count(fofse_volume_plan plan);
fofse_status fofse_volume_plan_set_variant(fofse_volume_plan plan, int variant);

/* Device scratch for fofse_extrapolate_volume_batch with this plan on the
 * current device: 256 bytes of work-queue counter plus, per resident CTA of
 * the FP32 kernel, the block's float-float 3-D transform (then its exact W)
 * and its exact initial spectrum per held bin: 24 K + 32 Tt bytes per CTA for
 * K = T^2 Tt bins (about 60 MB on 152 SMs at 64 x 64 x 4, one CTA per SM),
 * the largest over the plan's launch shapes, so that one workspace serves every
 * variant.  0 for FP64 plans (they need none) and for a NULL plan. */
size_t fofse_volume_workspace_bytes(fofse_volume_plan plan, int n_blocks);

/* Frees the plan's tables (synchronises the device, so not while a CUDA graph
 * is being captured on it).  NULL is ignored. */
void fofse_volume_plan_destroy(fofse_volume_plan plan);

/*
 * fofse_extrapolate_volume_batch -- extrapolate every block of d_blocks.
 *   d_blocks          device array of n_blocks fofse_volume_block (any position:
 *                     samples outside the video are not in A)
 *   d_video, d_avail  device video (float32) and availability (uint8):
 *                     `frames` frames back to back, each height rows of
 *                     `pitch` elements (frame stride height * pitch)
 *   d_out_blocks      n_blocks x b x b floats, B_hat row-major (required)
 *   d_path            nullable; n_blocks x iters x 3 int32 (u1, u2, u3)
 *   d_coef            nullable; n_blocks x iters x 2 doubles (re, im of c)
 *   d_w0              nullable; n_blocks doubles, W[0] = sum of w
 *   d_block_status    nullable; n_blocks int32 (FOFSE_BLK_*); blocks that are
 *                     not OK get B_hat = 0 and an all-zero path and coef
 *   d_workspace       fofse_volume_workspace_bytes() bytes, caller-owned,
 *                     256-byte aligned; required for FOFSE_FP32 plans (NULL
 *                     for FP64 plans); not to be shared by calls that may run
 *                     at the same time
 *   stream            cudaStream_t
 * Returns FOFSE_OK once queued (n_blocks = 0 launches nothing), FOFSE_E_ARG for
 * a NULL plan or required pointer (the workspace of an FP32 plan included), a
 * non-positive size, or a current device other than the one the plan was
 * created on; FOFSE_E_CUDA if the launch failed.
 */
fofse_status fofse_extrapolate_volume_batch(fofse_volume_plan plan,
                                            const fofse_volume_block* d_blocks, int n_blocks,
                                            const float* d_video, const uint8_t* d_avail,
                                            int frames, int height, int width, int pitch,
                                            float* d_out_blocks, int32_t* d_path, double* d_coef,
                                            double* d_w0, int32_t* d_block_status,
                                            void* d_workspace, void* stream);

/*
 * fofse_volume_backward -- gradients of a loss on the volume batch's B_hat
 * along the frozen selection path (not in the paper: the adjoint of the
 * recursion of fofse_extrapolate_volume_batch with every u_i fixed, as
 * fofse_backward does for images).  With p_i = sum_A w r_{i-1} conj(phi_i),
 * c_i = gamma p_i / W[0], g_i = g_{i-1} + (1 + s(u_i)) Re(c_i phi_i) and
 * W = DFT(w) on the grid, the reverse sweep is a triangular solve on W's
 * values at the sums and differences of the path's indices (pbar_i, the
 * adjoint of p_i, from the DFT of dl/dB_hat at u_i), then a pass over the
 * trace per sample of A: dl/df = w sum_i Re(pbar_i phi_i), dl/dw = sum_i
 * r_{i-1} Re(pbar_i phi_i) + dl/dW[0], dl/drho through w = rho^d (d the
 * distance to the centre of B in frame `depth`), and dl/dgamma.  FP32 (FP64
 * for the rho sums); two kernels (per block: W by separable DFTs and the
 * solve; over chunks of each block's samples: the sample pass).
 *   d_blocks .. pitch    the forward call's blocks and video
 *   d_path, d_coef, d_w0 the forward call's outputs for these blocks (path
 *                        n x iters x 3 int32, coefficients n x iters x 2 FP64,
 *                        W[0] n FP64)
 *   d_block_status       nullable; the forward's statuses: blocks not OK are
 *                        skipped (without it, blocks with W[0] <= 0)
 *   d_grad_blocks        dl/dB_hat, n x b x b float32
 *   d_grad_video         nullable; dl/df ACCUMULATED (+=) into a buffer of
 *                        the video's layout (atomics: overlapping volumes add)
 *   d_grad_rho_gamma     nullable; 2 floats, (dl/drho, dl/dgamma) ACCUMULATED
 *   d_workspace          fofse_volume_backward_workspace_bytes() bytes,
 *                        caller-owned, 256-byte aligned
 * Returns FOFSE_OK once queued (n_blocks = 0 launches nothing), FOFSE_E_ARG
 * for a NULL plan or required pointer, a non-positive size or a current
 * device other than the plan's, FOFSE_E_UNSUPPORTED where the solve's shared
 * memory (8 T^2 Tt bytes of W, the row transforms of w and the per-iteration
 * arrays) exceeds 227 KB, FOFSE_E_CUDA if a launch failed.  The plan's
 * precision does not matter (the coefficients are read as given).
 */
size_t fofse_volume_backward_workspace_bytes(fofse_volume_plan plan, int n_blocks);
fofse_status fofse_volume_backward(fofse_volume_plan plan, const fofse_volume_block* d_blocks,
                                   int n_blocks, const float* d_video, const uint8_t* d_avail,
                                   int frames, int height, int width, int pitch,
                                   const int32_t* d_path, const double* d_coef, const double* d_w0,
                                   const int32_t* d_block_status, const float* d_grad_blocks,
                                   float* d_grad_video, float* d_grad_rho_gamma, void* d_workspace,
                                   void* stream);

/* Static, human-readable name of a status code. */
const char* fofse_status_string(fofse_status status);

/* Library version, e.g. 100 for 0.1.0. */
int fofse_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FOFSE_H_ */
