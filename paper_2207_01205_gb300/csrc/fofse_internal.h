// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fofse.h"

namespace fofse {

// Per-block status beyond the public FOFSE_BLK_* values: the block's input
// staging did not complete within its bounded wait.
constexpr int kBlkTimeout = 3;
// Bits of the device error word.
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrParam = 2u;  // a device-side rho / gamma out of range

// Device copies of a plan's constant tables (allocated in fofse_plan_create).
struct PlanTables {
  const float2* w_ff;     // Ls*Ls: rho^dist as (hi, lo) float pair
  const double* w_f64;    // Ls*Ls
  const float* w_f32;     // Ls*Ls
  const float4* tw_ff;    // T/2: exp(-j 2 pi e / T) as (re.h, im.h, re.l, im.l)
  const double2* tw_f64;  // T/2
  const float2* tw_f32;   // T/2
  const float2* syn_f32;  // T: (cos, sin)(2 pi p / T)
  const double2* syn_f64; // T
  const float4* syn_ff;   // T: (cos.h, sin.h, cos.l, sin.l)(2 pi p / T)
  const double* dist;     // Ls*Ls: distance to the centre of B (Eq. 15)
  const float2* dct_cos_ff;  // 4T: cos(2 pi p / (4T)) as (hi, lo), the DCT basis' phases
  // nullable: the DCT basis' product table C (rows 0 .. 2T-2 of 2T (hi, lo)
  // pairs) of the complete support -- every sample of L outside B (and inside
  // the causal shape where that support is set) usable -- for the plan's own
  // rho; blocks whose support is complete copy it instead of rebuilding it
  const float2* dct_c_full;
};

struct PlanDev {
  int block, border, Ls, T, iters, support, precision;
  int variant;  // launch shape of the product kernel (0 = default)
  int compensation;  // FOFSE_COMP_CONSTANT (Eq. 14) or FOFSE_COMP_OFSE (Eq. 10-13)
  int basis;         // FOFSE_BASIS_DFT or FOFSE_BASIS_DCT
  float gamma_h, gamma_l;  // gamma as float pair
  double gamma;
  float rho;
  PlanTables tab;
  // nullable: this plan's (rho, gamma) in device memory, read by the kernels
  // instead of rho / gamma above (the weight tables in `tab` then come from
  // the same rho, rebuilt on the device for the call)
  const float* rho_gamma_dev;
};

// w = rho^dist of one plan into the three weight tables (FP64, float pair,
// float), rho and gamma read from device memory; out-of-range values give NaN
// weights and set kErrParam.
cudaError_t launch_plan_weights(const PlanDev& p, const float* rho_gamma, float2* w_ff,
                                double* w_f64, float* w_f32, unsigned* err, cudaStream_t s);

struct FwdArgs {
  PlanDev plan;
  int plan_index;
  const fofse_block* blocks;
  int n_blocks;
  const float* frame;
  const uint8_t* avail;
  int height, width, pitch;
  float* out_frame;
  float* out_blocks;
  int out_stride;     // floats per block row = out_ld * out_ld
  int out_ld;         // largest block side of the call
  fofse_trace_entry* trace;
  int trace_stride;
  float* w0;
  int32_t* status;
  int use_tma;
  int box_f, box_a;  // TMA box widths (elements) of the frame and mask tiles
  unsigned* err;
  int* queue;            // work-queue counter of this plan (zeroed before the launch); may be null
  void* scratch;         // global scratch, one slot per persistent CTA (may be null)
  size_t scratch_bytes;  // bytes available at scratch
  float2* gamma_out;     // nullable: compensation factor per iteration (trace layout)
};

struct BwdArgs {
  PlanDev plan;
  int plan_index;
  const fofse_block* blocks;
  int n_blocks;
  const float* frame;
  const uint8_t* avail;
  int height, width, pitch;
  const fofse_trace_entry* trace;
  int trace_stride;
  const float* w0;
  const float* grad_blocks;
  int grad_stride;
  int grad_ld;
  float* grad_frame;
  float* grad_rho_gamma;  // points at this plan's pair
  unsigned* err;
  // split form (set when the caller gives a workspace): the solve kernel
  // writes abar and W0bar per block, the sample kernel reads them
  float2* abar;      // n_blocks x trace_stride
  float* w0bar;      // n_blocks
  double* acc;       // n_blocks x 4 FP64 sums for d/drho (zeroed before the call)
  unsigned* cnt;     // n_blocks finished-CTA counters (zeroed before the call)
};

struct CurveArgs {
  PlanDev plan;
  int plan_index;
  const fofse_block* blocks;
  int n_blocks;
  const fofse_trace_entry* trace;
  int trace_stride;
  const float* truth;
  int height, width, pitch;
  float* sse;  // n_blocks x trace_stride
};

// FOFSE_E_CUDA for a failed CUDA call, remembered for fofse_last_cuda_error.
fofse_status record_cuda_error(cudaError_t e);

// Launchers (one per translation unit).  Return cudaSuccess or the launch error.
cudaError_t launch_forward(const FwdArgs& a, const CUtensorMap* tm_frame,
                           const CUtensorMap* tm_avail, cudaStream_t stream);
// Global scratch the forward kernel of this plan uses when given enough
// (0 if none); a plan with forward_needs_scratch() fails without it.
size_t forward_scratch_bytes(const PlanDev& p);
bool forward_needs_scratch(const PlanDev& p);
int forward_variant_count(const PlanDev& p);
cudaError_t launch_backward(const BwdArgs& a, cudaStream_t stream);
// Squared error over B after each iteration count (fofse_curve.cu).
cudaError_t launch_error_curve(const CurveArgs& a, cudaStream_t stream);
// The register-blocked filtered-exact forward (fofse_fwd3.cu): launch (needs
// scratch), the scratch it uses, and its number of launch shapes.
cudaError_t launch_forward_f3(const FwdArgs& a, const CUtensorMap* tm_frame,
                              const CUtensorMap* tm_avail, cudaStream_t stream);
size_t forward_f3_scratch_bytes(const PlanDev& p);
int forward_f3_variant_count(const PlanDev& p);
// FOFSE with the 2-D DCT-II basis (fofse_dct.cu): all bins in float-float.
cudaError_t launch_forward_dct(const FwdArgs& a, cudaStream_t stream);
cudaError_t launch_backward_dct(const BwdArgs& a, cudaStream_t stream);
int forward_dct_variant_count(const PlanDev& p);
// Elements (float2) of the DCT table C for fft_size T, and its build for the
// complete support of plan p into `out` (one CTA, queued on s).
size_t dct_table_elems(int T);
cudaError_t build_dct_table(const PlanDev& p, float2* out, cudaStream_t s);
// The same kernel with OFSE's compensation (fofse_ofse.cu); one launch shape.
cudaError_t launch_forward_ofse(const FwdArgs& a, const CUtensorMap* tm_frame,
                                const CUtensorMap* tm_avail, cudaStream_t stream);
size_t forward_ofse_scratch_bytes(const PlanDev& p);

}  // namespace fofse
