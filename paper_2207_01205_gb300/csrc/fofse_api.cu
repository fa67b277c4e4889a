// Host side of the C ABI declared in include/fofse.h: plan construction
// (constant tables computed in FP64 on the host), argument validation,
// TMA tensor-map encoding, kernel dispatch and the device error word.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fofse_internal.h"

using namespace fofse;

namespace fofse {

__global__ void fofse_plan_weights_kernel(const double* dist, int n, const float* rho_gamma,
                                          float2* w_ff, double* w_f64, float* w_f32,
                                          unsigned* err) {
  const float rho = rho_gamma[0], gamma = rho_gamma[1];
  const bool ok = rho > 0.f && rho <= 1.f && gamma > 0.f && gamma <= 1.f;  // false for NaN
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && !ok) atomicOr(err, kErrParam);
  if (i >= n) return;
  const double w = ok ? pow((double)rho, dist[i]) : __longlong_as_double(0x7ff8000000000000LL);  // Eq. 15
  const float hi = (float)w;
  w_ff[i] = make_float2(hi, (float)(w - (double)hi));
  w_f64[i] = w;
  w_f32[i] = hi;
}

cudaError_t launch_plan_weights(const PlanDev& p, const float* rho_gamma, float2* w_ff,
                                double* w_f64, float* w_f32, unsigned* err, cudaStream_t s) {
  const int n = p.Ls * p.Ls;
  fofse_plan_weights_kernel<<<(n + 255) / 256, 256, 0, s>>>(p.tab.dist, n, rho_gamma, w_ff, w_f64,
                                                            w_f32, err);
  return cudaGetLastError();
}

}  // namespace fofse

struct fofse_plan_s {
  int device;    // the device current at creation, which owns the tables (first
                 // member: host tests build a stand-in plan with only this set)
  PlanDev dev;   // scalars + device table pointers
  void* mem;     // one device allocation holding every table
  void* dct_mem; // the DCT basis' shared complete-support table (allocated with the basis)
};

namespace {

__device__ unsigned g_err_word;  // device error word (FOFSE kErr* bits)

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kMaxIters = 4096;

unsigned* err_word_ptr() {
  static std::mutex mu;
  static unsigned* cache[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_err_word) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<unsigned*>(p);
  }
  return cache[dev];
}

// Scratch of fofse_extrapolate_batch_noalloc: the per-plan work-queue
// counters, in a fixed array that every device loading this library keeps
// until the process exits (kNoAllocCounters ints = 256 bytes).  Host code must
// not pass `g_noalloc_queue` itself to a kernel (on the host it only names a
// stand-in); it passes the device address looked up below.
constexpr int kNoAllocCounters = 64;
static __device__ __align__(256) int g_noalloc_queue[kNoAllocCounters];

// Device address of g_noalloc_queue on the current device, looked up once per
// device (the first call on a device does this; later calls reuse it).
int* noalloc_queue_ptr() {
  static std::mutex mu;
  static int* cache[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    int* ptr = nullptr;
    if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_queue) != cudaSuccess) return nullptr;
    cache[dev] = ptr;
  }
  return cache[dev];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode_2d(CUtensorMap* map, CUtensorMapDataType ty, int esize, const void* base, int width,
               int height, int pitch, int box_w, int box_h) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * (cuuint64_t)esize};
  cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, ty, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Every plan of a call must belong to the current device: its tables live in
// that device's memory, and the kernels run on the current device.  False for
// a NULL plan, and when no device is current.
bool plans_on_current_device(const fofse_plan* plans, int n_plans) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  for (int i = 0; i < n_plans; ++i)
    if (!plans[i] || plans[i]->device != dev) return false;
  return true;
}

bool supported_T(int T) { return T == 32 || T == 64 || T == 128; }

// The DCT basis runs in one kernel: fft_size 32 or 64, FOFSE_FP32 or
// FOFSE_FP32_FULLFF, constant compensation.
bool dct_supported(const PlanDev& p) {
  if (p.basis != FOFSE_BASIS_DCT) return true;
  return (p.T == 32 || p.T == 64) && (p.precision == FOFSE_FP32 || p.precision == FOFSE_FP32_FULLFF) &&
         p.compensation == FOFSE_COMP_CONSTANT;
}

// CUDA runtime error behind the most recent FOFSE_E_CUDA of this thread
thread_local int g_last_cuda = 0;
fofse_status cuda_fail(cudaError_t e) {
  g_last_cuda = static_cast<int>(e);
  return FOFSE_E_CUDA;
}

constexpr int kMaxPlans = 64;
constexpr size_t kCounterBytes = 256;  // one int work-queue counter per plan

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Backward workspace: abar (n x imax float2), W0bar (n floats), then the
// FP64 d/drho accumulators (n x 4) and the finished-CTA counters (n), the
// last two contiguous so that one memset clears them.
struct BwdLayout {
  size_t abar, w0bar, acc, cnt, total, clear;
  BwdLayout(int n, int imax) {
    abar = 0;
    w0bar = align256((size_t)n * imax * sizeof(float2));
    acc = w0bar + align256((size_t)n * sizeof(float));
    cnt = acc + align256((size_t)n * 4 * sizeof(double));
    total = cnt + align256((size_t)n * sizeof(unsigned));
    clear = total - acc;
  }
};

// Device-side (rho, gamma): per plan, the three weight tables rebuilt for the
// call (and, for a DCT plan of fft_size 32 or 64, its complete-support table
// C for the call's rho) sit at the start of the workspace, before the forward
// or backward part.
size_t override_plan_bytes(const PlanDev& d) {
  const size_t N = (size_t)d.Ls * d.Ls;
  size_t b = align256(N * sizeof(float2)) + align256(N * sizeof(double)) + align256(N * sizeof(float));
  if (d.basis == FOFSE_BASIS_DCT && (d.T == 32 || d.T == 64))
    b += align256(dct_table_elems(d.T) * sizeof(float2));
  return b;
}
size_t override_bytes(const fofse_plan* plans, int n_plans) {
  size_t b = 0;
  for (int i = 0; i < n_plans; ++i) b += override_plan_bytes(plans[i]->dev);
  return b;
}

// Points plan `pi`'s weight tables at its part of the override region and
// queues their rebuild from d_rho_gamma[2 pi], [2 pi + 1] on `s`.
cudaError_t apply_override(const fofse_plan* plans, int pi, const float* d_rho_gamma,
                           unsigned char* region, unsigned* err, PlanDev& P, cudaStream_t s) {
  size_t off = 0;
  for (int i = 0; i < pi; ++i) off += override_plan_bytes(plans[i]->dev);
  const size_t N = (size_t)P.Ls * P.Ls;
  float2* wff = reinterpret_cast<float2*>(region + off);
  double* w64 = reinterpret_cast<double*>(region + off + align256(N * sizeof(float2)));
  float* w32 = reinterpret_cast<float*>(region + off + align256(N * sizeof(float2)) +
                                        align256(N * sizeof(double)));
  const float* rg = d_rho_gamma + 2 * pi;
  cudaError_t e = launch_plan_weights(P, rg, wff, w64, w32, err, s);
  P.tab.w_ff = wff;
  P.tab.w_f64 = w64;
  P.tab.w_f32 = w32;
  P.tab.dct_c_full = nullptr;  // the plan's own table is for its own rho
  P.rho_gamma_dev = rg;
  if (e == cudaSuccess && P.basis == FOFSE_BASIS_DCT && (P.T == 32 || P.T == 64)) {
    // the complete-support table for this call's rho, by the plan's build
    float2* tab = reinterpret_cast<float2*>(region + off + align256(N * sizeof(float2)) +
                                            align256(N * sizeof(double)) + align256(N * sizeof(float)));
    e = build_dct_table(P, tab, s);
    if (e == cudaSuccess) P.tab.dct_c_full = tab;
  }
  return e;
}

// Plans run one after another on the stream and share one scratch region.
size_t scratch_bytes(const fofse_plan* plans, int n_plans) {
  size_t m = 0;
  for (int i = 0; i < n_plans; ++i) {
    const size_t b = forward_scratch_bytes(plans[i]->dev);
    m = b > m ? b : m;
  }
  return (m + 255) & ~size_t(255);
}

}  // namespace

extern "C" {

const char* fofse_status_string(fofse_status s) {
  switch (s) {
    case FOFSE_OK: return "ok";
    case FOFSE_E_ARG: return "invalid argument";
    case FOFSE_E_UNSUPPORTED: return "unsupported configuration";
    case FOFSE_E_NOMEM: return "out of device memory";
    case FOFSE_E_CUDA: return "CUDA error";
    case FOFSE_E_TIMEOUT: return "device wait timed out";
    case FOFSE_E_STATE: return "call out of order";
  }
  return "unknown status";
}

int fofse_version(void) { return 100; }

fofse_status fofse_plan_create(int block, int border, int fft_size, float rho, float gamma,
                               int iters, fofse_plan* out) {
  if (!out) return FOFSE_E_ARG;
  if (block < 1 || border < 0 || iters < 1 || iters > kMaxIters) return FOFSE_E_ARG;
  if (!(rho > 0.f && rho <= 1.f) || !(gamma > 0.f && gamma <= 1.f)) return FOFSE_E_ARG;
  if (fft_size < 2 || (fft_size & (fft_size - 1)) != 0) return FOFSE_E_ARG;
  const int Ls = block + 2 * border;
  if (fft_size < Ls) return FOFSE_E_ARG;
  if (!supported_T(fft_size)) return FOFSE_E_UNSUPPORTED;
  const int T = fft_size;
  const int N = Ls * Ls;

  // distances to the centre of B in FP64 (Eq. 15); the weights rho^dist are
  // built from them on the device (the same kernel rebuilds them for a call
  // that passes rho and gamma in device memory)
  std::vector<double> dist(N);
  const double c = border + (block - 1) / 2.0;
  for (int m = 0; m < Ls; ++m)
    for (int n = 0; n < Ls; ++n)
      dist[m * Ls + n] = std::sqrt((m - c) * (m - c) + (n - c) * (n - c));
  std::vector<float4> tw_ff(T / 2);
  std::vector<double2> tw_f64(T / 2);
  std::vector<float2> tw_f32(T / 2);
  for (int e = 0; e < T / 2; ++e) {  // exp(-j 2 pi e / T), integer phase
    const double cr = std::cos(kTwoPi * e / T), ci = -std::sin(kTwoPi * e / T);
    const float hr = (float)cr, hi = (float)ci;
    tw_ff[e] = make_float4(hr, hi, (float)(cr - hr), (float)(ci - hi));
    tw_f64[e] = make_double2(cr, ci);
    tw_f32[e] = make_float2(hr, hi);
  }
  std::vector<float2> syn_f32(T);
  std::vector<double2> syn_f64(T);
  std::vector<float4> syn_ff(T);
  std::vector<float2> dct_cos(4 * T);
  for (int p = 0; p < 4 * T; ++p) {  // cos(2 pi p / (4T)), integer phase
    const double v = std::cos(kTwoPi * p / (4.0 * T));
    const float h = (float)v;
    dct_cos[p] = make_float2(h, (float)(v - (double)h));
  }
  for (int p = 0; p < T; ++p) {
    const double cr = std::cos(kTwoPi * p / T), ci = std::sin(kTwoPi * p / T);
    const float hr = (float)cr, hi = (float)ci;
    syn_f32[p] = make_float2(hr, hi);
    syn_f64[p] = make_double2(cr, ci);
    syn_ff[p] = make_float4(hr, hi, (float)(cr - hr), (float)(ci - hi));
  }

  // one allocation, 256-byte aligned sections
  size_t off = 0;
  auto sec = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_wff = sec(sizeof(float2) * N), o_w64 = sec(sizeof(double) * N),
               o_w32 = sec(sizeof(float) * N), o_tff = sec(sizeof(float4) * (T / 2)),
               o_t64 = sec(sizeof(double2) * (T / 2)), o_t32 = sec(sizeof(float2) * (T / 2)),
               o_s32 = sec(sizeof(float2) * T), o_s64 = sec(sizeof(double2) * T),
               o_sff = sec(sizeof(float4) * T), o_dist = sec(sizeof(double) * N),
               o_dcos = sec(sizeof(float2) * 4 * T),
               o_rg = sec(sizeof(float2));
  const size_t total = off;
  std::vector<unsigned char> host(total, 0);
  std::memcpy(&host[o_dist], dist.data(), sizeof(double) * N);
  std::memcpy(&host[o_dcos], dct_cos.data(), sizeof(float2) * 4 * T);
  const float2 rg = make_float2(rho, gamma);
  std::memcpy(&host[o_rg], &rg, sizeof(float2));
  std::memcpy(&host[o_tff], tw_ff.data(), sizeof(float4) * (T / 2));
  std::memcpy(&host[o_t64], tw_f64.data(), sizeof(double2) * (T / 2));
  std::memcpy(&host[o_t32], tw_f32.data(), sizeof(float2) * (T / 2));
  std::memcpy(&host[o_s32], syn_f32.data(), sizeof(float2) * T);
  std::memcpy(&host[o_s64], syn_f64.data(), sizeof(double2) * T);
  std::memcpy(&host[o_sff], syn_ff.data(), sizeof(float4) * T);

  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, total);
  if (e == cudaErrorMemoryAllocation) return FOFSE_E_NOMEM;
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpy(mem, host.data(), total, cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(mem);
    return cuda_fail(e);
  }
  fofse_plan p = new (std::nothrow) fofse_plan_s;
  if (!p) {
    cudaFree(mem);
    return FOFSE_E_NOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(mem);
  PlanDev& d = p->dev;
  d.block = block;
  d.border = border;
  d.Ls = Ls;
  d.T = T;
  d.iters = iters;
  d.support = FOFSE_SUPPORT_FULL;
  d.precision = FOFSE_FP32;
  d.variant = 0;
  d.compensation = FOFSE_COMP_CONSTANT;
  d.basis = FOFSE_BASIS_DFT;
  d.rho = rho;
  d.gamma = (double)gamma;
  d.gamma_h = gamma;
  d.gamma_l = 0.f;
  d.tab.w_ff = reinterpret_cast<const float2*>(base + o_wff);
  d.tab.w_f64 = reinterpret_cast<const double*>(base + o_w64);
  d.tab.w_f32 = reinterpret_cast<const float*>(base + o_w32);
  d.tab.tw_ff = reinterpret_cast<const float4*>(base + o_tff);
  d.tab.tw_f64 = reinterpret_cast<const double2*>(base + o_t64);
  d.tab.tw_f32 = reinterpret_cast<const float2*>(base + o_t32);
  d.tab.syn_f32 = reinterpret_cast<const float2*>(base + o_s32);
  d.tab.syn_f64 = reinterpret_cast<const double2*>(base + o_s64);
  d.tab.syn_ff = reinterpret_cast<const float4*>(base + o_sff);
  d.tab.dist = reinterpret_cast<const double*>(base + o_dist);
  d.tab.dct_cos_ff = reinterpret_cast<const float2*>(base + o_dcos);
  d.tab.dct_c_full = nullptr;
  d.rho_gamma_dev = nullptr;
  {
    unsigned* err = err_word_ptr();
    cudaError_t e2 = err ? cudaSuccess : cudaGetLastError();
    if (e2 == cudaSuccess)
      e2 = launch_plan_weights(d, reinterpret_cast<const float*>(base + o_rg),
                               reinterpret_cast<float2*>(base + o_wff),
                               reinterpret_cast<double*>(base + o_w64),
                               reinterpret_cast<float*>(base + o_w32), err, 0);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(0);
    if (e2 != cudaSuccess) {
      cudaFree(mem);
      delete p;
      return cuda_fail(e2);
    }
  }
  p->mem = mem;
  p->dct_mem = nullptr;
  cudaGetDevice(&p->device);
  *out = p;
  return FOFSE_OK;
}

namespace {
// (Re)builds the DCT basis' complete-support table of a DCT plan (fft_size 32
// or 64) for its current support shape; synchronous.  On failure the plan
// keeps no table (its blocks then build C themselves) and the error is
// returned.
fofse_status refresh_dct_table(fofse_plan plan) {
  PlanDev& d = plan->dev;
  d.tab.dct_c_full = nullptr;
  if (d.basis != FOFSE_BASIS_DCT || (d.T != 32 && d.T != 64)) return FOFSE_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return FOFSE_E_ARG;
  cudaError_t e = cudaSuccess;
  if (!plan->dct_mem) {
    e = cudaMalloc(&plan->dct_mem, sizeof(float2) * dct_table_elems(d.T));
    if (e != cudaSuccess) {
      plan->dct_mem = nullptr;
      return e == cudaErrorMemoryAllocation ? FOFSE_E_NOMEM : cuda_fail(e);
    }
  }
  e = build_dct_table(d, static_cast<float2*>(plan->dct_mem), 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return cuda_fail(e);
  d.tab.dct_c_full = static_cast<const float2*>(plan->dct_mem);
  return FOFSE_OK;
}
}  // namespace

fofse_status fofse_plan_set_support(fofse_plan plan, int shape) {
  if (!plan || (shape != FOFSE_SUPPORT_FULL && shape != FOFSE_SUPPORT_CAUSAL_L)) return FOFSE_E_ARG;
  plan->dev.support = shape;
  return refresh_dct_table(plan);
}

fofse_status fofse_plan_set_compensation(fofse_plan plan, int compensation) {
  if (!plan || (compensation != FOFSE_COMP_CONSTANT && compensation != FOFSE_COMP_OFSE))
    return FOFSE_E_ARG;
  plan->dev.compensation = compensation;
  if (plan->dev.variant >= forward_variant_count(plan->dev)) plan->dev.variant = 0;
  return FOFSE_OK;
}

fofse_status fofse_plan_set_basis(fofse_plan plan, int basis) {
  if (!plan || (basis != FOFSE_BASIS_DFT && basis != FOFSE_BASIS_DCT)) return FOFSE_E_ARG;
  plan->dev.basis = basis;
  if (plan->dev.variant >= forward_variant_count(plan->dev)) plan->dev.variant = 0;
  return refresh_dct_table(plan);
}

fofse_status fofse_plan_set_precision(fofse_plan plan, int precision) {
  if (!plan || (precision != FOFSE_FP32 && precision != FOFSE_FP64_VALIDATE &&
                precision != FOFSE_FP32_FULLFF))
    return FOFSE_E_ARG;
  plan->dev.precision = precision;
  if (plan->dev.variant >= forward_variant_count(plan->dev)) plan->dev.variant = 0;
  return FOFSE_OK;
}

int fofse_plan_variant_count(fofse_plan plan) {
  return plan ? forward_variant_count(plan->dev) : 0;
}

fofse_status fofse_plan_set_variant(fofse_plan plan, int variant) {
  if (!plan || variant < 0 || variant >= forward_variant_count(plan->dev)) return FOFSE_E_ARG;
  plan->dev.variant = variant;
  return FOFSE_OK;
}

fofse_status fofse_plan_get_shape(fofse_plan plan, int* block, int* border, int* fft_size,
                                  int* iters) {
  if (!plan) return FOFSE_E_ARG;
  if (block) *block = plan->dev.block;
  if (border) *border = plan->dev.border;
  if (fft_size) *fft_size = plan->dev.T;
  if (iters) *iters = plan->dev.iters;
  return FOFSE_OK;
}

void fofse_plan_destroy(fofse_plan plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  cudaFree(plan->mem);
  if (plan->dct_mem) cudaFree(plan->dct_mem);
  delete plan;
}

size_t fofse_workspace_bytes(const fofse_plan* plans, int n_plans, int n_blocks) {
  if (!plans || n_plans < 1 || n_plans > kMaxPlans || n_blocks < 0) return 0;
  int imax = 0;
  for (int i = 0; i < n_plans; ++i) {
    if (!plans[i]) return 0;
    imax = plans[i]->dev.iters > imax ? plans[i]->dev.iters : imax;
  }
  const size_t fwd = kCounterBytes + scratch_bytes(plans, n_plans);
  const size_t bwd = BwdLayout(n_blocks, imax).total;
  return override_bytes(plans, n_plans) + (fwd > bwd ? fwd : bwd);
}

fofse_status fofse_extrapolate_batch(const fofse_plan* plans, int n_plans,
                                     const fofse_block* d_blocks, int n_blocks,
                                     const float* d_frame, const uint8_t* d_avail, int height,
                                     int width, int pitch, const float* d_rho_gamma,
                                     float* d_out_frame, float* d_out_blocks,
                                     fofse_trace_entry* d_trace, float* d_w0,
                                     int32_t* d_block_status, void* d_workspace, void* stream) {
  return fofse_extrapolate_batch_gamma(plans, n_plans, d_blocks, n_blocks, d_frame, d_avail,
                                       height, width, pitch, d_rho_gamma, d_out_frame,
                                       d_out_blocks, d_trace, d_w0, d_block_status, nullptr,
                                       d_workspace, stream);
}

fofse_status fofse_extrapolate_batch_gamma(const fofse_plan* plans, int n_plans,
                                           const fofse_block* d_blocks, int n_blocks,
                                           const float* d_frame, const uint8_t* d_avail,
                                           int height, int width, int pitch,
                                           const float* d_rho_gamma, float* d_out_frame,
                                           float* d_out_blocks, fofse_trace_entry* d_trace,
                                           float* d_w0, int32_t* d_block_status,
                                           float* d_gamma, void* d_workspace, void* stream) {
  if (!plans || n_plans < 1 || n_plans > kMaxPlans || n_blocks < 0) return FOFSE_E_ARG;
  if (n_blocks > 0 && (!d_blocks || !d_frame || !d_avail)) return FOFSE_E_ARG;
  if (height < 1 || width < 1 || pitch < width) return FOFSE_E_ARG;
  if (d_rho_gamma && !d_workspace) return FOFSE_E_ARG;  // the rebuilt weights live there
  if (!plans_on_current_device(plans, n_plans)) return FOFSE_E_ARG;
  int bmax = 0, imax = 0;
  for (int i = 0; i < n_plans; ++i) {
    if (plans[i]->dev.precision != plans[0]->dev.precision) return FOFSE_E_ARG;
    bmax = plans[i]->dev.block > bmax ? plans[i]->dev.block : bmax;
    imax = plans[i]->dev.iters > imax ? plans[i]->dev.iters : imax;
  }
  // OFSE and the per-iteration factors exist only in the register-blocked
  // FOFSE_FP32 kernel, which needs the workspace
  for (int i = 0; i < n_plans; ++i) {
    const PlanDev& q = plans[i]->dev;
    const bool needs_f3 = d_gamma || q.compensation == FOFSE_COMP_OFSE;
    if (needs_f3 && (q.precision != FOFSE_FP32 || !d_workspace)) return FOFSE_E_UNSUPPORTED;
    if (!dct_supported(q)) return FOFSE_E_UNSUPPORTED;
  }
  if (n_blocks == 0) return FOFSE_OK;
  unsigned* err = err_word_ptr();
  if (!err) return cuda_fail(cudaGetLastError());
  const size_t scratch = scratch_bytes(plans, n_plans);
  for (int i = 0; i < n_plans; ++i)  // T = 128 needs its FFT scratch
    if (forward_needs_scratch(plans[i]->dev) && !d_workspace) return FOFSE_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* queue = nullptr;
  unsigned char* scratch_base = nullptr;
  unsigned char* region = static_cast<unsigned char*>(d_workspace);
  if (d_workspace) {
    unsigned char* fw = region + override_bytes(plans, n_plans);
    queue = reinterpret_cast<int*>(fw);
    scratch_base = fw + kCounterBytes;
    const cudaError_t e = cudaMemsetAsync(queue, 0, kCounterBytes, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }

  const uintptr_t fa = reinterpret_cast<uintptr_t>(d_frame), aa = reinterpret_cast<uintptr_t>(d_avail);
  const bool tma_ok = encode_fn() && (fa % 16 == 0) && (aa % 16 == 0) && (pitch % 16 == 0);
  // largest blocks first (longest-processing-time order across plans)
  int order[kMaxPlans];
  for (int i = 0; i < n_plans; ++i) order[i] = i;
  for (int i = 1; i < n_plans; ++i)
    for (int j = i; j > 0; --j) {
      const PlanDev& a = plans[order[j]]->dev;
      const PlanDev& b = plans[order[j - 1]]->dev;
      if ((double)a.iters * a.T * a.T <= (double)b.iters * b.T * b.T) break;
      const int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  for (int oi = 0; oi < n_plans; ++oi) {
    const int pi = order[oi];
    const PlanDev& P = plans[pi]->dev;
    FwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.plan = P;
    a.plan_index = pi;
    a.blocks = d_blocks;
    a.n_blocks = n_blocks;
    a.frame = d_frame;
    a.avail = d_avail;
    a.height = height;
    a.width = width;
    a.pitch = pitch;
    a.out_frame = d_out_frame;
    a.out_blocks = d_out_blocks;
    a.out_stride = bmax * bmax;
    a.out_ld = bmax;
    a.trace = d_trace;
    a.trace_stride = imax;
    a.w0 = d_w0;
    a.status = d_block_status;
    a.err = err;
    a.queue = queue ? queue + pi : nullptr;
    a.scratch = scratch_base;
    a.scratch_bytes = scratch_base ? scratch : 0;
    a.gamma_out = reinterpret_cast<float2*>(d_gamma);
    if (d_rho_gamma) {
      const cudaError_t eo = apply_override(plans, pi, d_rho_gamma, region, err, a.plan, s);
      if (eo != cudaSuccess) return cuda_fail(eo);
    }
    a.box_f = round_up(P.Ls + 3, 4);
    a.box_a = round_up(P.Ls + 15, 16);
    CUtensorMap tf, ta;
    std::memset(&tf, 0, sizeof(tf));
    std::memset(&ta, 0, sizeof(ta));
    a.use_tma = 0;
    if (tma_ok && a.box_f <= 256 && a.box_a <= 256 && P.Ls <= 256 &&
        encode_2d(&tf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d_frame, width, height, pitch, a.box_f,
                  P.Ls) &&
        encode_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d_avail, width, height, pitch, a.box_a,
                  P.Ls))
      a.use_tma = 1;
    cudaError_t e = launch_forward(a, &tf, &ta, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return FOFSE_OK;
}

// fofse_extrapolate_batch without a workspace: see include/fofse.h.  The
// work-queue counters come from the library's fixed device array instead of
// the caller's workspace, and with no scratch for the exact spectra
// FOFSE_FP32 plans run the all-bins float-float kernel (the plan's launch
// shape variant is ignored); DCT and FP64-validation plans run their usual
// kernels.  Nothing here allocates or frees device memory.
fofse_status fofse_extrapolate_batch_noalloc(const fofse_plan* plans, int n_plans,
                                             const fofse_block* d_blocks, int n_blocks,
                                             const float* d_frame, const uint8_t* d_avail,
                                             int height, int width, int pitch,
                                             float* d_out_frame, float* d_out_blocks,
                                             fofse_trace_entry* d_trace, float* d_w0,
                                             int32_t* d_block_status, void* stream) {
  if (!plans || n_plans < 1 || n_blocks < 0) return FOFSE_E_ARG;
  if (n_plans > kNoAllocCounters) return FOFSE_E_ARG;  // one counter per plan in the fixed array
  if (n_blocks > 0 && (!d_blocks || !d_frame || !d_avail)) return FOFSE_E_ARG;
  if (height < 1 || width < 1 || pitch < width) return FOFSE_E_ARG;
  if (!plans_on_current_device(plans, n_plans)) return FOFSE_E_ARG;
  int bmax = 0, imax = 0;
  for (int i = 0; i < n_plans; ++i) {
    if (plans[i]->dev.precision != plans[0]->dev.precision) return FOFSE_E_ARG;
    // a 128 x 128 FFT needs 256 KB of scratch per SM, beyond the fixed array;
    // OFSE needs the scratch of the register-blocked kernel
    if (forward_needs_scratch(plans[i]->dev)) return FOFSE_E_UNSUPPORTED;
    if (plans[i]->dev.compensation == FOFSE_COMP_OFSE) return FOFSE_E_UNSUPPORTED;
    if (!dct_supported(plans[i]->dev)) return FOFSE_E_UNSUPPORTED;
    bmax = plans[i]->dev.block > bmax ? plans[i]->dev.block : bmax;
    imax = plans[i]->dev.iters > imax ? plans[i]->dev.iters : imax;
  }
  if (n_blocks == 0) return FOFSE_OK;
  unsigned* err = err_word_ptr();
  int* queue = noalloc_queue_ptr();
  if (!err || !queue) return cuda_fail(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the counters keep the previous call's values: clear them on this stream
  cudaError_t e0 = cudaMemsetAsync(queue, 0, sizeof(int) * kNoAllocCounters, s);
  if (e0 != cudaSuccess) return cuda_fail(e0);
  const uintptr_t fa = reinterpret_cast<uintptr_t>(d_frame), aa = reinterpret_cast<uintptr_t>(d_avail);
  const bool tma_ok = encode_fn() && (fa % 16 == 0) && (aa % 16 == 0) && (pitch % 16 == 0);
  for (int pi = 0; pi < n_plans; ++pi) {
    const PlanDev& P = plans[pi]->dev;
    FwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.plan = P;
    a.plan_index = pi;
    a.blocks = d_blocks;
    a.n_blocks = n_blocks;
    a.frame = d_frame;
    a.avail = d_avail;
    a.height = height;
    a.width = width;
    a.pitch = pitch;
    a.out_frame = d_out_frame;
    a.out_blocks = d_out_blocks;
    a.out_stride = bmax * bmax;
    a.out_ld = bmax;
    a.trace = d_trace;
    a.trace_stride = imax;
    a.w0 = d_w0;
    a.status = d_block_status;
    a.err = err;
    a.queue = queue + pi;
    a.scratch = nullptr;  // FOFSE_FP32 then runs every bin in float-float (no scratch)
    a.scratch_bytes = 0;
    a.box_f = round_up(P.Ls + 3, 4);
    a.box_a = round_up(P.Ls + 15, 16);
    CUtensorMap tf, ta;
    std::memset(&tf, 0, sizeof(tf));
    std::memset(&ta, 0, sizeof(ta));
    a.use_tma = 0;
    if (tma_ok && a.box_f <= 256 && a.box_a <= 256 && P.Ls <= 256 &&
        encode_2d(&tf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d_frame, width, height, pitch, a.box_f,
                  P.Ls) &&
        encode_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d_avail, width, height, pitch, a.box_a,
                  P.Ls))
      a.use_tma = 1;
    const cudaError_t e = launch_forward(a, &tf, &ta, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return FOFSE_OK;
}

fofse_status fofse_error_curve(const fofse_plan* plans, int n_plans, const fofse_block* d_blocks,
                               int n_blocks, const fofse_trace_entry* d_trace,
                               const float* d_truth, int height, int width, int pitch,
                               float* d_sse, void* stream) {
  if (!plans || n_plans < 1 || n_plans > kMaxPlans || n_blocks < 0) return FOFSE_E_ARG;
  if (n_blocks > 0 && (!d_blocks || !d_trace || !d_truth || !d_sse)) return FOFSE_E_ARG;
  if (height < 1 || width < 1 || pitch < width) return FOFSE_E_ARG;
  if (!plans_on_current_device(plans, n_plans)) return FOFSE_E_ARG;
  int imax = 0;
  for (int i = 0; i < n_plans; ++i) {
    if (plans[i]->dev.block > 32) return FOFSE_E_UNSUPPORTED;
    imax = plans[i]->dev.iters > imax ? plans[i]->dev.iters : imax;
  }
  if (n_blocks == 0) return FOFSE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int pi = 0; pi < n_plans; ++pi) {
    CurveArgs a;
    std::memset(&a, 0, sizeof(a));
    a.plan = plans[pi]->dev;
    a.plan_index = pi;
    a.blocks = d_blocks;
    a.n_blocks = n_blocks;
    a.trace = d_trace;
    a.trace_stride = imax;
    a.truth = d_truth;
    a.height = height;
    a.width = width;
    a.pitch = pitch;
    a.sse = d_sse;
    const cudaError_t e = launch_error_curve(a, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return FOFSE_OK;
}

fofse_status fofse_backward(const fofse_plan* plans, int n_plans, const fofse_block* d_blocks,
                            int n_blocks, const float* d_frame, const uint8_t* d_avail,
                            int height, int width, int pitch, const float* d_rho_gamma,
                            const fofse_trace_entry* d_trace, const float* d_w0,
                            const float* d_grad_blocks, float* d_grad_frame,
                            float* d_grad_rho_gamma, void* d_workspace, void* stream) {
  if (!plans || n_plans < 1 || n_plans > kMaxPlans || n_blocks < 0) return FOFSE_E_ARG;
  if (n_blocks > 0 && (!d_blocks || !d_frame || !d_avail || !d_trace || !d_w0 || !d_grad_blocks))
    return FOFSE_E_ARG;
  if (height < 1 || width < 1 || pitch < width) return FOFSE_E_ARG;
  if (d_rho_gamma && !d_workspace) return FOFSE_E_ARG;
  if (!plans_on_current_device(plans, n_plans)) return FOFSE_E_ARG;
  int bmax = 0, imax = 0;
  for (int i = 0; i < n_plans; ++i) {
    if (plans[i]->dev.precision == FOFSE_FP64_VALIDATE) return FOFSE_E_UNSUPPORTED;
    if (plans[i]->dev.compensation == FOFSE_COMP_OFSE) return FOFSE_E_UNSUPPORTED;
    if (!dct_supported(plans[i]->dev)) return FOFSE_E_UNSUPPORTED;
    bmax = plans[i]->dev.block > bmax ? plans[i]->dev.block : bmax;
    imax = plans[i]->dev.iters > imax ? plans[i]->dev.iters : imax;
  }
  if (n_blocks == 0 || (!d_grad_frame && !d_grad_rho_gamma)) return FOFSE_OK;
  unsigned* err = err_word_ptr();
  if (!err) return cuda_fail(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const BwdLayout L(n_blocks, imax);
  unsigned char* region = static_cast<unsigned char*>(d_workspace);
  unsigned char* ws = region ? region + override_bytes(plans, n_plans) : nullptr;
  if (ws) {
    const cudaError_t e = cudaMemsetAsync(ws + L.acc, 0, L.clear, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  for (int pi = 0; pi < n_plans; ++pi) {
    BwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.plan = plans[pi]->dev;
    a.plan_index = pi;
    a.blocks = d_blocks;
    a.n_blocks = n_blocks;
    a.frame = d_frame;
    a.avail = d_avail;
    a.height = height;
    a.width = width;
    a.pitch = pitch;
    a.trace = d_trace;
    a.trace_stride = imax;
    a.w0 = d_w0;
    a.grad_blocks = d_grad_blocks;
    a.grad_stride = bmax * bmax;
    a.grad_ld = bmax;
    a.grad_frame = d_grad_frame;
    a.grad_rho_gamma = d_grad_rho_gamma ? d_grad_rho_gamma + 2 * pi : nullptr;
    a.err = err;
    if (d_rho_gamma) {
      const cudaError_t eo = apply_override(plans, pi, d_rho_gamma, region, err, a.plan, s);
      if (eo != cudaSuccess) return cuda_fail(eo);
    }
    if (ws) {
      a.abar = reinterpret_cast<float2*>(ws + L.abar);
      a.w0bar = reinterpret_cast<float*>(ws + L.w0bar);
      a.acc = reinterpret_cast<double*>(ws + L.acc);
      a.cnt = reinterpret_cast<unsigned*>(ws + L.cnt);
    }
    cudaError_t e = launch_backward(a, s);
    if (e == cudaErrorNotSupported) return FOFSE_E_UNSUPPORTED;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return FOFSE_OK;
}

int fofse_last_cuda_error(void) { return g_last_cuda; }

const char* fofse_last_cuda_error_string(void) { return cudaGetErrorName(static_cast<cudaError_t>(g_last_cuda)); }

fofse_status fofse_check(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned* err = err_word_ptr();
  if (!err) return cuda_fail(cudaGetLastError());
  unsigned v = 0;
  if ((e = cudaMemcpy(&v, err, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
  if (v) {
    unsigned z = 0;
    if ((e = cudaMemcpy(err, &z, sizeof(z), cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_fail(e);
  }
  if (v & kErrTimeout) return FOFSE_E_TIMEOUT;
  if (v & kErrParam) return FOFSE_E_ARG;
  return FOFSE_OK;
}

}  // extern "C"

namespace fofse {
// FOFSE_E_CUDA for `e`, remembered for fofse_last_cuda_error (used by the
// translation units outside this file)
fofse_status record_cuda_error(cudaError_t e) { return cuda_fail(e); }
}  // namespace fofse
