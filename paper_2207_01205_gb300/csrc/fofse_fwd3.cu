// Register-blocked filtered-exact forward with the constant compensation of
// Eq. 14 (the kernel itself is in fofse_fwd3.cuh).
#include "fofse_fwd3.cuh"

namespace fofse {
namespace {

// Launch shapes (threads per block, minimum resident blocks per SM that the
// register allocation is held to); variant 0 is the default, the autotuner
// may pick another per plan.  Fewer warps per block means less of the
// per-iteration work (top-2 merge, certainty test, coefficient) repeated per
// warp; the limit is the register file (2 registers per held bin): measured
// on the GB300, one warp per block is fastest at fft_size 32, two at 64 and
// eight at 128.
template <int T> struct PickF3;
template <> struct PickF3<32> {
  using V0 = VariantF3<32, 32, 16>;
  using V1 = VariantF3<32, 64, 12>;
  using V2 = VariantF3<32, 128, 6>;
  static constexpr int NV = 3;
};
template <> struct PickF3<64> {
  using V0 = VariantF3<64, 64, 6>;
  using V1 = VariantF3<64, 128, 6>;
  using V2 = VariantF3<64, 32, 6>;
  static constexpr int NV = 3;
};
template <> struct PickF3<128> {
  using V0 = VariantF3<128, 256, 1>;
  using V1 = VariantF3<128, 512, 1>;
  using V2 = VariantF3<128, 1024, 1>;
  static constexpr int NV = 3;
};

template <int T>
cudaError_t launch_T3(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta, cudaStream_t s) {
  using Pk = PickF3<T>;
  switch (a.plan.variant) {
    case 1: return Pk::V1::launch(a, tf, ta, s);
    case 2: return Pk::V2::launch(a, tf, ta, s);
    default: return Pk::V0::launch(a, tf, ta, s);
  }
}
template <int T> cudaError_t scratch_T3(int iters, size_t* bytes) {
  using Pk = PickF3<T>;
  size_t b0 = 0, b1 = 0, b2 = 0;
  cudaError_t e = Pk::V0::scratch(iters, &b0);
  if (e == cudaSuccess && Pk::NV > 1) e = Pk::V1::scratch(iters, &b1);
  if (e == cudaSuccess && Pk::NV > 2) e = Pk::V2::scratch(iters, &b2);
  *bytes = b0 > b1 ? (b0 > b2 ? b0 : b2) : (b1 > b2 ? b1 : b2);
  return e;
}

}  // namespace

cudaError_t launch_forward_f3(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta,
                              cudaStream_t s) {
  if (a.plan.compensation == FOFSE_COMP_OFSE) return launch_forward_ofse(a, tf, ta, s);
  if (a.plan.T == 32) return launch_T3<32>(a, tf, ta, s);
  if (a.plan.T == 64) return launch_T3<64>(a, tf, ta, s);
  if (a.plan.T == 128) return launch_T3<128>(a, tf, ta, s);
  return cudaErrorInvalidValue;
}

size_t forward_f3_scratch_bytes(const PlanDev& p) {
  if (p.compensation == FOFSE_COMP_OFSE) return forward_ofse_scratch_bytes(p);
  size_t b = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (p.T == 32) e = scratch_T3<32>(p.iters, &b);
  if (p.T == 64) e = scratch_T3<64>(p.iters, &b);
  if (p.T == 128) e = scratch_T3<128>(p.iters, &b);
  return e == cudaSuccess ? b : 0;
}

int forward_f3_variant_count(const PlanDev& p) {
  if (p.compensation == FOFSE_COMP_OFSE) return 1;
  if (p.T == 32) return PickF3<32>::NV;
  if (p.T == 64) return PickF3<64>::NV;
  if (p.T == 128) return PickF3<128>::NV;
  return 1;
}

}  // namespace fofse
