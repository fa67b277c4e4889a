// Register-blocked filtered-exact forward with OFSE's orthogonality deficiency
// compensation (Sec. 3, Eq. 10-13) instead of the constant factor of Eq. 14.
// The selection (Eq. 9) and the working spectrum are those of the product
// kernel (fofse_fwd3.cuh); each iteration adds the exact value of
// Q[u] = sum_l P[l] W[u - l] at the winner and takes c = P[u]^2 / Q[u].
// One launch shape per fft_size (the product kernel's default one).
#include "fofse_fwd3.cuh"

namespace fofse {
namespace {

template <int T> struct PickOfse;
template <> struct PickOfse<32> { using V = VariantF3<32, 32, 16, true>; };
template <> struct PickOfse<64> { using V = VariantF3<64, 64, 6, true>; };
template <> struct PickOfse<128> { using V = VariantF3<128, 256, 1, true>; };

template <int T> size_t scratch_ofse(int iters) {
  size_t b = 0;
  return PickOfse<T>::V::scratch(iters, &b) == cudaSuccess ? b : 0;
}

}  // namespace

cudaError_t launch_forward_ofse(const FwdArgs& a, const CUtensorMap* tf, const CUtensorMap* ta,
                                cudaStream_t s) {
  if (a.plan.T == 32) return PickOfse<32>::V::launch(a, tf, ta, s);
  if (a.plan.T == 64) return PickOfse<64>::V::launch(a, tf, ta, s);
  if (a.plan.T == 128) return PickOfse<128>::V::launch(a, tf, ta, s);
  return cudaErrorInvalidValue;
}

size_t forward_ofse_scratch_bytes(const PlanDev& p) {
  if (p.T == 32) return scratch_ofse<32>(p.iters);
  if (p.T == 64) return scratch_ofse<64>(p.iters);
  if (p.T == 128) return scratch_ofse<128>(p.iters);
  return 0;
}

}  // namespace fofse
