// Backward (adjoint) FOFSE kernel -- placeholder until the adjoint lands.
#include "fofse_internal.h"

namespace fofse {
cudaError_t launch_backward(const BwdArgs&, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace fofse
