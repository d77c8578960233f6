// Step kernels with the random sputtering matrix, for one population storage
// type (a unit of its own so that it compiles in parallel with the others).
#include "step_impl.cuh"

namespace lbm {
LBM_INSTANTIATE_STEP(LBM_FP16_DEV, true, kPhysCarrier)
}  // namespace lbm
