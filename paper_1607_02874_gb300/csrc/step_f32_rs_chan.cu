// Step kernels of the validation-channel variant with the random sputtering
// matrix, for one population storage type (a unit of its own so that it
// compiles in parallel with the others).
#include "step_impl.cuh"

namespace lbm {
LBM_INSTANTIATE_STEP(LBM_FP32, true, kPhysChannel)
}  // namespace lbm
