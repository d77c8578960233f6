// Step kernels of the validation-channel variant (inert solid, body force,
// species relaxation time), for one population storage type (a unit of its
// own so that it compiles in parallel with the others).
#include "step_impl.cuh"

namespace lbm {
LBM_INSTANTIATE_STEP(LBM_BF16_DEV, false, kPhysChannel)
}  // namespace lbm
