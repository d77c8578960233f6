// Step kernel, state readers and export for one population storage type.
#include "step_impl.cuh"

namespace lbm {
LBM_INSTANTIATE_STORAGE(LBM_FP16_DEV)
}  // namespace lbm
