// Register-resident kernel of the first-order filter, adjoint (transposed) steps, y pass (columns).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(1, true, 1, false)
}  // namespace rfvh
