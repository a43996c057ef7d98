// Register-resident kernel of the third-order filter, adjoint (transposed) steps, y pass (columns).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(3, true, 1, false)
}  // namespace rfvh
