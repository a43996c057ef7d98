// Register-resident kernel of the third-order filter, forward steps, y pass (columns).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(3, false, 1, false)
}  // namespace rfvh
