// Register-resident kernel of the first-order filter with carried coasts,
// forward steps, y pass (columns).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(1, false, 1, true)
}  // namespace rfvh
