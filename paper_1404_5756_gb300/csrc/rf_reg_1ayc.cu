// Register-resident kernel of the first-order filter with carried coasts,
// transposed steps, y pass (columns).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(1, true, 1, true)
}  // namespace rfvh
