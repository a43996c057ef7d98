// Register-resident kernel of the first-order filter with carried coasts,
// transposed steps, x pass (rows).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(1, true, 0, true)
}  // namespace rfvh
