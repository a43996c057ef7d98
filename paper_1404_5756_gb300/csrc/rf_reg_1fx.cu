// Register-resident kernel of the first-order filter, forward steps, x pass (rows).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(1, false, 0, false)
}  // namespace rfvh
