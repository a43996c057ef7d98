// Register-resident kernel of the third-order filter, adjoint (transposed) steps, x pass (rows).
#include "rf_reg_impl.cuh"

namespace rfvh {
RF_REG_INSTANTIATE(3, true, 0, false)
}  // namespace rfvh
