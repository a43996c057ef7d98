// Tile kernels of the order-3 filter, adjoint steps.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(3, true)
}  // namespace rfvh
