// Tile kernels of the order-1 filter, adjoint steps.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(1, true)
}  // namespace rfvh
