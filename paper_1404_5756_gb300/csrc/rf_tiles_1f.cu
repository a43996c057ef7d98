// Tile kernels of the order-1 filter, forward steps.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(1, false)
}  // namespace rfvh
