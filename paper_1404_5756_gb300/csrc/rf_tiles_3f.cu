// Tile kernels of the order-3 filter, forward steps.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(3, false)
}  // namespace rfvh
