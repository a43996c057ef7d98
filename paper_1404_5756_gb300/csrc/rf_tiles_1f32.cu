// Tile kernels of the order-1 filter, forward steps, 32 lanes per line.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(1, false, 32, false)
}  // namespace rfvh
