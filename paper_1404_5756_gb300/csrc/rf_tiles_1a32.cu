// Tile kernels of the order-1 filter, adjoint steps, 32 lanes per line.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(1, true, 32, false)
}  // namespace rfvh
