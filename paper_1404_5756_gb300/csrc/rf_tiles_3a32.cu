// Tile kernels of the order-3 filter, adjoint steps, 32 lanes per line.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(3, true, 32, false)
}  // namespace rfvh
