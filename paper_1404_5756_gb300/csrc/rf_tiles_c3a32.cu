// Tile kernels of the order-3 filter, transposed steps, 32 lanes per line,
// constant-extension coasts.
#include "rf_launch_impl.cuh"

namespace rfvh {
RF_INSTANTIATE(3, true, 32, true)
}  // namespace rfvh
