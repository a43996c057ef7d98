// rf_launch.h -- launch entry points of the tile kernels.  They are
// instantiated in four translation units (filter order 3 or 1, forward or
// adjoint: rf_tiles_*.cu) that compile in parallel; the planner sees only
// these declarations.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "rf_tile.cuh"

namespace rfvh {

// (lines per CTA, slices per thread) of a tile-kernel launch.
struct TileShape {
    int R, B;
};

// One domain: grid (line blocks) x (CTA rows along the slices).
template <int ORDER, bool ADJ>
void launch_shape(const TileArgs &a, TileShape sh, int64_t nlines, int64_t groups,
                  size_t smem, cudaStream_t st);

// Resident CTAs per SM of a shape (MULTI: the multi-domain kernel), after
// raising the kernel's shared-memory limit to smem; 0 if it cannot run.
template <int ORDER, bool ADJ, bool MULTI>
int shape_occupancy(TileShape sh, size_t smem);

// Many domains: persistent CTAs over the work list in m.
template <int ORDER, bool ADJ>
void launch_multi(const MultiArgs &m, TileShape sh, unsigned grid, size_t smem, cudaStream_t st);

#define RF_DECLARE(O, A)                                                                   \
    extern template void launch_shape<O, A>(const TileArgs &, TileShape, int64_t, int64_t, \
                                            size_t, cudaStream_t);                         \
    extern template int shape_occupancy<O, A, false>(TileShape, size_t);                   \
    extern template int shape_occupancy<O, A, true>(TileShape, size_t);                    \
    extern template void launch_multi<O, A>(const MultiArgs &, TileShape, unsigned, size_t, \
                                            cudaStream_t);
RF_DECLARE(3, false)
RF_DECLARE(3, true)
RF_DECLARE(1, false)
RF_DECLARE(1, true)
#undef RF_DECLARE

}  // namespace rfvh
