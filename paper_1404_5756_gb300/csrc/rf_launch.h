// rf_launch.h -- launch entry points of the tile kernels.  They are
// instantiated in six translation units (rf_tiles_*.cu: filter order 3 or 1,
// forward or adjoint, 32 or 16 lanes per line, 16 lanes for order 3 only)
// that compile in parallel; the planner sees only these declarations.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "rf_tile.cuh"

namespace rfvh {

// (lines per CTA, slices per thread, lanes per line) of a tile-kernel
// launch; the lanes per line must match the direction's chunking.
struct TileShape {
    int R, B, P;
};

// Launchers of the shapes with P lanes per line (one translation unit per
// filter order, direction and P).
template <int ORDER, bool ADJ, int P>
void launch_shape_p(const TileArgs &a, TileShape sh, int64_t nlines, int64_t groups,
                    size_t smem, cudaStream_t st);
template <int ORDER, bool ADJ, bool MULTI, int P>
int shape_occupancy_p(TileShape sh, size_t smem);
template <int ORDER, bool ADJ, int P>
void launch_multi_p(const MultiArgs &m, TileShape sh, unsigned grid, size_t smem, cudaStream_t st);

#define RF_DECLARE(O, A, P)                                                                   \
    extern template void launch_shape_p<O, A, P>(const TileArgs &, TileShape, int64_t,       \
                                                 int64_t, size_t, cudaStream_t);             \
    extern template int shape_occupancy_p<O, A, false, P>(TileShape, size_t);                 \
    extern template int shape_occupancy_p<O, A, true, P>(TileShape, size_t);                  \
    extern template void launch_multi_p<O, A, P>(const MultiArgs &, TileShape, unsigned,     \
                                                 size_t, cudaStream_t);
RF_DECLARE(3, false, 32)
RF_DECLARE(3, true, 32)
RF_DECLARE(3, false, 16)
RF_DECLARE(3, true, 16)
RF_DECLARE(1, false, 32)
RF_DECLARE(1, true, 32)
#undef RF_DECLARE

// One domain: grid (line blocks) x (CTA rows along the slices).  16 lanes
// per line exist for the third-order filter only.
template <int ORDER, bool ADJ>
inline void launch_shape(const TileArgs &a, TileShape sh, int64_t nlines, int64_t groups,
                         size_t smem, cudaStream_t st)
{
    if constexpr (ORDER == 3)
        if (sh.P == 16) return launch_shape_p<ORDER, ADJ, 16>(a, sh, nlines, groups, smem, st);
    if (sh.P == 32) launch_shape_p<ORDER, ADJ, 32>(a, sh, nlines, groups, smem, st);
}

// Resident CTAs per SM of a shape (MULTI: the multi-domain kernel), after
// raising the kernel's shared-memory limit to smem; 0 if it cannot run.
template <int ORDER, bool ADJ, bool MULTI>
inline int shape_occupancy(TileShape sh, size_t smem)
{
    if constexpr (ORDER == 3)
        if (sh.P == 16) return shape_occupancy_p<ORDER, ADJ, MULTI, 16>(sh, smem);
    return sh.P == 32 ? shape_occupancy_p<ORDER, ADJ, MULTI, 32>(sh, smem) : 0;
}

// Many domains: persistent CTAs over the work list in m.
template <int ORDER, bool ADJ>
inline void launch_multi(const MultiArgs &m, TileShape sh, unsigned grid, size_t smem,
                         cudaStream_t st)
{
    if constexpr (ORDER == 3)
        if (sh.P == 16) return launch_multi_p<ORDER, ADJ, 16>(m, sh, grid, smem, st);
    if (sh.P == 32) launch_multi_p<ORDER, ADJ, 32>(m, sh, grid, smem, st);
}

}  // namespace rfvh
