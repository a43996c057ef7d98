// rf_launch.h -- launch entry points of the tile kernels.  They are
// instantiated in twelve translation units (rf_tiles_*.cu: filter order 3 or
// 1, forward or adjoint, 32 or 16 lanes per line -- 16 for order 3 only --,
// zero-input or constant-extension coasts) that compile in parallel; the
// planner sees only these declarations.
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

// The shapes the constant-extension kernels are built for (a short list: the
// option is not the default; kept in step with rf_launch_impl.cuh).
constexpr TileShape kCstShapes[] = {{8, 4, 32}, {4, 4, 32},  {2, 4, 32}, {1, 4, 32},
                                    {8, 1, 32}, {1, 1, 32},  {16, 4, 16}, {8, 4, 16},
                                    {8, 2, 16}, {8, 1, 16}};

inline bool cst_shape(TileShape sh)
{
    for (const TileShape &c : kCstShapes)
        if (c.R == sh.R && c.B == sh.B && c.P == sh.P) return true;
    return false;
}

// Launchers of the shapes with P lanes per line (one translation unit per
// filter order, direction, P and coast treatment).
template <int ORDER, bool ADJ, int P, bool CST>
void launch_shape_p(const TileArgs &a, TileShape sh, int64_t nlines, int64_t groups,
                    size_t smem, cudaStream_t st);
template <int ORDER, bool ADJ, bool MULTI, int P, bool CST>
int shape_occupancy_p(TileShape sh, size_t smem);
template <int ORDER, bool ADJ, int P, bool CST>
void launch_multi_p(const MultiArgs &m, TileShape sh, unsigned grid, size_t smem, cudaStream_t st);

#define RF_DECLARE(O, A, P, C)                                                                \
    extern template void launch_shape_p<O, A, P, C>(const TileArgs &, TileShape, int64_t,    \
                                                    int64_t, size_t, cudaStream_t);          \
    extern template int shape_occupancy_p<O, A, false, P, C>(TileShape, size_t);              \
    extern template int shape_occupancy_p<O, A, true, P, C>(TileShape, size_t);               \
    extern template void launch_multi_p<O, A, P, C>(const MultiArgs &, TileShape, unsigned,  \
                                                    size_t, cudaStream_t);
RF_DECLARE(3, false, 32, false)
RF_DECLARE(3, true, 32, false)
RF_DECLARE(3, false, 16, false)
RF_DECLARE(3, true, 16, false)
RF_DECLARE(1, false, 32, false)
RF_DECLARE(1, true, 32, false)
RF_DECLARE(3, false, 32, true)
RF_DECLARE(3, true, 32, true)
RF_DECLARE(3, false, 16, true)
RF_DECLARE(3, true, 16, true)
RF_DECLARE(1, false, 32, true)
RF_DECLARE(1, true, 32, true)
#undef RF_DECLARE

// One domain: grid (line blocks) x (CTA rows along the slices).  16 lanes
// per line exist for the third-order filter only; cst selects the
// constant-extension kernels.
template <int ORDER, bool ADJ>
inline void launch_shape(const TileArgs &a, TileShape sh, bool cst, int64_t nlines,
                         int64_t groups, size_t smem, cudaStream_t st)
{
    if constexpr (ORDER == 3)
        if (sh.P == 16) {
            if (cst) return launch_shape_p<ORDER, ADJ, 16, true>(a, sh, nlines, groups, smem, st);
            return launch_shape_p<ORDER, ADJ, 16, false>(a, sh, nlines, groups, smem, st);
        }
    if (sh.P != 32) return;
    if (cst) launch_shape_p<ORDER, ADJ, 32, true>(a, sh, nlines, groups, smem, st);
    else launch_shape_p<ORDER, ADJ, 32, false>(a, sh, nlines, groups, smem, st);
}

// Resident CTAs per SM of a shape (MULTI: the multi-domain kernel), after
// raising the kernel's shared-memory limit to smem; 0 if it cannot run or is
// not built.
template <int ORDER, bool ADJ, bool MULTI>
inline int shape_occupancy(TileShape sh, bool cst, size_t smem)
{
    if (cst && !cst_shape(sh)) return 0;
    if constexpr (ORDER == 3)
        if (sh.P == 16)
            return cst ? shape_occupancy_p<ORDER, ADJ, MULTI, 16, true>(sh, smem)
                       : shape_occupancy_p<ORDER, ADJ, MULTI, 16, false>(sh, smem);
    if (sh.P != 32) return 0;
    return cst ? shape_occupancy_p<ORDER, ADJ, MULTI, 32, true>(sh, smem)
               : shape_occupancy_p<ORDER, ADJ, MULTI, 32, false>(sh, smem);
}

// Many domains: persistent CTAs over the work list in m.
template <int ORDER, bool ADJ>
inline void launch_multi(const MultiArgs &m, TileShape sh, bool cst, unsigned grid, size_t smem,
                         cudaStream_t st)
{
    if constexpr (ORDER == 3)
        if (sh.P == 16) {
            if (cst) return launch_multi_p<ORDER, ADJ, 16, true>(m, sh, grid, smem, st);
            return launch_multi_p<ORDER, ADJ, 16, false>(m, sh, grid, smem, st);
        }
    if (sh.P != 32) return;
    if (cst) launch_multi_p<ORDER, ADJ, 32, true>(m, sh, grid, smem, st);
    else launch_multi_p<ORDER, ADJ, 32, false>(m, sh, grid, smem, st);
}

}  // namespace rfvh
