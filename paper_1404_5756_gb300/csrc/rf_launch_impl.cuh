// rf_launch_impl.cuh -- host-side launch code of the tile kernels (one
// domain and many domains).  Included by the translation units that
// instantiate it for one filter order, direction, lanes-per-line value and
// coast treatment each (rf_tiles_*.cu), so the kernels compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "rf_launch.h"
#include "rf_tile.cuh"

namespace rfvh {
namespace {

// The kernels of one shape: the constant-extension ones are separate
// templates (their own launch bounds).
template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
constexpr auto single_kernel()
{
    if constexpr (CST) return &tile_kernel_cst<ORDER, ADJ, R, B, P>;
    else return &tile_kernel<ORDER, ADJ, R, B, P, false>;
}

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
constexpr auto multi_kernel()
{
    if constexpr (CST) return &tile_multi_kernel_cst<ORDER, ADJ, R, B, P>;
    else return &tile_multi_kernel<ORDER, ADJ, R, B, P, false>;
}

// Raise a kernel's dynamic shared-memory limit once per device and size, so
// a launch inside a stream capture makes no attribute call.
constexpr int kAttrDevices = 64;
template <int ORDER, bool ADJ, int R, int B, int P, bool CST, bool MULTI>
void smem_attr(size_t smem)
{
    static std::mutex mu;
    static size_t done[kAttrDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < kAttrDevices && smem <= done[dev]) return;
    if (MULTI)
        cudaFuncSetAttribute(multi_kernel<ORDER, ADJ, R, B, P, CST>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        cudaFuncSetAttribute(single_kernel<ORDER, ADJ, R, B, P, CST>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < kAttrDevices) done[dev] = smem;
}

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
void launch_tile(const TileArgs &a, int64_t nlines, int64_t groups, size_t smem,
                 cudaStream_t st)
{
    smem_attr<ORDER, ADJ, R, B, P, CST, false>(smem);
    dim3 grid((unsigned)((nlines + R - 1) / R), (unsigned)groups);
    single_kernel<ORDER, ADJ, R, B, P, CST>()<<<grid, R * P, smem, st>>>(a);
}

template <int ORDER, bool ADJ, int R, int B, int P, bool CST, bool MULTI>
int tile_occupancy(size_t smem)
{
    smem_attr<ORDER, ADJ, R, B, P, CST, MULTI>(smem);
    int blocks = 0;
    cudaError_t e;
    if (MULTI)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, multi_kernel<ORDER, ADJ, R, B, P, CST>(), R * P, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, single_kernel<ORDER, ADJ, R, B, P, CST>(), R * P, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

template <int ORDER, bool ADJ, int R, int B, int P, bool CST>
void launch_multi_rb(const MultiArgs &m, unsigned grid, size_t smem, cudaStream_t st)
{
    smem_attr<ORDER, ADJ, R, B, P, CST, true>(smem);
    multi_kernel<ORDER, ADJ, R, B, P, CST>()<<<grid, R * P, smem, st>>>(m);
}

}  // namespace

// The shapes the tile kernel is built for (kept in step with the shape lists
// of the planner, kShapes* there and kCstShapes in rf_launch.h); each
// translation unit builds the shapes of one lanes-per-line value, of the
// zero-input coasts (the full list) or of the constant-extension coasts (a
// short list).
#define RF_FOR_EACH_SHAPE(X)                                                          \
    X(8, 4, 32) X(8, 2, 32) X(8, 1, 32) X(4, 4, 32) X(2, 4, 32) X(1, 4, 32) X(1, 1, 32) \
    X(1, 8, 32) X(2, 8, 32) X(4, 8, 32) X(8, 8, 32) X(16, 4, 32) X(16, 8, 32)          \
    X(4, 4, 16) X(8, 4, 16) X(16, 4, 16) X(8, 8, 16) X(16, 8, 16) X(8, 2, 16)          \
    X(16, 2, 16) X(8, 1, 16)
#define RF_FOR_EACH_CST_SHAPE(X)                                                      \
    X(8, 4, 32) X(4, 4, 32) X(2, 4, 32) X(1, 4, 32) X(8, 1, 32) X(1, 1, 32)            \
    X(16, 4, 16) X(8, 4, 16) X(8, 2, 16) X(8, 1, 16)

template <int ORDER, bool ADJ, int P, bool CST>
void launch_shape_p(const TileArgs &a, TileShape sh, int64_t nlines, int64_t groups,
                    size_t smem, cudaStream_t st)
{
#define RF_SHAPE(r, b, p)                                                        \
    if constexpr (p == P)                                                        \
        if (sh.R == r && sh.B == b) {                                            \
            launch_tile<ORDER, ADJ, r, b, p, CST>(a, nlines, groups, smem, st);  \
            return;                                                              \
        }
    if constexpr (CST) {
        RF_FOR_EACH_CST_SHAPE(RF_SHAPE)
    } else {
        RF_FOR_EACH_SHAPE(RF_SHAPE)
    }
#undef RF_SHAPE
}

template <int ORDER, bool ADJ, bool MULTI, int P, bool CST>
int shape_occupancy_p(TileShape sh, size_t smem)
{
#define RF_SHAPE(r, b, p)                                                        \
    if constexpr (p == P)                                                        \
        if (sh.R == r && sh.B == b) return tile_occupancy<ORDER, ADJ, r, b, p, CST, MULTI>(smem);
    if constexpr (CST) {
        RF_FOR_EACH_CST_SHAPE(RF_SHAPE)
    } else {
        RF_FOR_EACH_SHAPE(RF_SHAPE)
    }
#undef RF_SHAPE
    return 0;
}

template <int ORDER, bool ADJ, int P, bool CST>
void launch_multi_p(const MultiArgs &m, TileShape sh, unsigned grid, size_t smem, cudaStream_t st)
{
#define RF_SHAPE(r, b, p)                                                \
    if constexpr (p == P)                                                \
        if (sh.R == r && sh.B == b) {                                    \
            launch_multi_rb<ORDER, ADJ, r, b, p, CST>(m, grid, smem, st); \
            return;                                                      \
        }
    if constexpr (CST) {
        RF_FOR_EACH_CST_SHAPE(RF_SHAPE)
    } else {
        RF_FOR_EACH_SHAPE(RF_SHAPE)
    }
#undef RF_SHAPE
}

#undef RF_FOR_EACH_SHAPE
#undef RF_FOR_EACH_CST_SHAPE

#define RF_INSTANTIATE(O, A, P, CST)                                                         \
    template void launch_shape_p<O, A, P, CST>(const TileArgs &, TileShape, int64_t, int64_t, \
                                               size_t, cudaStream_t);                         \
    template int shape_occupancy_p<O, A, false, P, CST>(TileShape, size_t);                   \
    template int shape_occupancy_p<O, A, true, P, CST>(TileShape, size_t);                    \
    template void launch_multi_p<O, A, P, CST>(const MultiArgs &, TileShape, unsigned, size_t, \
                                               cudaStream_t);

}  // namespace rfvh
