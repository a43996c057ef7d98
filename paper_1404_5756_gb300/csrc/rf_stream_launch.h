// rf_stream_launch.h -- launch entry point of the streaming column kernel
// (rf_stream.cuh), instantiated in rf_stream_3.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "rf_stream.cuh"

namespace rfvh {

constexpr int kStreamDepth = 10;  // rows read ahead

// Grid of a pass: (column blocks of 32, slice-pair blocks of kStreamWarps).
inline dim3 stream_grid(int64_t ncols, int64_t npairs)
{
    return dim3((unsigned)((ncols + 31) / 32), (unsigned)((npairs + kStreamWarps - 1) / kStreamWarps));
}

template <bool ADJ>
void stream_launch(const StreamArgs &a, cudaStream_t st);

// One pass over the m.nd domains of m as one grid of `grid` = m.cta0[m.nd]
// CTAs.
template <bool ADJ>
void stream_launch_multi(const StreamMulti &m, unsigned grid, cudaStream_t st);

extern template void stream_launch<false>(const StreamArgs &, cudaStream_t);
extern template void stream_launch<true>(const StreamArgs &, cudaStream_t);
extern template void stream_launch_multi<false>(const StreamMulti &, unsigned, cudaStream_t);
extern template void stream_launch_multi<true>(const StreamMulti &, unsigned, cudaStream_t);

}  // namespace rfvh
