// Streaming column kernel of the third-order filter, forward and transposed
// steps (y pass).
#include "rf_stream_launch.h"

namespace rfvh {

template <bool ADJ>
void stream_launch(const StreamArgs &a, cudaStream_t st)
{
    stream_kernel<ADJ, kStreamDepth><<<stream_grid(a.ncols, a.npairs), kStreamWarps * 32, 0, st>>>(a);
}

template <bool ADJ>
void stream_launch_multi(const StreamMulti &m, unsigned grid, cudaStream_t st)
{
    stream_multi_kernel<ADJ, kStreamDepth><<<grid, kStreamWarps * 32, 0, st>>>(m);
}

template void stream_launch<false>(const StreamArgs &, cudaStream_t);
template void stream_launch<true>(const StreamArgs &, cudaStream_t);
template void stream_launch_multi<false>(const StreamMulti &, unsigned, cudaStream_t);
template void stream_launch_multi<true>(const StreamMulti &, unsigned, cudaStream_t);

}  // namespace rfvh
