// Streaming column kernel of the third-order filter, forward and transposed
// steps (y pass).
#include "rf_stream_launch.h"

namespace rfvh {

template <bool ADJ>
void stream_launch(const StreamArgs &a, cudaStream_t st)
{
    stream_kernel<ADJ, kStreamDepth>
        <<<stream_grid(a.ncols, a.npairs), kStreamThreads, stream_smem_bytes(a.scratch), st>>>(a);
}

template <bool ADJ>
void stream_launch_multi(const StreamMulti &m, unsigned grid, cudaStream_t st)
{
    int ends = 0;
    for (int d = 0; d < m.nd; ++d) ends = ends > m.dom[d].scratch ? ends : m.dom[d].scratch;
    stream_multi_kernel<ADJ, kStreamDepth><<<grid, kStreamThreads, stream_smem_bytes(ends), st>>>(m);
}

template void stream_launch<false>(const StreamArgs &, cudaStream_t);
template void stream_launch<true>(const StreamArgs &, cudaStream_t);
template void stream_launch_multi<false>(const StreamMulti &, unsigned, cudaStream_t);
template void stream_launch_multi<true>(const StreamMulti &, unsigned, cudaStream_t);

}  // namespace rfvh
