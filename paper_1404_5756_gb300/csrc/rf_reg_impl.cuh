// rf_reg_impl.cuh -- host-side launch code of the register-resident kernel,
// included by the translation units that instantiate it (rf_reg_*.cu).
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "rf_reg_launch.h"

namespace rfvh {
namespace {

// Raise a kernel's dynamic shared-memory limit once per device and size, so
// a launch inside a stream capture makes no attribute call.
constexpr int kRegAttrDevices = 64;
template <int ORDER, bool ADJ, int DIR, int C, int P, bool CARRY, bool MULTI = false>
void reg_smem_attr(size_t smem)
{
    static std::mutex mu;
    static size_t done[kRegAttrDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < kRegAttrDevices && smem <= done[dev]) return;
    if (MULTI)
        cudaFuncSetAttribute(reg_multi_kernel<ORDER, ADJ, DIR, C, P, kRegWarps, reg_pairs(ORDER), CARRY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        cudaFuncSetAttribute(reg_kernel<ORDER, ADJ, DIR, C, P, kRegWarps, reg_pairs(ORDER), CARRY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < kRegAttrDevices) done[dev] = smem;
}

}  // namespace

#define RF_FOR_EACH_REG_SHAPE(X) X(16, 8) X(16, 16) X(24, 16) X(16, 32) X(24, 32) X(32, 32)

template <int ORDER, bool ADJ, int DIR, bool CARRY>
bool reg_launch(const RegArgs &a, RegShape sh, size_t smem, cudaStream_t st)
{
#define RF_REG_SHAPE(c, p)                                                                \
    if (sh.C == c && sh.P == p) {                                                         \
        reg_smem_attr<ORDER, ADJ, DIR, c, p, CARRY>(smem);                                \
        reg_kernel<ORDER, ADJ, DIR, c, p, kRegWarps, reg_pairs(ORDER), CARRY>                    \
            <<<reg_grid(DIR, sh, a.nlines, a.ngroups), kRegWarps * 32, smem, st>>>(a);    \
        return true;                                                                      \
    }
    RF_FOR_EACH_REG_SHAPE(RF_REG_SHAPE)
#undef RF_REG_SHAPE
    return false;
}

template <int ORDER, bool ADJ, int DIR, bool CARRY>
bool reg_launch_multi(const RegMulti &m, RegShape sh, size_t smem, unsigned grid, cudaStream_t st)
{
#define RF_REG_SHAPE(c, p)                                                                \
    if (sh.C == c && sh.P == p) {                                                         \
        reg_smem_attr<ORDER, ADJ, DIR, c, p, CARRY, true>(smem);                          \
        reg_multi_kernel<ORDER, ADJ, DIR, c, p, kRegWarps, reg_pairs(ORDER), CARRY>              \
            <<<grid, kRegWarps * 32, smem, st>>>(m);                                      \
        return true;                                                                      \
    }
    RF_FOR_EACH_REG_SHAPE(RF_REG_SHAPE)
#undef RF_REG_SHAPE
    return false;
}

template <int ORDER, bool ADJ, int DIR, bool CARRY>
int reg_occupancy(RegShape sh, size_t smem)
{
#define RF_REG_SHAPE(c, p)                                                                 \
    if (sh.C == c && sh.P == p) {                                                          \
        reg_smem_attr<ORDER, ADJ, DIR, c, p, CARRY>(smem);                                 \
        int blocks = 0;                                                                    \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                 \
                &blocks, reg_kernel<ORDER, ADJ, DIR, c, p, kRegWarps, reg_pairs(ORDER), CARRY>,   \
                kRegWarps * 32, smem)                                                      \
            != cudaSuccess) {                                                              \
            cudaGetLastError();                                                            \
            return 0;                                                                      \
        }                                                                                  \
        return blocks;                                                                     \
    }
    RF_FOR_EACH_REG_SHAPE(RF_REG_SHAPE)
#undef RF_REG_SHAPE
    return 0;
}

#undef RF_FOR_EACH_REG_SHAPE

#define RF_REG_INSTANTIATE(O, A, D, K)                                                   \
    template bool reg_launch<O, A, D, K>(const RegArgs &, RegShape, size_t, cudaStream_t); \
    template bool reg_launch_multi<O, A, D, K>(const RegMulti &, RegShape, size_t,         \
                                               unsigned, cudaStream_t);                     \
    template int reg_occupancy<O, A, D, K>(RegShape, size_t);

}  // namespace rfvh
