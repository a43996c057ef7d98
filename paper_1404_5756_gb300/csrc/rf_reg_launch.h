// rf_reg_launch.h -- launch entry points of the register-resident kernel
// (rf_reg.cuh).  It is instantiated per filter order, forward/adjoint and
// direction in eight translation units (rf_reg_*.cu), plus four for the
// carried-coast first-order kernels (rf_reg_1*c.cu), that compile in
// parallel; each holds the (chunk length, lanes per line) pairs below.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "rf_reg.cuh"

namespace rfvh {

constexpr int kRegWarps = 4;   // warps per CTA
// Slice pairs per thread: one for the third-order filter (168 registers at
// 32-point chunks, three CTAs and twelve warps per SM), two for the first
// order (its two-term steps leave room for four slices at two CTAs per SM).
constexpr int reg_pairs(int order) { return order == 3 ? 1 : 2; }

struct RegShape {
    int C, P;   // chunk length, lanes per line
};

// Built (C, P) pairs, in the order the planner tries them: the first with
// P C >= n serves lines of n points (up to 128, 256, 384, 512, 768, 1024).
// Chunks of 32 points spill registers at fewer than 32 lanes, so the
// mid-length lines take 16-point chunks on more lanes.
constexpr RegShape kRegShapes[] = {{16, 8}, {16, 16}, {24, 16}, {16, 32}, {24, 32}, {32, 32}};

// Launch one pass.  Returns false if (C, P) is not built.  CARRY: the
// carried-coast kernels (first order only, in their own translation units).
template <int ORDER, bool ADJ, int DIR, bool CARRY = false>
bool reg_launch(const RegArgs &a, RegShape sh, size_t smem, cudaStream_t st);

// Launch one pass over the m.nd domains of m (all of chunking sh) as one
// grid of `grid` = m.cta0[m.nd] CTAs.  Returns false if (C, P) is not built.
template <int ORDER, bool ADJ, int DIR, bool CARRY = false>
bool reg_launch_multi(const RegMulti &m, RegShape sh, size_t smem, unsigned grid,
                      cudaStream_t st);

// Resident CTAs per SM with `smem` bytes of dynamic shared memory (0: cannot
// run or not built).
template <int ORDER, bool ADJ, int DIR, bool CARRY = false>
int reg_occupancy(RegShape sh, size_t smem);

#define RF_REG_DECLARE(O, A, D, K)                                                               \
    extern template bool reg_launch<O, A, D, K>(const RegArgs &, RegShape, size_t, cudaStream_t); \
    extern template bool reg_launch_multi<O, A, D, K>(const RegMulti &, RegShape, size_t,         \
                                                      unsigned, cudaStream_t);                    \
    extern template int reg_occupancy<O, A, D, K>(RegShape, size_t);
RF_REG_DECLARE(3, false, 0, false)
RF_REG_DECLARE(3, false, 1, false)
RF_REG_DECLARE(3, true, 0, false)
RF_REG_DECLARE(3, true, 1, false)
RF_REG_DECLARE(1, false, 0, false)
RF_REG_DECLARE(1, false, 1, false)
RF_REG_DECLARE(1, true, 0, false)
RF_REG_DECLARE(1, true, 1, false)
RF_REG_DECLARE(1, false, 0, true)
RF_REG_DECLARE(1, false, 1, true)
RF_REG_DECLARE(1, true, 0, true)
RF_REG_DECLARE(1, true, 1, true)
#undef RF_REG_DECLARE

// Grid of a pass: x: (row blocks of 32/P rows, slice groups / warps per
// CTA); y: (column blocks of kRegWarps * 32/P columns, slice groups).
inline dim3 reg_grid(int dir, RegShape sh, int64_t nlines, int64_t ngroups)
{
    const int64_t lpw = 32 / sh.P;
    if (dir == 0)
        return dim3((unsigned)((nlines + lpw - 1) / lpw),
                    (unsigned)((ngroups + kRegWarps - 1) / kRegWarps));
    const int64_t R = kRegWarps * lpw;
    return dim3((unsigned)((nlines + R - 1) / R), (unsigned)ngroups);
}

}  // namespace rfvh
