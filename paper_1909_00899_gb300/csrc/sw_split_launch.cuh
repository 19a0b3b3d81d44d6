// Launch helper of the split-query s16x2 kernels (scan-F and lazy-F
// translation units).
#pragma once
#include <mutex>

#include "sw_launch.cuh"
#include "sw_split.cuh"

namespace swg {

template <int L, int S, bool D0, bool LAZY, bool ENDS = false, bool PIECES = false, bool AC = false>
int launch_split_inst(const BatchArgs &a, int num_sms, cudaStream_t st)
{
    auto kern = sw_split_kernel<L, S, D0, LAZY, ENDS, PIECES, AC>;
    constexpr size_t kMaxSmem = (size_t)34 * L * SegPad<S, 4>::value * 4;
    static SmemAttrOnce attr;  // one per kernel instantiation
    const int attr_err = set_smem_attr_once(attr, kern, kMaxSmem);
    if (attr_err != (int)cudaSuccess)
        return attr_err;
    const size_t smem = (size_t)(a.A + 2) * L * SegPad<S, 4>::value * 4;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BATCH_THREADS, smem);
    if (err != cudaSuccess)
        return (int)err;
    if (per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (!a.n_work_dev) {
        const int64_t per_block = (BATCH_THREADS / 32) * (32 / L);
        // pieces of long sequences: at most n_work more items
        const int64_t items = PIECES ? 2 * a.n_work : a.n_work;
        const int64_t need = (items + per_block - 1) / per_block;
        if (need < grid)
            grid = need;
    }
    if (grid < 1)
        return (int)cudaSuccess;
    kern<<<(unsigned)grid, BATCH_THREADS, smem, st>>>(a);
    return (int)cudaGetLastError();
}

// Layouts (virtual lanes x segment length) whose scan-F scores run the
// always-corrected pass when every substitution score is >= -o (measured
// faster there on GB300; at 64 x 20 and 32 x 12 / 32 x 20 the 80-register
// three-CTA budget leaves it no room, and the one-thread layouts have no
// carry to correct).
constexpr bool split_ac(int VL, int SS)
{
    return VL >= 16 && !(SS == 12 || SS == 20);
}

// the layouts (virtual lanes, two per thread) and both passes of one method
// (ENDS: scan-F with end cells)
template <bool LAZY, bool ENDS = false>
int launch_split_plan(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    const bool d0 = a.min_m >= -a.o;
#define SWG_CASE(VL, SS)                                                                                       \
    if (pl.L == VL && pl.S == SS)                                                                              \
        return d0 ? launch_split_inst<VL / 2, SS, true, LAZY, ENDS, false, !LAZY && !ENDS && split_ac(VL, SS)>( \
                        a, num_sms, st)                                                                        \
                  : launch_split_inst<VL / 2, SS, false, LAZY, ENDS>(a, num_sms, st);
    SWG_CASE(2, 16)
    SWG_CASE(2, 32)
    SWG_CASE(16, 8)
    SWG_CASE(16, 32)
    SWG_CASE(32, 8)
    SWG_CASE(32, 12)
    SWG_CASE(32, 16)
    SWG_CASE(32, 20)
    SWG_CASE(32, 24)
    SWG_CASE(32, 32)
    SWG_CASE(32, 40)
    SWG_CASE(64, 8)
    SWG_CASE(64, 16)
    SWG_CASE(64, 20)
    SWG_CASE(64, 24)
    SWG_CASE(64, 28)
    SWG_CASE(64, 32)
    SWG_CASE(64, 40)
#undef SWG_CASE
    return (int)cudaErrorInvalidValue;
}

// Launches that split long sequences into pieces (scores, scan-F or
// lazy-F): the layouts of at most 1024 query positions, the only ones a
// splitting call uses.
template <bool LAZY>
int launch_split_plan_pieces(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    const bool d0 = a.min_m >= -a.o;
#define SWG_CASE(VL, SS)                                                                                    \
    if (pl.L == VL && pl.S == SS)                                                                           \
        return d0 ? launch_split_inst<VL / 2, SS, true, LAZY, false, true, !LAZY && split_ac(VL, SS)>(a, num_sms, \
                                                                                                      st)   \
                  : launch_split_inst<VL / 2, SS, false, LAZY, false, true>(a, num_sms, st);
    SWG_CASE(2, 16)
    SWG_CASE(2, 32)
    SWG_CASE(16, 8)
    SWG_CASE(16, 32)
    SWG_CASE(32, 8)
    SWG_CASE(32, 12)
    SWG_CASE(32, 16)
    SWG_CASE(32, 20)
    SWG_CASE(32, 24)
    SWG_CASE(32, 32)
    SWG_CASE(64, 8)
    SWG_CASE(64, 16)
#undef SWG_CASE
    return (int)cudaErrorInvalidValue;
}

}  // namespace swg
