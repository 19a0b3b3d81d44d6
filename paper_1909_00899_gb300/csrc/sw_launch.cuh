// Launch helper shared by the per-lane-type kernel translation units.
#pragma once
#include <mutex>

#include "sw_batch.cuh"

namespace swg {

template <class LT, int L, int S, bool LAZY, bool ENDS = false, bool PIECES = false>
int launch_batch_inst(const BatchArgs &a, int num_sms, cudaStream_t st)
{
    auto kern = sw_batch_kernel<LT, L, S, LAZY, ENDS, PIECES>;
    // alphabet of at most 32 residues + the unknown and the inert rows
    constexpr size_t kMaxSmem = (size_t)34 * L * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    });
    if (attr_err != cudaSuccess)
        return (int)attr_err;
    const size_t smem = (size_t)(a.A + 2) * L * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BATCH_THREADS, smem);
    if (err != cudaSuccess)
        return (int)err;
    if (per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (!a.n_work_dev) {
        // no more blocks than there are work units for their warps (pieces
        // of long sequences: at most n_work more items)
        const int64_t items = PIECES ? 2 * a.n_work : a.n_work;
        const int64_t units = (items + LT::CELLS - 1) / LT::CELLS;
        const int64_t per_block = (BATCH_THREADS / 32) * (32 / L);
        const int64_t need = (units + per_block - 1) / per_block;
        if (need < grid)
            grid = need;
    }
    if (grid < 1)
        return (int)cudaSuccess;
    kern<<<(unsigned)grid, BATCH_THREADS, smem, st>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace swg
