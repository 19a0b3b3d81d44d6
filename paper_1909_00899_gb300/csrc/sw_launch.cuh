// Launch helper shared by the per-lane-type kernel translation units.
#pragma once
#include <mutex>

#include "sw_batch.cuh"

namespace swg {

// The dynamic shared-memory limit is an attribute of a kernel on each
// device: set it once per kernel and device (the current one).  Each
// launcher instantiation owns its flags (every kernel here has the same
// function type, so the flags cannot live in a helper keyed by that type).
constexpr int kMaxDev = 64;
struct SmemAttrOnce {
    std::once_flag once[kMaxDev];
    cudaError_t err[kMaxDev];
};

template <class Kern>
int set_smem_attr_once(SmemAttrOnce &st, Kern kern, size_t bytes)
{
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return (int)e;
    if (dev < 0 || dev >= kMaxDev)
        return (int)cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    std::call_once(st.once[dev], [&] {
        st.err[dev] = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    return (int)st.err[dev];
}

template <class LT, int L, int S, bool LAZY, bool ENDS = false, bool PIECES = false>
int launch_batch_inst(const BatchArgs &a, int num_sms, cudaStream_t st)
{
    auto kern = sw_batch_kernel<LT, L, S, LAZY, ENDS, PIECES>;
    // alphabet of at most 32 residues + the unknown and the inert rows
    constexpr size_t kMaxSmem = (size_t)34 * L * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
    static SmemAttrOnce attr;  // one per kernel instantiation
    const int attr_err = set_smem_attr_once(attr, kern, kMaxSmem);
    if (attr_err != (int)cudaSuccess)
        return attr_err;
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
