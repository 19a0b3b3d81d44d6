// Launch helpers of the multi-query kernels (sw_k_multi*.cu).
#pragma once
#include "sw_launch.cuh"
#include "sw_multi.cuh"

namespace swg {

// KIND: MULTI_FUSED (tiles, all chunks of a unit in one CTA), MULTI_PHASE
// (single-chunk queries), MULTI_CHUNKS (the (query, chunk) phase walk)
template <int L, int S, bool D0, bool AC, int KIND>
int multi_split_inst(const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A)
{
    auto kern = KIND == MULTI_PHASE    ? sw_multi_phase_kernel<L, S, D0, AC>
                : KIND == MULTI_CHUNKS ? sw_multi_chunks_kernel<L, S, D0, AC>
                                       : sw_multi_split_kernel<L, S, D0, AC>;
    constexpr size_t kMaxSmem = (size_t)34 * L * SegPad<S, 4>::value * 4;
    static SmemAttrOnce attr;
    const int attr_err = set_smem_attr_once(attr, kern, kMaxSmem);
    if (attr_err != (int)cudaSuccess)
        return attr_err;
    if (per_sm) {  // occupancy query only
        const size_t smem = (size_t)(A + 2) * L * SegPad<S, 4>::value * 4;
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, BATCH_THREADS, smem);
    }
    const size_t smem = (size_t)(a->A + 2) * L * SegPad<S, 4>::value * 4;
    if (grid < 1)
        return (int)cudaSuccess;
    kern<<<(unsigned)grid, BATCH_THREADS, smem, st>>>(*a);
    return (int)cudaGetLastError();
}

template <class LT, int S>
int multi_i32_inst(const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A)
{
    auto kern = sw_multi_i32_kernel<LT, S>;
    constexpr size_t kMaxSmem = (size_t)34 * 32 * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
    static SmemAttrOnce attr;
    const int attr_err = set_smem_attr_once(attr, kern, kMaxSmem);
    if (attr_err != (int)cudaSuccess)
        return attr_err;
    if (per_sm) {
        const size_t smem = (size_t)(A + 2) * 32 * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, BATCH_THREADS, smem);
    }
    const size_t smem = (size_t)(a->A + 2) * 32 * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
    if (grid < 1)
        return (int)cudaSuccess;
    kern<<<(unsigned)grid, BATCH_THREADS, smem, st>>>(*a);
    return (int)cudaGetLastError();
}

// One translation unit's split layouts: VL virtual lanes (L = VL / 2
// threads) x S positions, the always-corrected pass where the per-query
// kernels run it (split_ac), the general pass when some score is below -o.
// KIND: the kernel kind of the translation unit
#define SWG_MULTI_CASE(VL, SS)                                                                           \
    if (VL_ == VL && S_ == SS)                                                                           \
        return d0 ? multi_split_inst<VL / 2, SS, true, split_ac(VL, SS), KIND>(a, grid, st, per_sm, A) \
                  : multi_split_inst<VL / 2, SS, false, false, KIND>(a, grid, st, per_sm, A);

}  // namespace swg
