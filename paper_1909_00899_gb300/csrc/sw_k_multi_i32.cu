// Multi-query launches on int32 lanes (32 lanes x 8, 16 or 32 positions):
// the pairs that could overflow the packed lanes.  The shorter corrected
// pass (LaneI32D) when every score is >= -(o + e).
#include "sw_multi_launch.cuh"

namespace swg {

static int multi_i32(int S, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A)
{
    if (S == 8)
        return d0 ? multi_i32_inst<LaneI32D, 8>(a, grid, st, per_sm, A)
                  : multi_i32_inst<LaneI32, 8>(a, grid, st, per_sm, A);
    if (S == 16)
        return d0 ? multi_i32_inst<LaneI32D, 16>(a, grid, st, per_sm, A)
                  : multi_i32_inst<LaneI32, 16>(a, grid, st, per_sm, A);
    if (S == 32)
        return d0 ? multi_i32_inst<LaneI32D, 32>(a, grid, st, per_sm, A)
                  : multi_i32_inst<LaneI32, 32>(a, grid, st, per_sm, A);
    return (int)cudaErrorInvalidValue;
}

int launch_multi_i32(int S, const MultiArgs &a, int grid, cudaStream_t st)
{
    return multi_i32(S, a.min_m >= -(a.o + a.e), &a, grid, st, nullptr, a.A);
}

int multi_i32_blocks_per_sm(int S, bool d0, int A)
{
    int per_sm = 0;
    const int r = multi_i32(S, d0, nullptr, 0, nullptr, &per_sm, A);
    return r == (int)cudaSuccess ? per_sm : 0;
}

}  // namespace swg
