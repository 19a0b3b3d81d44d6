// Multi-query launches on the split s16x2 layouts of 16 and 32 virtual
// lanes (8 and 16 threads per alignment): the phase kernel of single-chunk
// queries.
#include "sw_multi_launch.cuh"
#include "sw_split_launch.cuh"

namespace swg {

int multi_phase_narrow(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A)
{
    constexpr int KIND = MULTI_PHASE;
    SWG_MULTI_CASE(16, 8)
    SWG_MULTI_CASE(16, 32)
    SWG_MULTI_CASE(32, 8)
    SWG_MULTI_CASE(32, 12)
    SWG_MULTI_CASE(32, 16)
    SWG_MULTI_CASE(32, 20)
    SWG_MULTI_CASE(32, 24)
    SWG_MULTI_CASE(32, 32)
    SWG_MULTI_CASE(32, 40)
    return -1;
}

}  // namespace swg
