// Multi-query launches on the split s16x2 layouts of 64 virtual lanes (32
// threads per alignment): the (query, chunk) phase walk of queries of
// several chunks.
#include "sw_multi_launch.cuh"
#include "sw_split_launch.cuh"

namespace swg {

int multi_chunks_wide(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A)
{
    constexpr int KIND = MULTI_CHUNKS;
    SWG_MULTI_CASE(64, 8)
    SWG_MULTI_CASE(64, 16)
    SWG_MULTI_CASE(64, 20)
    SWG_MULTI_CASE(64, 24)
    SWG_MULTI_CASE(64, 28)
    SWG_MULTI_CASE(64, 32)
    SWG_MULTI_CASE(64, 40)
    return -1;
}

}  // namespace swg
