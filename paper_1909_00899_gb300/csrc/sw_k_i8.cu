// s8x4-lane instantiations of the scan-F kernel (four alignments per register).
#include "sw_launch.cuh"

namespace swg {

int launch_batch_i8(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st)
{
#define SWG_CASE(LL, SS)                          \
    if (pl.L == LL && pl.S == SS)                 \
        return launch_batch_inst<LaneI8x4, LL, SS, false>(a, num_sms, st);
    SWG_CASE(8, 16)
    SWG_CASE(16, 16)
    SWG_CASE(32, 16)
#undef SWG_CASE
    return (int)cudaErrorInvalidValue;
}

}  // namespace swg
