// Split-query s16x2 scan-F instantiations with end cells (the first cell in
// column order that reaches each alignment's score).
#include "sw_split_launch.cuh"

namespace swg {

int launch_batch_q16_ends(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    return launch_split_plan<false, true>(pl, a, num_sms, st);
}

}  // namespace swg
