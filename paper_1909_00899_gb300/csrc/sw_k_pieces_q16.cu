// Split-query s16x2 instantiations for launches that split long database
// sequences into pieces (scores of one-chunk queries, scan-F and lazy-F).
#include "sw_split_launch.cuh"

namespace swg {

int launch_batch_q16_pieces(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    return lazy ? launch_split_plan_pieces<true>(pl, a, num_sms, st)
                : launch_split_plan_pieces<false>(pl, a, num_sms, st);
}

}  // namespace swg
