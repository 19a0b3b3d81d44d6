// Split-query s16x2 lazy-F instantiations (Alg. 1 over the 2L virtual
// lanes): the plain-method comparison on the same layout as the scan-F
// split kernels.
#include "sw_split_launch.cuh"

namespace swg {

int launch_batch_q16_lazy(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    return launch_split_plan<true>(pl, a, num_sms, st);
}

}  // namespace swg
