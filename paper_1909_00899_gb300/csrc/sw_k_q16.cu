// Split-query s16x2 scan-F instantiations (two query halves of one alignment
// per register).  Plans count virtual lanes: a plan of 2L lanes runs on L
// threads.  Each layout has the D0 pass (every substitution score >= -o, the
// usual case) and the general one; the lazy-F comparison kernels are in
// sw_k_q16l.cu.
#include "sw_split_launch.cuh"

namespace swg {

int launch_batch_q16_lazy(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st);

int launch_batch_q16(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    return lazy ? launch_batch_q16_lazy(pl, a, num_sms, st) : launch_split_plan<false>(pl, a, num_sms, st);
}

}  // namespace swg
