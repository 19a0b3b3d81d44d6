// s16x2-lane instantiations of the scan-F kernel (two alignments per register;
// the shorter corrected pass of LaneI16x2D when the matrix allows it).
#include "sw_launch.cuh"

namespace swg {

int launch_batch_i16(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    // the profile biased by o must stay >= 0: every substitution score >= -o
    const bool d0 = a.min_m >= -a.o;
#define SWG_CASE(LL, SS)                                                          \
    if (pl.L == LL && pl.S == SS)                                                 \
        return lazy ? launch_batch_inst<LaneI16x2, LL, SS, true>(a, num_sms, st)  \
               : d0 ? launch_batch_inst<LaneI16x2D, LL, SS, false>(a, num_sms, st) \
                    : launch_batch_inst<LaneI16x2, LL, SS, false>(a, num_sms, st);
    SWG_CASE(8, 8)
    SWG_CASE(8, 16)
    SWG_CASE(16, 8)
    SWG_CASE(16, 16)
    SWG_CASE(32, 8)
    SWG_CASE(32, 12)
    SWG_CASE(32, 16)
    SWG_CASE(16, 32)
    SWG_CASE(32, 24)
    SWG_CASE(32, 32)
#undef SWG_CASE
    return (int)cudaErrorInvalidValue;
}

}  // namespace swg
