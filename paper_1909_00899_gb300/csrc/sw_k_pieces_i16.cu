// s16x2- and s8x4-lane instantiations for launches that split long database
// sequences into pieces (scores of one-chunk queries, scan-F and lazy-F).
#include "sw_launch.cuh"

namespace swg {

int launch_batch_i16_pieces(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st)
{
    const bool d0 = a.min_m >= -a.o;
#define SWG_CASE(LL, SS)                                                                          \
    if (pl.L == LL && pl.S == SS)                                                                 \
        return lazy ? launch_batch_inst<LaneI16x2, LL, SS, true, false, true>(a, num_sms, st)     \
               : d0 ? launch_batch_inst<LaneI16x2D, LL, SS, false, false, true>(a, num_sms, st)   \
                    : launch_batch_inst<LaneI16x2, LL, SS, false, false, true>(a, num_sms, st);
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

int launch_batch_i8_pieces(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st)
{
#define SWG_CASE(LL, SS)              \
    if (pl.L == LL && pl.S == SS)     \
        return launch_batch_inst<LaneI8x4, LL, SS, false, false, true>(a, num_sms, st);
    SWG_CASE(8, 16)
    SWG_CASE(16, 16)
    SWG_CASE(32, 16)
#undef SWG_CASE
    return (int)cudaErrorInvalidValue;
}

}  // namespace swg
