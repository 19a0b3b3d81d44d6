// Pair-kernel instantiations with end cells: the split s16x2 classes
// (virtual lanes, two per thread) and the int32 classes of the rescore.
#include "sw_pairs.cuh"

namespace swg {

int launch_pairs_ends(int lane, int L, int S, const PairArgs &a, const int32_t *list, const int32_t *count_dev,
                      int64_t n_hint, int num_sms, cudaStream_t st)
{
    const bool d0_16 = a.min_m >= -a.o;
#define SWG_CASEQ(VL, SS)                                                                                         \
    if (L == VL && S == SS)                                                                                       \
        return d0_16 ? launch_pairs_split_inst<VL / 2, SS, true, true>(a, list, count_dev, n_hint, num_sms, st)  \
                     : launch_pairs_split_inst<VL / 2, SS, false, true>(a, list, count_dev, n_hint, num_sms, st);
#define SWG_CASE32(LL, SS)                                                                                        \
    if (L == LL && S == SS)                                                                                       \
        return launch_pairs_inst<LaneI32, LL, SS, false, true>(a, list, count_dev, n_hint, num_sms, st);
    if (lane == LK_I16X2Q) {
        SWG_CASEQ(16, 8)
        SWG_CASEQ(16, 10)
        SWG_CASEQ(32, 8)
        SWG_CASEQ(32, 12)
        SWG_CASEQ(32, 16)
    } else if (lane == LK_I32) {
        SWG_CASE32(4, 8)
        SWG_CASE32(8, 8)
        SWG_CASE32(16, 8)
        SWG_CASE32(16, 10)
        SWG_CASE32(32, 8)
        SWG_CASE32(32, 16)
    }
#undef SWG_CASEQ
#undef SWG_CASE32
    return (int)cudaErrorInvalidValue;
}

}  // namespace swg
