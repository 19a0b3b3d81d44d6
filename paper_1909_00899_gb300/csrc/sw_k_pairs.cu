// Pair-kernel instantiations: query-length classes per lane type (the split
// s16x2 classes count virtual lanes, two per thread).
#include <algorithm>

#include "sw_pairs.cuh"

namespace swg {

int launch_pairs(int lane, int L, int S, bool lazy, const PairArgs &a, const int32_t *list, const int32_t *count_dev,
                 int64_t n_hint, int num_sms, cudaStream_t st)
{
    // shorter corrected pass (sw_lanes.cuh): int32 when min(M) >= -(o+e),
    // s16x2 when min(M) >= -o
    const bool d0_32 = (int64_t)a.min_m >= -(int64_t)a.o - a.e;
    const bool d0_16 = a.min_m >= -a.o;
#define SWG_CASE(LT, LL, SS)                                                        \
    if (L == LL && S == SS)                                                         \
        return launch_pairs_inst<LT, LL, SS, false>(a, list, count_dev, n_hint, num_sms, st);
#define SWG_CASE16(LL, SS)                                                          \
    if (L == LL && S == SS)                                                         \
        return d0_16 ? launch_pairs_inst<LaneI16x2D, LL, SS, false>(a, list, count_dev, n_hint, num_sms, st) \
                     : launch_pairs_inst<LaneI16x2, LL, SS, false>(a, list, count_dev, n_hint, num_sms, st);
#define SWG_CASE_LAZY(LL, SS)                                                       \
    if (L == LL && S == SS)                                                         \
        return lazy    ? launch_pairs_inst<LaneI32, LL, SS, true>(a, list, count_dev, n_hint, num_sms, st)  \
               : d0_32 ? launch_pairs_inst<LaneI32D, LL, SS, false>(a, list, count_dev, n_hint, num_sms, st) \
                       : launch_pairs_inst<LaneI32, LL, SS, false>(a, list, count_dev, n_hint, num_sms, st);
    if (lane == LK_I32) {
        SWG_CASE_LAZY(4, 8)
        SWG_CASE_LAZY(8, 8)
        SWG_CASE_LAZY(16, 8)
        SWG_CASE_LAZY(16, 10)
        SWG_CASE_LAZY(32, 8)
        SWG_CASE_LAZY(32, 16)
    } else if (lane == LK_I16X2) {
        SWG_CASE16(8, 8)
        SWG_CASE16(16, 8)
        SWG_CASE16(16, 10)
        SWG_CASE16(32, 8)
        SWG_CASE16(32, 16)
    } else if (lane == LK_I16X2Q) {
        // virtual lanes (two per thread), as the batch split layouts; AC:
        // the always-corrected pass, on the classes where it measured faster
        // on DNA reads vs windows (16 x 10: +4 %, 32 x 8: +3 %; the others
        // 2-10 % slower)
#define SWG_CASEQ(VL, SS)                                                                                          \
    if (L == VL && S == SS) {                                                                                      \
        constexpr bool AC = (VL == 16 && SS == 10) || (VL == 32 && SS == 8);                                       \
        return lazy    ? (d0_16 ? launch_pairs_split_inst<VL / 2, SS, true, false, true>(a, list, count_dev, n_hint, \
                                                                                        num_sms, st)               \
                                : launch_pairs_split_inst<VL / 2, SS, false, false, true>(a, list, count_dev,      \
                                                                                         n_hint, num_sms, st))     \
               : d0_16 ? launch_pairs_split_inst<VL / 2, SS, true, false, false, AC>(a, list, count_dev, n_hint,    \
                                                                                     num_sms, st)                  \
                       : launch_pairs_split_inst<VL / 2, SS, false>(a, list, count_dev, n_hint, num_sms, st);      \
    }
        SWG_CASEQ(16, 8)
        SWG_CASEQ(16, 10)
        SWG_CASEQ(32, 8)
        SWG_CASEQ(32, 12)
        SWG_CASEQ(32, 16)
#undef SWG_CASEQ
    } else if (lane == LK_I8X4) {
        SWG_CASE(LaneI8x4, 8, 16)
        SWG_CASE(LaneI8x4, 16, 10)
        SWG_CASE(LaneI8x4, 16, 16)
        SWG_CASE(LaneI8x4, 32, 16)
    }
#undef SWG_CASE
#undef SWG_CASE16
#undef SWG_CASE_LAZY
    return (int)cudaErrorInvalidValue;
}

}  // namespace swg
