// Multi-query launches on the split s16x2 layouts of 64 virtual lanes (32
// threads per alignment): the fused-chunk kernel; and the dispatch over
// every split layout and kernel kind.
#include "sw_multi_launch.cuh"
#include "sw_split_launch.cuh"

namespace swg {

int multi_split_narrow(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A);
int multi_phase_narrow(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A);
int multi_phase_wide(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A);
int multi_chunks_narrow(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A);
int multi_chunks_wide(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm, int A);

static int multi_split_wide(int VL_, int S_, bool d0, const MultiArgs *a, int grid, cudaStream_t st, int *per_sm,
                            int A)
{
    constexpr int KIND = MULTI_FUSED;
    SWG_MULTI_CASE(64, 8)
    SWG_MULTI_CASE(64, 16)
    SWG_MULTI_CASE(64, 20)
    SWG_MULTI_CASE(64, 24)
    SWG_MULTI_CASE(64, 28)
    SWG_MULTI_CASE(64, 32)
    SWG_MULTI_CASE(64, 40)
    return -1;
}

static int multi_split(int VL, int S, int kind, bool d0, const MultiArgs *a, int grid, cudaStream_t st,
                       int *per_sm, int A)
{
    int r = kind == MULTI_PHASE    ? multi_phase_narrow(VL, S, d0, a, grid, st, per_sm, A)
            : kind == MULTI_CHUNKS ? multi_chunks_narrow(VL, S, d0, a, grid, st, per_sm, A)
                                   : multi_split_narrow(VL, S, d0, a, grid, st, per_sm, A);
    if (r == -1)
        r = kind == MULTI_PHASE    ? multi_phase_wide(VL, S, d0, a, grid, st, per_sm, A)
            : kind == MULTI_CHUNKS ? multi_chunks_wide(VL, S, d0, a, grid, st, per_sm, A)
                                   : multi_split_wide(VL, S, d0, a, grid, st, per_sm, A);
    return r == -1 ? (int)cudaErrorInvalidValue : r;
}

int launch_multi_split(int VL, int S, int kind, const MultiArgs &a, int grid, cudaStream_t st)
{
    return multi_split(VL, S, kind, a.min_m >= -a.o, &a, grid, st, nullptr, a.A);
}

int multi_split_blocks_per_sm(int VL, int S, int kind, bool d0, int A)
{
    int per_sm = 0;
    const int r = multi_split(VL, S, kind, d0, nullptr, 0, nullptr, &per_sm, A);
    return r == (int)cudaSuccess ? per_sm : 0;
}

int multi_groups_per_cta(int lanes)
{
    return (BATCH_THREADS / 32) * (32 / (lanes / 2));
}

}  // namespace swg
