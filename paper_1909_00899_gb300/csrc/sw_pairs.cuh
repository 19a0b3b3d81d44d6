// Pair kernel: n independent alignments, each with its own query (reads
// against their own reference windows).  Each group of L lanes takes CELLS
// pairs, writes their striped profiles into its own slice of shared memory
// (biased by +o, straight from the query residues and the substitution
// matrix held in the launch parameters), then runs the same per-column
// scan-F core as the batch kernel.  Pairs arrive pre-sorted into
// query-length classes so that one launch covers queries of at most L*S
// positions (single chunk).
#pragma once
#include "sw_batch.cuh"
#include "sw_split.cuh"

namespace swg {

// ENDS (int32 lanes, scan-F): also the end cell of each pair's best
// alignment into p.q_end / p.r_end (1-based, -1 when the score is 0).
template <class LT, int L, int S, bool LAZY, bool ENDS = false>
__global__ void __launch_bounds__(256) sw_pairs_kernel(const PairArgs p, const int32_t *__restrict__ list,
                                                       const int32_t *__restrict__ count_dev, int64_t n_list)
{
    static_assert(!ENDS || (LT::CELLS == 1 && !LAZY), "pair end cells: int32 scan-F");
    using T = typename LT::T;
    using Elem = typename LT::Elem;
    constexpr int CELLS = LT::CELLS;
    constexpr int V = LT::VEC;
    constexpr int SP = SegPad<S, V>::value;
    constexpr int G = 32 / L;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int A = p.A;
    const int cell_elems = (A + 2) * L * SP;  // rows 0..A-1, unknown residue A, inert A+1
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const int gid = (threadIdx.x >> 5) * G + grp;
    Elem *gprof = reinterpret_cast<Elem *>(smem_raw) + (size_t)gid * CELLS * cell_elems;
    const Elem *pbase[CELLS];
#pragma unroll
    for (int c = 0; c < CELLS; ++c)
        pbase[c] = gprof + c * cell_elems;

    // entries of list to process: the class size, or a count on the device
    const int64_t n_work = count_dev ? (int64_t)(*count_dev) : n_list;
    const int64_t units = (n_work + CELLS - 1) / CELLS;
    unsigned long long lazy_steps = 0;

    for (;;) {
        unsigned int ubase = 0;
        if (lane == 0)
            ubase = atomicAdd(p.counter, (unsigned int)G);
        ubase = __shfl_sync(FULL, ubase, 0);
        if ((int64_t)ubase >= units)
            break;
        const int64_t unit = (int64_t)ubase + grp;
        int pid[CELLS];
        int64_t start[CELLS];
        int len[CELLS];
        int my_n = 0;
#pragma unroll
        for (int c = 0; c < CELLS; ++c) {
            const int64_t w = unit * CELLS + c;
            const bool ok = unit < units && w < n_work;
            pid[c] = ok ? (list ? list[w] : (int)w) : -1;
            int64_t qs = 0;
            int ql = 0;
            if (ok) {
                qs = p.q_off[pid[c]];
                ql = (int)(p.q_off[pid[c] + 1] - qs);
                start[c] = p.r_off[pid[c]];
                len[c] = (int)(p.r_off[pid[c] + 1] - start[c]);
            } else {
                start[c] = 0;
                len[c] = 0;
            }
            if (ql == 0)
                len[c] = 0;  // empty query: score 0
            my_n = max(my_n, len[c]);
            // this cell's striped profile: lane gl fills segment positions
            Elem *dst = gprof + c * cell_elems;
            for (int pos = gl; pos < L * SP; pos += L) {
                const int l = pos / SP;
                const int j = pos - l * SP;
                const int qp = l * S + j;
                // query code (>= A: an unknown residue), -1 past the query end
                const int code = (j < S && qp < ql) ? (int)p.q[qs + qp] : -1;
#pragma unroll 4
                for (int a = 0; a <= A + 1; ++a) {
                    int v = LT::PAD;
                    if (code >= 0 && a <= A)
                        v = (code < A && a < A ? (int)p.M[code * A + a] : (int)p.min_m) + LT::prof_bias(p.o);
                    dst[((a * (SP / V) + j / V) * L + l) * V + (j % V)] = (Elem)v;
                }
            }
        }
        __syncwarp(FULL);
        const int ncols = (int)__reduce_max_sync(FULL, (unsigned)my_n);
        if constexpr (ENDS) {
            int er = -1, eq = -1;
            const T mx = striped_unit<LT, L, S, false, true>(pbase, p.r, start, len, ncols, A, p.o, p.e, p.one,
                                                             false, false, nullptr, gl, lazy_steps, &er, &eq);
            if (gl == 0 && pid[0] >= 0) {
                const int sc = (int)mx;
                p.scores[pid[0]] = sc;
                p.q_end[pid[0]] = sc > 0 ? eq + 1 : -1;
                p.r_end[pid[0]] = sc > 0 ? er + 1 : -1;
            }
        } else {
            const T mx = striped_unit<LT, L, S, LAZY>(pbase, p.r, start, len, ncols, A, p.o, p.e, p.one, false,
                                                      false, nullptr, gl, lazy_steps);
            if (gl == 0)
                write_scores<LT>(mx, LT::consts(p.o, p.e, S, p.one), pid, false, p.flag_thresh, p.scores);
        }
        __syncwarp(FULL);  // profiles are rewritten by the next unit
    }
    // j-steps of the lazy-F correction loop, counted once per warp
    if (LAZY && p.lazy_steps && lane == 0 && lazy_steps)
        atomicAdd(p.lazy_steps, lazy_steps);
}

// Shared memory of one warp: CELLS profiles per group, 32 / L groups.
template <class LT, int S>
constexpr size_t pair_smem_per_warp(int A)
{
    return (size_t)32 * LT::CELLS * (A + 2) * SegPad<S, LT::VEC>::value * sizeof(typename LT::Elem);
}

template <class LT, int L, int S, bool LAZY, bool ENDS = false>
int launch_pairs_inst(const PairArgs &a, const int32_t *list, const int32_t *count_dev, int64_t n_hint,
                      int num_sms, cudaStream_t st)
{
    auto kern = sw_pairs_kernel<LT, L, S, LAZY, ENDS>;
    const size_t per_warp = pair_smem_per_warp<LT, S>(a.A);
    int warps = (int)std::min<size_t>(8, std::max<size_t>(1, (size_t)(96 * 1024) / per_warp));
    const size_t smem = per_warp * warps;
    if (smem > 200 * 1024)
        return (int)cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return (int)err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (err != cudaSuccess)
        return (int)err;
    if (per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    const int64_t units = (n_hint + LT::CELLS - 1) / LT::CELLS;
    const int64_t per_block = (int64_t)warps * (32 / L);
    const int64_t need = (units + per_block - 1) / per_block;
    if (need < grid)
        grid = need;
    if (grid < 1)
        return (int)cudaSuccess;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(a, list, count_dev, n_hint);
    return (int)cudaGetLastError();
}

// Split-query s16x2 pair kernel: a group of L threads takes one pair and
// holds the first half of its query in the low halves and the second half
// in the high halves (2L virtual lanes, sw_split.cuh); each group stages its
// pair's profile as (low position, high position) pairs in its own slice of
// shared memory, row A the unknown residue, row A+1 inert.  ENDS: also the
// end cell of each pair's best alignment (1-based, -1 when the score is 0).
// LAZY: the lazy-F loop instead of the scan (the comparison on the same layout).
// AC: scan-F scores with the always-corrected pass (sw_split.cuh).
template <int L, int S, bool D0, bool ENDS = false, bool LAZY = false, bool AC = false>
__global__ void __launch_bounds__(256) sw_pairs_split_kernel(const PairArgs p, const int32_t *__restrict__ list,
                                                             const int32_t *__restrict__ count_dev, int64_t n_list)
{
    static_assert(!(ENDS && LAZY), "end cells: scan-F only");
    static_assert(!AC || (D0 && !ENDS && !LAZY), "always-corrected pass: D0 scan-F scores");
    unsigned long long lazy_steps = 0;
    constexpr int SP = SegPad<S, 4>::value;
    constexpr int QH = L * S;  // positions per half
    constexpr int G = 32 / L;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int A = p.A;
    const int cell_elems = (A + 2) * L * SP;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const int gid = (threadIdx.x >> 5) * G + grp;
    uint32_t *gprof = reinterpret_cast<uint32_t *>(smem_raw) + (size_t)gid * cell_elems;
    const int pb = split_pb<D0>(p.o);
    const LaneQ16::K k = LaneQ16::consts_pb(p.o, p.e, S, p.one, pb);
    const int64_t n_work = count_dev ? (int64_t)(*count_dev) : n_list;

    for (;;) {
        unsigned int ubase = 0;
        if (lane == 0)
            ubase = atomicAdd(p.counter, (unsigned int)G);
        ubase = __shfl_sync(FULL, ubase, 0);
        if ((int64_t)ubase >= n_work)
            break;
        const int64_t w = (int64_t)ubase + grp;
        int pid[1];
        pid[0] = w < n_work ? (list ? list[w] : (int)w) : -1;
        int64_t qs = 0, start = 0;
        int ql = 0, len = 0;
        if (pid[0] >= 0) {
            qs = p.q_off[pid[0]];
            ql = (int)(p.q_off[pid[0] + 1] - qs);
            start = p.r_off[pid[0]];
            len = (int)(p.r_off[pid[0] + 1] - start);
        }
        if (ql == 0)
            len = 0;  // empty query: score 0
        for (int pos = gl; pos < L * SP; pos += L) {
            const int l = pos / SP;
            const int j = pos - l * SP;
            const int plo = l * S + j, phi = QH + l * S + j;
            // query codes (>= A: an unknown residue), -1 past the query end
            const int clo = (j < S && plo < ql) ? (int)p.q[qs + plo] : -1;
            const int chi = (j < S && phi < ql) ? (int)p.q[qs + phi] : -1;
            for (int a = 0; a <= A + 1; ++a) {
                int lo = LaneQ16::PAD, hi = LaneQ16::PAD;
                if (a <= A) {
                    if (clo >= 0)
                        lo = (clo < A && a < A ? (int)p.M[clo * A + a] : (int)p.min_m) + pb;
                    if (chi >= 0)
                        hi = (chi < A && a < A ? (int)p.M[chi * A + a] : (int)p.min_m) + pb;
                }
                gprof[((a * (SP / 4) + j / 4) * L + l) * 4 + (j % 4)] =
                    (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
            }
        }
        __syncwarp(FULL);
        const int ncols = (int)__reduce_max_sync(FULL, (unsigned)len);
        if constexpr (ENDS) {
            int er = -1, eq = -1;
            const uint32_t mx = split_unit<L, S, D0, false, true>(gprof, p.r, start, len, ncols, A, p.o, p.e,
                                                                  p.one, false, false, nullptr, gl, nullptr, &er,
                                                                  &eq);
            if (gl == 0 && pid[0] >= 0) {
                const int sc = LaneQ16::score(mx, 0, k);
                p.scores[pid[0]] = sc;
                p.q_end[pid[0]] = sc > 0 ? eq + 1 : -1;
                p.r_end[pid[0]] = sc > 0 ? er + 1 : -1;
            }
        } else {
            const uint32_t mx = split_unit<L, S, D0, LAZY, false, AC>(gprof, p.r, start, len, ncols, A, p.o, p.e,
                                                                      p.one, false, false, nullptr, gl, &lazy_steps);
            if (gl == 0)
                write_scores<LaneQ16>(mx, k, pid, false, p.flag_thresh, p.scores);
        }
        __syncwarp(FULL);  // the profile is rewritten by the next unit
    }
    // j-steps of the lazy-F correction loop, counted once per warp
    if (LAZY && p.lazy_steps && lane == 0 && lazy_steps)
        atomicAdd(p.lazy_steps, lazy_steps);
}

template <int L, int S, bool D0, bool ENDS = false, bool LAZY = false, bool AC = false>
int launch_pairs_split_inst(const PairArgs &a, const int32_t *list, const int32_t *count_dev, int64_t n_hint,
                            int num_sms, cudaStream_t st)
{
    auto kern = sw_pairs_split_kernel<L, S, D0, ENDS, LAZY, AC>;
    const size_t per_warp = (size_t)32 * (a.A + 2) * SegPad<S, 4>::value * 4;
    int warps = (int)std::min<size_t>(8, std::max<size_t>(1, (size_t)(96 * 1024) / per_warp));
    const size_t smem = per_warp * warps;
    if (smem > 200 * 1024)
        return (int)cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return (int)err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (err != cudaSuccess)
        return (int)err;
    if (per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    const int64_t per_block = (int64_t)warps * (32 / L);
    const int64_t need = (n_hint + per_block - 1) / per_block;
    if (need < grid)
        grid = need;
    if (grid < 1)
        return (int)cudaSuccess;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(a, list, count_dev, n_hint);
    return (int)cudaGetLastError();
}

}  // namespace swg
