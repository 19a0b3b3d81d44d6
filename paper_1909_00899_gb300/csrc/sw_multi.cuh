// Many independent queries against one resident database in one persistent
// launch per layout (the ragged batch; the paper's independent alignments,
// Sec. III, across queries as well as database sequences).
//
// Work unit: (query q, tile t), where a tile is K * GPC consecutive entries
// (K = k_items)
// of the database's order, exactly by length (longest first), and GPC is the
// number of lane groups of a CTA: every group takes K sequences of the tile,
// the k-th ones of all groups adjacent in the order, so the groups of a CTA
// finish each step together.  A single-chunk query stages its profile once
// per unit for all K steps.
// Units are numbered tile-major (unit = t * n_queries + q): the longest
// tiles of every query go first, which keeps the launch's tail short without
// splitting long sequences.  Persistent CTAs pull units from one counter.
//
// A unit runs every chunk of its query in order inside the CTA: the CTA
// stages chunk c's profile into shared memory, every group aligns its
// sequence against it (Alg. 6 per column, as in the per-query kernels), and
// the chunk boundary row -- the corrected H - o and the F leaving the chunk,
// per reference column, 8 bytes -- goes to the group's own slot of max_len
// columns in global memory (a few KB per group in practice, so it stays in
// L2) instead of a row of every database residue per query.  The score is
// the maximum over the chunks.
//
// That is the fused-chunk kernel, for queries of more than one chunk.
// Single-chunk queries run the phase kernel below instead, whose inner loop
// is the per-query kernel's (measured 5-20 % faster than the fused-chunk
// structure on those layouts).
//
// Overflow: the packed launches score every pair; a packed lane's running
// maximum never decreases, so a pair whose value left the lane range ends at
// or above the rescore threshold.  Only pairs with min(m, n) >= skip_len (the
// threshold over max(M); an alignment of m x n cells scores at most
// max(M) * min(m, n)) can get there: the longest database sequences against
// the longest queries, a prefix of the length order.  A second launch on
// int32 lanes walks exactly those candidates and rescores the ones whose
// packed score reached the threshold, skipping units that have none.
#pragma once
#include <cuda/atomic>

#include "sw_split.cuh"

namespace swg {

constexpr unsigned MULTI_FULL = 0xffffffffu;

// The unit counter is fetched by one thread and broadcast through shared
// memory; every thread reads it before the chunk-0 staging barrier, so the
// next fetch (after the loop's top barrier) cannot overwrite an unread value.
template <int L, int S, bool D0, bool AC>
__global__ void __launch_bounds__(BATCH_THREADS, SplitMinBlocks<S, D0, false, AC>::value)
    sw_multi_split_kernel(const MultiArgs p)
{
    constexpr int G = 32 / L;
    constexpr int GPC = (BATCH_THREADS / 32) * G;
    constexpr int SP = SegPad<S, 4>::value;
    constexpr int QH = L * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sprof = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ unsigned long long s_unit;

    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = (int)(threadIdx.x >> 5) * G + lane / L;
    const int K = p.k_items;
    const int64_t per_tile = (int64_t)GPC * K;
    const int64_t n_tiles = (p.n_items + per_tile - 1) / per_tile;
    const int64_t n_units = n_tiles * p.n_queries;
    const int pb = split_pb<D0>(p.o);
    const LaneQ16::K k = LaneQ16::consts_pb(p.o, p.e, S, p.one, pb);
    int2 *bnd = p.bnd ? reinterpret_cast<int2 *>(p.bnd + ((int64_t)blockIdx.x * GPC + grp) * p.bnd_stride) : nullptr;
    const int total = (p.A + 2) * L * SP;

    // stage chunk c of query Q: virtual lanes l and L + l paired in one
    // word; row A: an unknown residue (the smallest entry), row A+1: inert
    auto stage = [&](const MultiQuery &Q, int c) {
        const int8_t *gprof = Q.prof + (size_t)c * p.A * 2 * QH;
        const int qbase = c * 2 * QH;
        for (int idx = threadIdx.x; idx < total; idx += BATCH_THREADS) {
            const int a = idx / (L * SP);
            const int rem = idx - a * (L * SP);
            const int l = rem / SP;
            const int j = rem - l * SP;
            int lo = LaneQ16::PAD, hi = LaneQ16::PAD;
            if (a <= p.A && j < S) {
                const int plo = l * S + j, phi = QH + l * S + j;
                if (qbase + plo < Q.qlen)
                    lo = (a < p.A ? (int)gprof[(size_t)a * 2 * QH + plo] : (int)p.min_m) + pb;
                if (qbase + phi < Q.qlen)
                    hi = (a < p.A ? (int)gprof[(size_t)a * 2 * QH + phi] : (int)p.min_m) + pb;
            }
            sprof[((a * (SP / 4) + j / 4) * L + l) * 4 + (j % 4)] =
                (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
        }
    };

    for (;;) {
        if (threadIdx.x == 0)
            s_unit = atomicAdd(p.counter, 1ull);
        __syncthreads();  // s_unit visible; every group done with the last unit's profile
        const int64_t u = (int64_t)s_unit;
        if (u >= n_units)
            break;
        const int64_t t = u / p.n_queries;
        const MultiQuery Q = p.queries[u - t * p.n_queries];
        for (int kk = 0; kk < K; ++kk) {
            const int64_t w = t * per_tile + (int64_t)kk * GPC + grp;
            int seq = w < p.n_items ? p.order[w] : -1;
            int64_t start = 0;
            int len = 0;
            if (seq >= 0) {
                start = p.off[seq];
                len = (int)(p.off[seq + 1] - start);
            }
            const int ncols = (int)__reduce_max_sync(MULTI_FULL, (unsigned)len);
            int best = 0;
            for (int c = 0; c < Q.C; ++c) {
                if (Q.C > 1 || kk == 0) {  // a single-chunk profile is staged once per unit
                    if (kk > 0 || c > 0)
                        __syncthreads();  // every group is done with the staged profile
                    stage(Q, c);
                    __syncthreads();
                }
                const uint32_t mx = split_unit<L, S, D0, false, false, AC>(sprof, p.db, start, len, ncols, p.A,
                                                                           p.o, p.e, p.one, c > 0, c + 1 < Q.C, bnd,
                                                                           gl, nullptr, nullptr, nullptr, 0);
                best = max(best, LaneQ16::score(mx, 0, k));
            }
            if (gl == 0 && seq >= 0)
                p.scores[Q.row * p.row_stride + seq] = best;
        }
    }
}

// Single-chunk queries: every CTA walks the queries in order.  For each one
// whose items are not all taken yet it stages the profile once, and its
// warps pull sequences from that query's own counter exactly as the
// per-query kernel does (longest first, no barrier between sequences); the
// CTA's warps meet at a barrier only when the query's sequences run out,
// where the remaining ones are the shortest.  Per query the work is the
// per-query kernel's, without a launch or a tail of its own.
template <int L, int S, bool D0, bool AC>
__global__ void __launch_bounds__(BATCH_THREADS, SplitMinBlocks<S, D0, false, AC>::value)
    sw_multi_phase_kernel(const MultiArgs p)
{
    constexpr int G = 32 / L;
    constexpr int SP = SegPad<S, 4>::value;
    constexpr int QH = L * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sprof = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ int s_skip;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const int pb = split_pb<D0>(p.o);
    const LaneQ16::K k = LaneQ16::consts_pb(p.o, p.e, S, p.one, pb);
    const int total = (p.A + 2) * L * SP;
    for (int qi = 0; qi < p.n_queries; ++qi) {
        __syncthreads();  // every warp is done with the previous query's profile
        if (threadIdx.x == 0)
            s_skip = *reinterpret_cast<volatile unsigned long long *>(p.counter + qi) >=
                     (unsigned long long)p.n_items;
        __syncthreads();
        if (s_skip)
            continue;  // its sequences are all taken
        const MultiQuery Q = p.queries[qi];
        // stage the profile: virtual lanes l and L + l paired in one word;
        // row A: an unknown residue (the smallest entry), row A+1: inert
        for (int idx = threadIdx.x; idx < total; idx += BATCH_THREADS) {
            const int a = idx / (L * SP);
            const int rem = idx - a * (L * SP);
            const int l = rem / SP;
            const int j = rem - l * SP;
            int lo = LaneQ16::PAD, hi = LaneQ16::PAD;
            if (a <= p.A && j < S) {
                const int plo = l * S + j, phi = QH + l * S + j;
                if (plo < Q.qlen)
                    lo = (a < p.A ? (int)Q.prof[(size_t)a * 2 * QH + plo] : (int)p.min_m) + pb;
                if (phi < Q.qlen)
                    hi = (a < p.A ? (int)Q.prof[(size_t)a * 2 * QH + phi] : (int)p.min_m) + pb;
            }
            sprof[((a * (SP / 4) + j / 4) * L + l) * 4 + (j % 4)] =
                (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
        }
        __syncthreads();
        int32_t *scores = p.scores + Q.row * p.row_stride;
        for (;;) {
            unsigned long long ubase = 0;
            if (lane == 0)
                ubase = atomicAdd(p.counter + qi, (unsigned long long)G);
            ubase = __shfl_sync(MULTI_FULL, ubase, 0);
            if ((int64_t)ubase >= p.n_items)
                break;
            const int64_t w = (int64_t)ubase + grp;
            int seq = w < p.n_items ? p.order[w] : -1;
            const int64_t start = seq >= 0 ? p.off[seq] : 0;
            const int len = seq >= 0 ? (int)(p.off[seq + 1] - start) : 0;
            const int ncols = (int)__reduce_max_sync(MULTI_FULL, (unsigned)len);
            const uint32_t mx = split_unit<L, S, D0, false, false, AC>(sprof, p.db, start, len, ncols, p.A, p.o, p.e,
                                                                       p.one, false, false, nullptr, gl);
            if (gl == 0 && seq >= 0)
                scores[seq] = LaneQ16::score(mx, 0, k);
        }
    }
}

// Queries of several chunks: the phase walk over (query, chunk) phases.
// Every CTA walks the phases in order (query by query, chunk by chunk),
// stages each phase's profile chunk once and pulls its sequences, longest
// first, from the phase's own counter, as the per-query chunk launches do.
// The chunk boundary rows are one row of every database residue, reused by
// every query: phase (q, c) reads what (q, c - 1) wrote and writes what
// (q, c + 1) reads, in place, as the per-query launches do.  Each sequence
// of the order carries the last phase that finished it: before a group
// aligns sequence w in phase P it waits until w is done with phase P - 1
// (acquire), and after it, publishes P (release, after the boundary row and
// the score).  A CTA enters phase P only once P - 1's counter is exhausted,
// so every sequence of P - 1 is already held by a resident warp of another
// CTA (this CTA's warps finished theirs at the phase barrier), and as both
// phases run longest first, P reaches a sequence long after P - 1 finished
// it: the wait is a formality with no cycle.  It is bounded all the same
// (p.wait_limit polls of about 256 ns, a second by default), after which the
// group sets the status word and goes on; once the word is set, later waits
// give up at their first poll, so a launch that lost a mark still ends in
// about a second.

// waits (acquire) until *mark >= need, at most `limit` polls; sets the
// status word when it gives up, and gives up at once when the word is set.
// Kept out of line: inlined, it changed the register allocation of the
// kernel's cell loop (more spills on the 64 x 40 layout).
static __device__ __noinline__ void multi_wait_mark(int32_t *mark, int need, int limit, int32_t *status)
{
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> d(*mark);
    int it = 0;
    while (d.load(cuda::memory_order_acquire) < need) {
        if (++it > limit || *reinterpret_cast<volatile int32_t *>(status) != 0) {
            atomicExch(status, 1);
            return;
        }
        __nanosleep(256);
    }
}

// reads a CTA-uniform value parked in shared memory afresh at each use, so
// that it holds no register across the cell loop
__device__ __forceinline__ int multi_uniform(const int &v) { return *reinterpret_cast<const volatile int *>(&v); }

template <int L, int S, bool D0, bool AC>
__global__ void __launch_bounds__(BATCH_THREADS, SplitMinBlocks<S, D0, false, AC>::value)
    sw_multi_chunks_kernel(const MultiArgs p)
{
    constexpr int G = 32 / L;
    constexpr int SP = SegPad<S, 4>::value;
    constexpr int QH = L * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sprof = reinterpret_cast<uint32_t *>(smem_raw);
    // the walk's state and the phase's query, kept in shared memory: the
    // cell loop needs every register (the S = 40 layouts spilled with the
    // query in registers, and loop state held across it costs moves)
    __shared__ MultiQuery s_q;
    __shared__ int s_phase, s_chunk, s_nchunks, s_query;
    // each group's item and sequence, parked over the cell loop
    __shared__ long long s_w[(BATCH_THREADS / 32) * G];
    __shared__ int s_seq[(BATCH_THREADS / 32) * G];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const int gslot = (int)(threadIdx.x >> 5) * G + grp;
    if (threadIdx.x == 0) {
        s_phase = -1;  // before the first phase: chunk -1 of a query of no chunks
        s_chunk = -1;
        s_nchunks = 0;
        s_query = -1;
    }
    for (;;) {
        __syncthreads();  // every warp is done with the previous phase's profile and record
        if (threadIdx.x == 0) {
            // the next phase whose sequences are not all taken
            int ph = s_phase, c = s_chunk, nc = s_nchunks, qi = s_query;
            for (;;) {
                ++ph;
                if (++c >= nc) {
                    c = 0;
                    if (++qi >= p.n_queries)
                        break;
                    s_q = p.queries[qi];
                    nc = s_q.C;
                    if (nc < 1) {
                        --ph;  // a query of no chunks has no phase
                        c = -1;
                        nc = 0;
                        continue;
                    }
                }
                if (*reinterpret_cast<volatile unsigned long long *>(p.counter + ph) < (unsigned long long)p.n_items)
                    break;
            }
            s_phase = ph;
            s_chunk = c;
            s_nchunks = nc;
            s_query = qi;
        }
        __syncthreads();
        if (s_query >= p.n_queries)
            break;
        // stage chunk c: virtual lanes l and L + l paired in one word;
        // row A: an unknown residue (the smallest entry), row A+1: inert
        {
            const int c = s_chunk;
            const int pb = split_pb<D0>(p.o);
            const int total = (p.A + 2) * L * SP;
            const int8_t *gprof = s_q.prof + (size_t)c * p.A * 2 * QH;
            const int qbase = c * 2 * QH;
            const int qlen = s_q.qlen;
            for (int idx = threadIdx.x; idx < total; idx += BATCH_THREADS) {
                const int a = idx / (L * SP);
                const int rem = idx - a * (L * SP);
                const int l = rem / SP;
                const int j = rem - l * SP;
                int lo = LaneQ16::PAD, hi = LaneQ16::PAD;
                if (a <= p.A && j < S) {
                    const int plo = l * S + j, phi = QH + l * S + j;
                    if (qbase + plo < qlen)
                        lo = (a < p.A ? (int)gprof[(size_t)a * 2 * QH + plo] : (int)p.min_m) + pb;
                    if (qbase + phi < qlen)
                        hi = (a < p.A ? (int)gprof[(size_t)a * 2 * QH + phi] : (int)p.min_m) + pb;
                }
                sprof[((a * (SP / 4) + j / 4) * L + l) * 4 + (j % 4)] =
                    (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
            }
        }
        __syncthreads();
        const bool has_prev = s_chunk > 0, has_next = s_chunk + 1 < s_nchunks;
        for (;;) {
            const int phase = multi_uniform(s_phase);
            unsigned long long ubase = 0;
            if (lane == 0)
                ubase = atomicAdd(p.counter + phase, (unsigned long long)G);
            ubase = __shfl_sync(MULTI_FULL, ubase, 0);
            if ((int64_t)ubase >= p.n_items)
                break;
            const int64_t w = (int64_t)ubase + grp;
            const int seq = w < p.n_items ? p.order[w] : -1;
            const int64_t start = seq >= 0 ? p.off[seq] : 0;
            const int len = seq >= 0 ? (int)(p.off[seq + 1] - start) : 0;
            // wait until this sequence is done with the previous phase
            if (w < p.n_items && phase > 0 && gl == 0)
                multi_wait_mark(p.done + w, phase - 1 + p.wait_skew, p.wait_limit, p.status);
            if (gl == 0) {
                s_w[gslot] = w < p.n_items ? w : -1;
                s_seq[gslot] = seq;
            }
            __syncwarp(MULTI_FULL);
            const int ncols = (int)__reduce_max_sync(MULTI_FULL, (unsigned)len);
            const uint32_t mx = split_unit<L, S, D0, false, false, AC>(sprof, p.db, start, len, ncols, p.A, p.o, p.e,
                                                                       p.one, has_prev, has_next, p.rows, gl);
            __syncwarp(MULTI_FULL);  // the group's boundary-row stores come before the mark
            if (gl == 0) {
                const long long wi = s_w[gslot];
                const int sq = s_seq[gslot];
                const int c2 = multi_uniform(s_chunk);
                if (sq >= 0) {
                    // the maximum over the chunks so far (chunk c - 1 wrote
                    // before it published its mark); h-space bias BX + pb - o
                    const int sc = max((int)(int16_t)(mx & 0xffffu), (int)(int16_t)(mx >> 16)) -
                                   (LaneQ16::BX + split_pb<D0>(p.o) - p.o);
                    int32_t *dst = p.scores + s_q.row * p.row_stride + sq;
                    *dst = c2 > 0 ? max(sc, *dst) : sc;
                }
                if (wi >= 0) {
                    __threadfence();
                    cuda::atomic_ref<int32_t, cuda::thread_scope_device> d(p.done[wi]);
                    // the phase from shared memory again, except on the 32 x 40
                    // layout, whose register allocation spilled that way (the
                    // allocation at 128 registers shifts with any change)
                    d.store((L == 16 && S == 40) ? phase : multi_uniform(s_phase), cuda::memory_order_release);
                }
            }
        }
    }
}

// int32 lanes, 32 lanes per alignment: the candidates that could overflow
// the packed lanes (min(m, n) >= skip_len, over the first n_items entries
// of the order) whose packed score reached the rescore threshold; a unit
// with none of them is skipped before its profile is staged.
template <class LT, int S>
__global__ void __launch_bounds__(BATCH_THREADS) sw_multi_i32_kernel(const MultiArgs p)
{
    constexpr int L = 32;
    constexpr int GPC = BATCH_THREADS / 32;
    constexpr int QC = L * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *sprof = reinterpret_cast<int32_t *>(smem_raw);
    __shared__ unsigned long long s_unit;

    const int gl = threadIdx.x & 31;
    const int grp = (int)(threadIdx.x >> 5);
    const int64_t n_tiles = (p.n_items + GPC - 1) / GPC;
    const int64_t n_units = n_tiles * p.n_queries;
    int2 *bnd = p.bnd ? reinterpret_cast<int2 *>(p.bnd + ((int64_t)blockIdx.x * GPC + grp) * p.bnd_stride) : nullptr;
    const int32_t *pbase[1] = {sprof};
    const int64_t bstart[1] = {0};
    unsigned long long lazy_steps = 0;

    for (;;) {
        if (threadIdx.x == 0)
            s_unit = atomicAdd(p.counter, 1ull);
        __syncthreads();
        const int64_t u = (int64_t)s_unit;
        if (u >= n_units)
            break;
        const int64_t t = u / p.n_queries;
        const MultiQuery Q = p.queries[u - t * p.n_queries];
        const int64_t w = t * GPC + grp;
        int seq = w < p.n_items ? p.order[w] : -1;
        int64_t start[1] = {0};
        int len[1] = {0};
        if (seq >= 0) {
            start[0] = p.off[seq];
            len[0] = (int)(p.off[seq + 1] - start[0]);
            // a candidate whose packed score stayed below the threshold is exact
            if (!(Q.qlen >= p.skip_len && len[0] >= p.skip_len) ||
                p.scores[Q.row * p.row_stride + seq] < p.flag_thresh) {
                seq = -1;
                len[0] = 0;
            }
        }
        if (!__syncthreads_or(seq >= 0))
            continue;  // nothing to rescore in this unit
        const int ncols = (int)__reduce_max_sync(MULTI_FULL, (unsigned)len[0]);
        int best = 0;
        for (int c = 0; c < Q.C; ++c) {
            if (c > 0)
                __syncthreads();
            const int8_t *gprof = Q.prof + (size_t)c * p.A * QC;
            const int qbase = c * QC;
            stage_profile<LT, L, S>(sprof, p.A, p.o, threadIdx.x, BATCH_THREADS, [&](int a, int l, int j) {
                if (qbase + l * S + j >= Q.qlen)
                    return -1024;
                return a < p.A ? (int)gprof[(size_t)a * QC + l * S + j] : (int)p.min_m;
            });
            __syncthreads();
            const int32_t mx = striped_unit<LT, L, S, false>(pbase, p.db, start, len, ncols, p.A, p.o, p.e, p.one,
                                                             c > 0, c + 1 < Q.C, bnd, gl, lazy_steps, nullptr,
                                                             nullptr, bstart);
            best = max(best, (int)mx);
        }
        if (gl == 0 && seq >= 0)
            p.scores[Q.row * p.row_stride + seq] = best;
    }
}

}  // namespace swg
