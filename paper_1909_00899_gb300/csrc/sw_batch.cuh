// Striped Smith-Waterman/Gotoh batch kernel: one query chunk against many
// database sequences.
//
// Layout (Alg. 1, Alg. 6): an alignment is owned by a group of L lanes of a
// warp (the paper's p vector lanes); lane l holds query positions
// l*S .. l*S+S-1 of the chunk (S = segLen) in registers: Ho[j] = H - o of
// the previous reference column and E[j].  A warp carries 32/L groups, each
// on its own database sequence (or 2 / 4 sequences for packed lanes).
//
// Per reference column (the paper's outer loop over i):
//   1. the residue is broadcast from a coalesced block load, the profile row
//      comes from shared memory (16-byte vector loads, conflict-free layout);
//   2. the diagonal for position 0 is lane l-1's last H of the previous
//      column ("HStore[segLen-1] <<< 1"), a width-L shuffle;
//   3. the segment pass computes H, E and F with F starting at 0 in every
//      lane (Alg. 6 main loop).  With stored X = H - o and the profile biased
//      by +o, one cell is
//          h  = max(Xd + P', E, 0)        (H before F; Max is taken on it)
//          ho = h - o
//          X  = max(F - o, ho)            (= H - o with H = max(h, F))
//          E' = max(E - e, X)             (next column)
//          F' = max(F - e, ho)            (next position; F - o is dominated
//                                          because e <= o)
//   4. the F leaving each lane enters the max-plus prefix scan over lanes
//      with weight S*e per hop (Alg. 4-6; log2 L shuffle steps instead of
//      the p-step loop): carry[l] = max_k<l (Fout[k] - (l-1-k)*S*e);
//   5. the carry is not applied now: the next column's pass raises the
//      previous H at position j (its diagonal) and E[j] by carry - o - j*e
//      before use (Alg. 6, "executed even lazier"), and the last element is
//      raised before the shuffle of step 2.  The raise of E is the reading
//      that keeps textbook Gotoh (a carried vertical gap may be followed by a
//      horizontal one); a warp-uniform test skips the raise when no lane has
//      a positive carry.
// The lazy-F variant (Alg. 1) instead runs up to L rounds of
// shift-and-correct after the pass and leaves as soon as, in every lane, the
// carried F after the extend step is <= the uncorrected H - o at that
// position.
//
// Long queries run as C chunks of L*S positions, one launch per chunk: the
// last lane of chunk c writes, per reference column, its corrected H - o and
// the F leaving the chunk; lane 0 of chunk c+1 takes them as its diagonal
// and incoming F.
#pragma once
#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swg {

constexpr int BATCH_THREADS = 256;

template <int S, int V>
struct SegPad {
    static constexpr int value = (S + V - 1) / V * V;
};

// One work unit (CELLS alignments, one query chunk) on a group of L lanes.
// pbase[c]: staged profile of cell c (biased by +o); ref + start[c]: the
// reference residues of cell c, len[c] of them; ncols: warp-uniform number
// of columns to run (max over the warp).  Returns the group's packed
// maximum of H.
template <class LT, int L, int S, bool LAZY>
__device__ __forceinline__ typename LT::T striped_unit(const typename LT::Elem *const *pbase, const uint8_t *ref,
                                                        const int64_t *start, const int *len, int ncols, int A,
                                                        int o, int e, bool has_prev, bool has_next, int2 *bnd,
                                                        int gl, unsigned long long &lazy_steps)
{
    using T = typename LT::T;
    constexpr int CELLS = LT::CELLS;
    constexpr int SP = SegPad<S, LT::VEC>::value;
    constexpr unsigned FULL = 0xffffffffu;

    const T negO = LT::splat(-o);
    const T negE = LT::splat(-e);
    const T negS1 = LT::splat(-(S - 1) * e);

    T Ho[S], E[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        Ho[j] = negO;
        E[j] = LT::zero();
    }
    T c_prev = LT::zero();  // carry into this lane from the previous column
    T hlast = negO;         // corrected H - o of the last position, previous column
    T hb_prev = negO;       // previous chunk's last H - o at the previous column
    T mx = LT::zero();

    for (int r0 = 0; r0 < ncols; r0 += L) {
        int myres[CELLS];
        int2 mybnd[CELLS];
#pragma unroll
        for (int c = 0; c < CELLS; ++c) {
            const int r = r0 + gl;
            // codes >= A read as the inert row A (never out of the staged profile)
            myres[c] = r < len[c] ? min((int)ref[start[c] + r], A) : A;
            mybnd[c] = make_int2(-o, 0);
            if (has_prev && r < len[c])
                mybnd[c] = bnd[start[c] + r];
        }
        const int cols = min(L, ncols - r0);
        for (int rr = 0; rr < cols; ++rr) {
            const int r = r0 + rr;
            int res[CELLS];
#pragma unroll
            for (int c = 0; c < CELLS; ++c)
                res[c] = __shfl_sync(FULL, myres[c], rr, L);
            T P[S];
            LT::template load_profile<L, S, SP>(pbase, res, gl, P);

            T hd = LT::shfl_up(hlast, 1, L);
            T F = LT::zero();
            if (has_prev) {
                int bh[CELLS], bf[CELLS];
#pragma unroll
                for (int c = 0; c < CELLS; ++c) {
                    bh[c] = __shfl_sync(FULL, mybnd[c].x, rr, L);
                    bf[c] = __shfl_sync(FULL, mybnd[c].y, rr, L);
                }
                if (gl == 0) {
                    hd = hb_prev;
                    F = LT::pack(bf);
                }
                hb_prev = LT::pack(bh);
            } else if (gl == 0) {
                hd = negO;
            }

            if constexpr (!LAZY) {
                if (__any_sync(FULL, LT::any_pos(c_prev))) {
                    // deferred correction by the previous column's carry
                    T d = LT::add(c_prev, negO);
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const T Ej = LT::max2(E[j], d);
                        const T h = LT::addmax_relu(hd, P[j], Ej);
                        hd = LT::max2(Ho[j], d);
                        d = LT::add(d, negE);
                        const T ho = LT::add(h, negO);
                        Ho[j] = LT::addmax(F, negO, ho);
                        E[j] = LT::addmax(Ej, negE, Ho[j]);
                        F = LT::addmax(F, negE, ho);
                        mx = LT::max2(mx, h);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const T h = LT::addmax_relu(hd, P[j], E[j]);
                        hd = Ho[j];
                        const T ho = LT::add(h, negO);
                        Ho[j] = LT::addmax(F, negO, ho);
                        E[j] = LT::addmax(E[j], negE, Ho[j]);
                        F = LT::addmax(F, negE, ho);
                        mx = LT::max2(mx, h);
                    }
                }
                // max-plus prefix scan of the F leaving each lane
                T x = F;
#pragma unroll
                for (int dd = 1; dd < L; dd <<= 1) {
                    const T y = LT::shfl_up(x, dd, L);
                    x = LT::addmax(y, LT::splat(-dd * S * e), x);
                }
                T cin = LT::shfl_up(x, 1, L);
                if (gl == 0)
                    cin = LT::zero();
                c_prev = cin;
                // two adds: each constant stays inside the lane range, so a
                // saturating lane floors at -128 instead of wrapping
                hlast = LT::max2(Ho[S - 1], LT::add(LT::add(cin, negO), negS1));
                if (has_next && gl == L - 1) {
#pragma unroll
                    for (int c = 0; c < CELLS; ++c)
                        if (r < len[c])
                            bnd[start[c] + r] = make_int2(LT::get(hlast, c), LT::get(x, c));
                }
            } else {
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const T h = LT::addmax_relu(hd, P[j], E[j]);
                    hd = Ho[j];
                    const T ho = LT::add(h, negO);
                    Ho[j] = LT::addmax(F, negO, ho);
                    E[j] = LT::addmax(E[j], negE, Ho[j]);
                    F = LT::addmax(F, negE, ho);
                    mx = LT::max2(mx, h);
                }
                // lazy-F: shift the carry into the next lane and correct
                T fb = F;  // F leaving this lane, corrected as rounds pass
                T Fc = LT::shfl_up(F, 1, L);
                if (gl == 0)
                    Fc = LT::zero();
                bool done = false;
                for (int k = 0; k < L && !done; ++k) {
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const T hold = Ho[j];
                        Ho[j] = LT::addmax(Fc, negO, hold);
                        E[j] = LT::max2(E[j], Ho[j]);
                        Fc = LT::add(Fc, negE);
                        ++lazy_steps;
                        if (__all_sync(FULL, Fc <= max(hold, 0))) {
                            done = true;
                            break;
                        }
                    }
                    if (!done) {
                        fb = LT::max2(fb, Fc);
                        Fc = LT::shfl_up(Fc, 1, L);
                        if (gl == 0)
                            Fc = LT::zero();
                    }
                }
                hlast = Ho[S - 1];
                if (has_next && gl == L - 1 && r < len[0])
                    bnd[start[0] + r] = make_int2(LT::get(hlast, 0), LT::get(fb, 0));
            }
        }
    }
#pragma unroll
    for (int dd = L / 2; dd >= 1; dd >>= 1)
        mx = LT::max2(mx, LT::shfl_xor(mx, dd, L));
    return mx;
}

// Stage one striped profile (biased by +o) into shared memory in the layout
// load_profile reads: [residue][SP / VEC][lane][VEC].  value(a, l, j) gives
// the raw score of residue a at lane l, segment index j (j < S) or a
// sentinel below -256 for positions past the query end; row A is inert.
template <class LT, int L, int S, class ValueFn>
__device__ __forceinline__ void stage_profile(typename LT::Elem *dst, int A, int o, int tid, int nthreads,
                                              ValueFn value)
{
    constexpr int V = LT::VEC;
    constexpr int SP = SegPad<S, V>::value;
    const int total = (A + 1) * L * SP;
    for (int idx = tid; idx < total; idx += nthreads) {
        const int a = idx / (L * SP);
        const int rem = idx - a * (L * SP);
        const int l = rem / SP;
        const int j = rem - l * SP;
        int v = LT::PAD;
        if (a < A && j < S) {
            const int raw = value(a, l, j);
            if (raw > -256)
                v = raw + o;
        }
        dst[((a * (SP / V) + j / V) * L + l) * V + (j % V)] = (typename LT::Elem)v;
    }
}

template <class LT, int L, int S, bool LAZY>
__global__ void __launch_bounds__(BATCH_THREADS) sw_batch_kernel(const BatchArgs p)
{
    using T = typename LT::T;
    using Elem = typename LT::Elem;
    constexpr int CELLS = LT::CELLS;
    constexpr int G = 32 / L;
    constexpr int QC = L * S;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(L >= 2 && L <= 32 && (L & (L - 1)) == 0, "lanes per alignment: power of two");
    static_assert(!LAZY || CELLS == 1, "lazy-F kernel uses int32 lanes");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Elem *sprof = reinterpret_cast<Elem *>(smem_raw);

    const int8_t *gprof = p.prof + (size_t)p.chunk * p.A * QC;
    const int qbase = p.chunk * QC;
    const int qlen = p.qlen;
    stage_profile<LT, L, S>(sprof, p.A, p.o, threadIdx.x, blockDim.x, [&](int a, int l, int j) {
        return qbase + l * S + j < qlen ? (int)gprof[(size_t)a * QC + l * S + j] : -1024;
    });
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const int64_t n_work = p.n_work_dev ? (int64_t)(*p.n_work_dev) : p.n_work;
    const int64_t units = (n_work + CELLS - 1) / CELLS;
    const bool has_prev = p.chunk > 0;
    const bool has_next = p.chunk + 1 < p.nchunks;
    const Elem *pbase[CELLS];
#pragma unroll
    for (int c = 0; c < CELLS; ++c)
        pbase[c] = sprof;
    unsigned long long lazy_steps = 0;

    for (;;) {
        unsigned int ubase = 0;
        if (lane == 0)
            ubase = atomicAdd(p.counter, (unsigned int)G);
        ubase = __shfl_sync(FULL, ubase, 0);
        if ((int64_t)ubase >= units)
            break;
        const int64_t unit = (int64_t)ubase + grp;
        int seq[CELLS];
        int64_t start[CELLS];
        int len[CELLS];
        int my_n = 0;
#pragma unroll
        for (int c = 0; c < CELLS; ++c) {
            const int64_t w = unit * CELLS + c;
            const bool ok = unit < units && w < n_work;
            seq[c] = ok ? (p.order ? p.order[w] : (int)w) : -1;
            start[c] = ok ? p.off[seq[c]] : 0;
            len[c] = ok ? (int)(p.off[seq[c] + 1] - start[c]) : 0;
            my_n = max(my_n, len[c]);
        }
        const int ncols = (int)__reduce_max_sync(FULL, (unsigned)my_n);
        const T mx = striped_unit<LT, L, S, LAZY>(pbase, p.db, start, len, ncols, p.A, p.o, p.e, has_prev,
                                                  has_next, p.bnd, gl, lazy_steps);
        if (gl == 0) {
#pragma unroll
            for (int c = 0; c < CELLS; ++c) {
                if (seq[c] >= 0) {
                    int s = LT::get(mx, c);
                    if (has_prev)
                        s = max(s, p.scores[seq[c]]);
                    p.scores[seq[c]] = s;
                }
            }
        }
    }
    // j-steps of the correction loop, counted once per warp
    if (LAZY && p.lazy_steps && lane == 0 && lazy_steps)
        atomicAdd(p.lazy_steps, lazy_steps);
}

}  // namespace swg
