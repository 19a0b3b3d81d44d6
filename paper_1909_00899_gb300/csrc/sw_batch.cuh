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
// pbase[c]: staged profile of cell c; ref + start[c]: the reference residues
// of cell c, len[c] of them; ncols: warp-uniform number of columns to run
// (max over the warp).  Returns the group's packed maximum of h (h-space).
// ENDS (int32 lanes only): also track, per lane, the first cell (column
// order) where the lane's maximum was reached, and reduce the group's best
// end cell into end_r / end_q (0-based reference column and position in the
// chunk, -1 when nothing scored above 0): larger score first, then smaller
// reference position, then smaller query position.
template <class LT, int L, int S, bool LAZY, bool ENDS = false>
__device__ __forceinline__ typename LT::T striped_unit(const typename LT::Elem *const *pbase, const uint8_t *ref,
                                                        const int64_t *start, const int *len, int ncols, int A,
                                                        int o, int e, uint32_t one, bool has_prev, bool has_next,
                                                        int2 *bnd, int gl, unsigned long long &lazy_steps,
                                                        int *end_r = nullptr, int *end_q = nullptr,
                                                        const int64_t *bstart = nullptr)
{
    // boundary rows are indexed from bstart[c] (default: the residues' start)
    const int64_t *bs = bstart ? bstart : start;
    using T = typename LT::T;
    constexpr int CELLS = LT::CELLS;
    constexpr int SP = SegPad<S, LT::VEC>::value;
    constexpr int LOGL = L == 1 ? 0 : L == 2 ? 1 : L == 4 ? 2 : L == 8 ? 3 : L == 16 ? 4 : 5;
    constexpr unsigned FULL = 0xffffffffu;

    const typename LT::K k = LT::consts(o, e, S, one);
    T negW[LOGL > 0 ? LOGL : 1];  // scan hop weights -(2^i)*S*e (none for one lane)
#pragma unroll
    for (int i = 0; i < LOGL; ++i)
        negW[i] = LT::splat(-(1 << i) * S * e);

    T X[S], E[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        X[j] = k.xinit;
        E[j] = k.hzero;
    }
    T c_prev = k.xzero;   // carry into this lane from the previous column
    T hlast = k.xinit;    // corrected X of the last position, previous column
    T hb_prev = k.xinit;  // previous chunk's last X at the previous column
    T mx = k.hzero;
    static_assert(!ENDS || (LT::CELLS == 1 && !LAZY), "end cells: int32 scan-F only");
    int best_r = -1, best_j = 0;  // first cell of this lane's maximum (ENDS)

    for (int r0 = 0; r0 < ncols; r0 += L) {
        int myres[CELLS];
        int2 mybnd[CELLS];
#pragma unroll
        for (int c = 0; c < CELLS; ++c) {
            const int r = r0 + gl;
            // codes >= A read as the unknown-residue row A; columns past the
            // sequence end read the inert row A+1
            myres[c] = r < len[c] ? min((int)ref[start[c] + r], A) : A + 1;
            mybnd[c] = make_int2(-o, 0);
            if (has_prev && r < len[c])
                mybnd[c] = bnd[bs[c] + r];
        }
        const int cols = min(L, ncols - r0);
        for (int rr = 0; rr < cols; ++rr) {
            const int r = r0 + rr;
            int res[CELLS];
#pragma unroll
            for (int c = 0; c < CELLS; ++c)
                res[c] = __shfl_sync(FULL, myres[c], rr, L);
            // the profile is fetched one 16-byte vector (VEC positions) at a
            // time inside the position loops, so only VEC values are live
            constexpr int V = LT::VEC;
            T Pv[V];

            T hd = __shfl_up_sync(FULL, hlast, 1, L);
            T F = k.xzero;
            if (has_prev) {
                int bh[CELLS], bf[CELLS];
#pragma unroll
                for (int c = 0; c < CELLS; ++c) {
                    bh[c] = __shfl_sync(FULL, mybnd[c].x, rr, L);
                    bf[c] = __shfl_sync(FULL, mybnd[c].y, rr, L);
                }
                if (gl == 0) {
                    hd = hb_prev;
                    F = LT::x_pack(bf);
                }
                hb_prev = LT::x_pack(bh);
            } else if (gl == 0) {
                hd = k.xinit;
            }

            T hpair = k.hzero;  // h of the previous (even) position, for vimax3
            if constexpr (!LAZY) {
                if (__any_sync(FULL, LT::carry_pos(c_prev, k))) {
                    // deferred correction by the previous column's carry:
                    // d_j = carry - o - j*e raises E[j] and the diagonal
                    T d = LT::d0_of(c_prev, k);
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        if (j % V == 0)
                            LT::template load_vec<L, SP>(pbase, res, gl, j / V, Pv);
                        T h;
                        if constexpr (LT::D0) {
                            // d_j is dominated in h by the raised diagonal
                            h = LT::h_of(hd, Pv[j % V], E[j], k);
                            hd = LT::xd_corr(X[j], d, k);
                            d = LT::dstep(d, k);
                            const T ho = LT::ho_of(h, k);
                            X[j] = LT::addmax(F, k.negO, ho);
                            E[j] = LT::e_next_corr(E[j], d, X[j], k);
                            F = LT::addmax(F, k.negE, ho);
                        } else {
                            const T Ej = LT::max2(E[j], d);
                            h = LT::h_of(hd, Pv[j % V], Ej, k);
                            hd = LT::xd_corr(X[j], d, k);
                            d = LT::dstep(d, k);
                            const T ho = LT::ho_of(h, k);
                            X[j] = LT::addmax(F, k.negO, ho);
                            E[j] = LT::e_next(Ej, X[j], k);
                            F = LT::addmax(F, k.negE, ho);
                        }
                        if constexpr (ENDS) {
                            if (h > mx) {
                                mx = h;
                                best_r = r;
                                best_j = j;
                            }
                        } else if (j & 1) {
                            mx = LT::max3(mx, hpair, h);
                        } else if (j == S - 1) {
                            mx = LT::max2(mx, h);
                        } else {
                            hpair = h;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        if (j % V == 0)
                            LT::template load_vec<L, SP>(pbase, res, gl, j / V, Pv);
                        const T h = LT::h_of(hd, Pv[j % V], E[j], k);
                        hd = X[j];
                        const T ho = LT::ho_of(h, k);
                        X[j] = LT::addmax(F, k.negO, ho);
                        E[j] = LT::e_next(E[j], X[j], k);
                        F = LT::addmax(F, k.negE, ho);
                        if constexpr (ENDS) {
                            if (h > mx) {
                                mx = h;
                                best_r = r;
                                best_j = j;
                            }
                        } else if (j & 1) {
                            mx = LT::max3(mx, hpair, h);
                        } else if (j == S - 1) {
                            mx = LT::max2(mx, h);
                        } else {
                            hpair = h;
                        }
                    }
                }
                // max-plus prefix scan of the F leaving each lane (log2 L steps)
                T x = F;
#pragma unroll
                for (int i = 0; i < LOGL; ++i) {
                    const T y = __shfl_up_sync(FULL, x, 1 << i, L);
                    x = LT::addmax(y, negW[i], x);
                }
                T cin = __shfl_up_sync(FULL, x, 1, L);
                if (gl == 0)
                    cin = k.xzero;
                c_prev = cin;
                hlast = LT::last_corr(X[S - 1], cin, k);
                if (has_next && gl == L - 1) {
#pragma unroll
                    for (int c = 0; c < CELLS; ++c)
                        if (r < len[c])
                            bnd[bs[c] + r] = make_int2(LT::x_true(hlast, c), LT::x_true(x, c));
                }
            } else {
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    if (j % V == 0)
                        LT::template load_vec<L, SP>(pbase, res, gl, j / V, Pv);
                    const T h = LT::h_of(hd, Pv[j % V], E[j], k);
                    hd = X[j];
                    const T ho = LT::ho_of(h, k);
                    X[j] = LT::addmax(F, k.negO, ho);
                    E[j] = LT::e_next(E[j], X[j], k);
                    F = LT::addmax(F, k.negE, ho);
                    if (j & 1)
                        mx = LT::max3(mx, hpair, h);
                    else if (j == S - 1)
                        mx = LT::max2(mx, h);
                    else
                        hpair = h;
                }
                // lazy-F (Alg. 1): shift the carry into the next lane and
                // correct, for at most L rounds
                T fb = F;  // F leaving this lane, corrected as rounds pass
                T Fc = __shfl_up_sync(FULL, F, 1, L);
                if (gl == 0)
                    Fc = k.xzero;
                bool done = false;
                for (int kk = 0; kk < L && !done; ++kk) {
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const T hold = X[j];
                        X[j] = LT::addmax(Fc, k.negO, hold);
                        E[j] = LT::e_raise(E[j], X[j], k);
                        Fc = LT::lazy_step(Fc, k);  // plain add: this loop is latency-bound
                        ++lazy_steps;
                        if (__all_sync(FULL, LT::lazy_dominated(Fc, hold, k))) {
                            done = true;
                            break;
                        }
                    }
                    if (!done) {
                        fb = LT::max2(fb, Fc);
                        Fc = __shfl_up_sync(FULL, Fc, 1, L);
                        if (gl == 0)
                            Fc = k.xzero;
                    }
                }
                hlast = X[S - 1];
                if (has_next && gl == L - 1) {
#pragma unroll
                    for (int c = 0; c < CELLS; ++c)
                        if (r < len[c])
                            bnd[bs[c] + r] = make_int2(LT::x_true(hlast, c), LT::x_true(fb, c));
                }
            }
        }
    }
    if constexpr (ENDS) {
        int bq = gl * S + best_j;
#pragma unroll
        for (int dd = L / 2; dd >= 1; dd >>= 1) {
            const T om = __shfl_xor_sync(FULL, mx, dd, L);
            const int orr = __shfl_xor_sync(FULL, best_r, dd, L);
            const int oq = __shfl_xor_sync(FULL, bq, dd, L);
            if (om > mx || (om == mx && (orr < best_r || (orr == best_r && oq < bq)))) {
                mx = om;
                best_r = orr;
                bq = oq;
            }
        }
        *end_r = mx > 0 ? best_r : -1;
        *end_q = mx > 0 ? bq : -1;
    } else {
#pragma unroll
        for (int dd = L / 2; dd >= 1; dd >>= 1)
            mx = LT::max2(mx, __shfl_xor_sync(FULL, mx, dd, L));
    }
    return mx;
}

// Scores of one unit: lane results decoded to true values (combined with
// the previous chunks' maximum), and for lane types whose cells can leak
// into each other after an overflow, every cell of a register raised to
// the flag threshold once one of them reached it.
template <class LT>
__device__ __forceinline__ void write_scores(typename LT::T mx, const typename LT::K &k, const int *seq,
                                             bool has_prev, int32_t flag_thresh, int32_t *scores)
{
    constexpr int CELLS = LT::CELLS;
    int s[CELLS];
    bool flag = false;
#pragma unroll
    for (int c = 0; c < CELLS; ++c) {
        s[c] = LT::score(mx, c, k);
        if (seq[c] >= 0) {
            if (has_prev)
                s[c] = max(s[c], scores[seq[c]]);
            flag |= s[c] >= flag_thresh;
        }
    }
#pragma unroll
    for (int c = 0; c < CELLS; ++c) {
        if (seq[c] >= 0) {
            if (LT::CROSS && flag)
                s[c] = max(s[c], flag_thresh);
            scores[seq[c]] = s[c];
        }
    }
}

// write_scores for launches that split long sequences into pieces: an id
// with PIECE_BIT set is a piece, whose score joins its sequence's by
// atomicMax (single-chunk launches only, so nothing to combine from an
// earlier chunk).
template <class LT>
__device__ __forceinline__ void write_scores_pieces(typename LT::T mx, const typename LT::K &k, const int *id,
                                                    int32_t flag_thresh, int32_t *scores)
{
    constexpr int CELLS = LT::CELLS;
    int s[CELLS];
    bool flag = false;
#pragma unroll
    for (int c = 0; c < CELLS; ++c) {
        s[c] = LT::score(mx, c, k);
        if (id[c] >= 0)
            flag |= s[c] >= flag_thresh;
    }
#pragma unroll
    for (int c = 0; c < CELLS; ++c) {
        if (id[c] >= 0) {
            if (LT::CROSS && flag)
                s[c] = max(s[c], flag_thresh);
            if (id[c] & PIECE_BIT)
                atomicMax(&scores[id[c] & ~PIECE_BIT], s[c]);  // the sequence's best piece
            else
                scores[id[c]] = s[c];
        }
    }
}

// Work item w of a launch that splits long sequences: items [0, n_pieces)
// are pieces (id with PIECE_BIT), then the entries of order, skipping the
// sequences that were split (id -1: nothing to do).
struct BatchItem {
    int id;
    int64_t start;
    int len;
};

__device__ __forceinline__ BatchItem batch_item(const BatchArgs &p, int64_t w, int64_t n_work, int n_pieces)
{
    BatchItem it{-1, 0, 0};
    if (w >= n_work)
        return it;
    if (w < n_pieces) {
        const Piece pc = p.pieces[w];
        it.id = pc.seq | PIECE_BIT;
        it.start = pc.start;
        it.len = pc.len;
        return it;
    }
    const int64_t k = w - n_pieces;
    const int s = p.order ? p.order[k] : (int)k;
    if (p.split[s])
        return it;
    it.id = s;
    it.start = p.off[s];
    it.len = (int)(p.off[s + 1] - it.start);
    return it;
}

// Stage one striped profile (biased by the lane type's profile bias) into
// shared memory in the layout load_profile reads: [residue][SP/VEC][lane][VEC].
// value(a, l, j) gives the raw score of residue a (0..A, row A: an unknown
// residue, scored as the smallest matrix entry) at lane l, segment index j
// (j < S), or a sentinel below -256 for positions past the query end; row
// A+1 is inert (columns past a sequence's end).
template <class LT, int L, int S, class ValueFn>
__device__ __forceinline__ void stage_profile(typename LT::Elem *dst, int A, int o, int tid, int nthreads,
                                              ValueFn value)
{
    constexpr int V = LT::VEC;
    constexpr int SP = SegPad<S, V>::value;
    const int total = (A + 2) * L * SP;
    for (int idx = tid; idx < total; idx += nthreads) {
        const int a = idx / (L * SP);
        const int rem = idx - a * (L * SP);
        const int l = rem / SP;
        const int j = rem - l * SP;
        int v = LT::PAD;
        if (a <= A && j < S) {
            const int raw = value(a, l, j);
            if (raw > -256)
                v = raw + LT::prof_bias(o);
        }
        dst[((a * (SP / V) + j / V) * L + l) * V + (j % V)] = (typename LT::Elem)v;
    }
}

// PIECES: the launch splits long sequences into pieces (scores only, one
// chunk); a separate instantiation so that the others stay as they are.
template <class LT, int L, int S, bool LAZY, bool ENDS = false, bool PIECES = false>
__global__ void __launch_bounds__(BATCH_THREADS) sw_batch_kernel(const BatchArgs p)
{
    using T = typename LT::T;
    using Elem = typename LT::Elem;
    constexpr int CELLS = LT::CELLS;
    constexpr int G = 32 / L;
    constexpr int QC = L * S;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(L >= 1 && L <= 32 && (L & (L - 1)) == 0, "lanes per alignment: power of two");
    static_assert(!LAZY || LT::VEC != 16, "lazy-F kernel: int32 or s16x2 lanes");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Elem *sprof = reinterpret_cast<Elem *>(smem_raw);

    const int8_t *gprof = p.prof + (size_t)p.chunk * p.A * QC;
    const int qbase = p.chunk * QC;
    const int qlen = p.qlen;
    stage_profile<LT, L, S>(sprof, p.A, p.o, threadIdx.x, blockDim.x, [&](int a, int l, int j) {
        if (qbase + l * S + j >= qlen)
            return -1024;
        return a < p.A ? (int)gprof[(size_t)a * QC + l * S + j] : (int)p.min_m;
    });
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    static_assert(!(PIECES && ENDS), "pieces: scores only");
    const int n_pieces = PIECES ? *p.n_pieces : 0;
    const int64_t n_work = (p.n_work_dev ? (int64_t)(*p.n_work_dev) : p.n_work) + n_pieces;
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
            if constexpr (PIECES) {
                const BatchItem it = batch_item(p, unit < units ? w : n_work, n_work, n_pieces);
                seq[c] = it.id;
                start[c] = it.start;
                len[c] = it.len;
            } else {
                const bool ok = unit < units && w < n_work;
                seq[c] = ok ? (p.order ? p.order[w] : (int)w) : -1;
                start[c] = ok ? p.off[seq[c]] : 0;
                len[c] = ok ? (int)(p.off[seq[c] + 1] - start[c]) : 0;
            }
            my_n = max(my_n, len[c]);
        }
        const int ncols = (int)__reduce_max_sync(FULL, (unsigned)my_n);
        if constexpr (ENDS) {
            int er = -1, eq = -1;
            const T mx = striped_unit<LT, L, S, false, true>(pbase, p.db, start, len, ncols, p.A, p.o, p.e, p.one,
                                                             has_prev, has_next, p.bnd, gl, lazy_steps, &er, &eq);
            if (gl == 0 && seq[0] >= 0) {
                // combine with the earlier chunks (smaller query positions)
                int s = (int)mx, qe = eq >= 0 ? qbase + eq + 1 : -1, re = er >= 0 ? er + 1 : -1;
                if (has_prev) {
                    const int ps = p.scores[seq[0]], pq = p.q_end[seq[0]], pr = p.r_end[seq[0]];
                    if (!(s > ps || (s == ps && s > 0 && (re < pr || (re == pr && qe < pq))))) {
                        s = ps;
                        qe = pq;
                        re = pr;
                    }
                }
                p.scores[seq[0]] = s;
                p.q_end[seq[0]] = s > 0 ? qe : -1;
                p.r_end[seq[0]] = s > 0 ? re : -1;
            }
        } else {
            const T mx = striped_unit<LT, L, S, LAZY>(pbase, p.db, start, len, ncols, p.A, p.o, p.e, p.one,
                                                      has_prev, has_next, p.bnd, gl, lazy_steps);
            if (gl == 0) {
                if constexpr (PIECES)
                    write_scores_pieces<LT>(mx, LT::consts(p.o, p.e, S, p.one), seq, p.flag_thresh, p.scores);
                else
                    write_scores<LT>(mx, LT::consts(p.o, p.e, S, p.one), seq, has_prev, p.flag_thresh, p.scores);
            }
        }
    }
    // j-steps of the correction loop, counted once per warp
    if (LAZY && p.lazy_steps && lane == 0 && lazy_steps)
        atomicAdd(p.lazy_steps, lazy_steps);
}

}  // namespace swg
