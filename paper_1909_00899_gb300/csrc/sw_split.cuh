// Split-query s16x2 batch kernel: both 16-bit halves of a register belong to
// the same alignment.  A chunk of the query has 2*L*S positions; lane l,
// segment index j holds position l*S + j of the first half in its low half
// and position L*S + l*S + j of the second half in its high half, i.e. the
// striped layout of Alg. 1 over 2L virtual lanes (virtual lane L + l lives
// in the high half of lane l).  The profile is packed per residue in shared
// memory, so a 16-byte load brings four positions of both halves with no
// byte permutes, and one residue per column is broadcast.
//
// Differences from the two-alignment s16x2 kernel (sw_batch.cuh):
//  - the diagonal of lane 0's high half is lane L-1's last low-half value
//    (position L*S - 1 precedes L*S);
//  - after the log2 L scan of both halves at once, the F leaving the first
//    half (the low half of lane L-1) is folded into the high halves with
//    weight (l+1)*S*e, and it is the carry into the high half of lane 0.
// Values use the biased X-space / h-space of LaneI16x2 (sw_lanes.cuh).
//
// D0 (shorter corrected pass): when every substitution score is >= -o the
// profile is biased by o instead of 128, so h-space and X-space coincide
// (delta = 0), and the deferred correction d_j no longer has to raise E before
// h.  The carry reaches cell j through the raised diagonal at least as high:
// the corrected H of cell j-1 is >= carry - (j-1)e, so the diagonal gives
// >= carry - (j-1)e + M >= carry - o - je = d_j whenever M >= -(o+e) (for
// j = 0 the same holds with lane l-1's last cell, whose corrected H is >=
// carry + e).  d_j is still folded into the next E, so per register-cell the
// corrected pass drops one ALU max and E's update needs no space conversion.
#pragma once
#include "sw_batch.cuh"

namespace swg {

struct LaneQ16 : LaneI16x2 {
    using Elem = uint32_t;              // staged profile: (low position, high position) pair
    static constexpr int CELLS = 1;     // one alignment per register
    static constexpr int VEC = 4;       // staged pairs per 16 bytes
    static constexpr bool CROSS = false;

    template <int L, int SP>
    __device__ __forceinline__ static void load_vec(const Elem *const *base, const int *res, int gl, int k, T *P)
    {
        const int4 v = reinterpret_cast<const int4 *>(base[0])[(res[0] * (SP / 4) + k) * L + gl];
        P[0] = (uint32_t)v.x;
        P[1] = (uint32_t)v.y;
        P[2] = (uint32_t)v.z;
        P[3] = (uint32_t)v.w;
    }
    // the alignment's maximum: both halves
    __device__ __forceinline__ static int score(T mx, int, const K &k)
    {
        return max((int)(int16_t)(mx & 0xffffu), (int)(int16_t)(mx >> 16)) - k.bh;
    }
};

// Profile bias of the split kernel: o when D0 (h-space = X-space), else 128.
template <bool D0>
__host__ __device__ __forceinline__ int split_pb(int o)
{
    return D0 ? o : LaneQ16::PB;
}

template <int L, int S, bool D0, bool LAZY = false, bool ENDS = false, bool AC = false>
// len: this group's reference length; ncols: the warp's longest (every
// lane runs ncols columns, columns past len use the inert row A+1).
// LAZY: the lazy-F loop of Alg. 1 over the 2L virtual lanes instead of the
// scan (the comparison kernel); lazy_steps counts its j-steps.
// ENDS (scan-F): also the group's end cell, the first cell in column order
// whose h reaches the maximum, as end_r (0-based column) and end_q (0-based
// position in the chunk), -1 when nothing scored above 0.  A lane half notes
// the column in which its running maximum rose above the group's running
// maximum (a few instructions per column; the group maximum is re-reduced
// only in such columns) and recovers the row there from the stored X: within
// a column the F a lane's pass starts from is 0 (every carry is deferred), so
// F - o stays below the h - o of the column's best cell and X[j] == h - o of
// the maximum holds exactly at the cells that reached it.  A half whose
// maximum ends below the alignment's score may keep a stale note; it never
// wins the final reduction.
// AC (always corrected; scan-F scores with D0): every column runs the
// corrected pass, with no warp vote on the carry (on protein data nearly
// every column carries F across lanes), and the zero floor of H moves from h
// to the diagonal.  h = max(Xd + P', E) is then one DPX add-max, and the
// diagonal max(X, d_j, -o) one vimax3, where the plain corrected pass needs
// an extra addition for the relu form.  Dropping the floor from h leaves
// every value exact above its floor (H >= 0, and E, F, X >= -o in X-space):
// a value under its floor only ever meets maxima with values that carry the
// floor, and the one place where it could be raised again -- the diagonal,
// where M is added -- takes the floor explicitly.  So h, the maximum and
// everything above -o are unchanged.
__device__ __forceinline__ uint32_t split_unit(const uint32_t *prof, const uint8_t *ref, int64_t start, int len,
                                               int ncols, int A, int o, int e, uint32_t one, bool has_prev,
                                               bool has_next, int2 *bnd, int gl,
                                               unsigned long long *lazy_steps = nullptr, int *end_r = nullptr,
                                               int *end_q = nullptr, int64_t bbase = -1)
{
    // boundary rows are indexed from bbase (default: the residues' start)
    const int64_t bb = bbase >= 0 ? bbase : start;
    static_assert(!(LAZY && ENDS), "end cells: scan-F only");
    static_assert(!AC || (D0 && !LAZY && !ENDS), "always-corrected pass: D0 scan-F scores only");
    using LT = LaneQ16;
    using T = uint32_t;
    constexpr int SP = SegPad<S, 4>::value;
    constexpr int LOGL = L == 1 ? 0 : L == 2 ? 1 : L == 4 ? 2 : L == 8 ? 3 : L == 16 ? 4 : 5;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int V = 4;

    const LT::K k = LT::consts_pb(o, e, S, one, split_pb<D0>(o));
    T negW[LOGL > 0 ? LOGL : 1];  // scan hop weights (none for one thread)
#pragma unroll
    for (int i = 0; i < LOGL; ++i)
        negW[i] = LT::splat(-(1 << i) * S * e);
    // fold of the first half's outgoing F into the second half: weight
    // (l+1)*S*e on the high half only
    const T wfold = (uint32_t)((-(gl + 1) * S * e) & 0xffff) << 16;
    const T neg_lo = 0x00008000u;  // low half -32768, never wins a max
    const uint32_t *pbase[1] = {prof};

    T X[S], E[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        X[j] = k.xinit;
        E[j] = k.hzero;
    }
    T c_prev = k.xzero;
    T hlast = k.xinit;
    const uint32_t xinit16 = (uint32_t)(LT::BX - o);
    uint32_t hb16 = xinit16;  // previous chunk's last X at the previous column (16 bits, lane 0)
    T mx = k.hzero;
    // ENDS: the running maximum kept per block of positions (ENB blocks of
    // whole pairs, the same one vimax3 per pair), so that a row recovery
    // scans only the block that reached the new maximum; four blocks where
    // the two-CTA register budget has room for them, else two
    constexpr int ENB = S >= 24 ? 4 : 2;
    static_assert(!ENDS || S % 2 == 0, "end cells: even segment length");
    T mxb[ENDS ? ENB : 1];
#pragma unroll
    for (int b = 0; b < (ENDS ? ENB : 1); ++b)
        mxb[b] = k.hzero;
    // run-time 65536: the half-word moves below stay IMADs on the FMA pipe
    const uint32_t m16 = one << 16;
    const int rot = (gl + L - 1) & (L - 1);  // source lane of the diagonal
    // ENDS, per half: the column, segment index and h-space value of the
    // half's last note (value 0: none)
    int br_lo = -1, bj_lo = 0, bv_lo = 0, br_hi = -1, bj_hi = 0, bv_hi = 0;
    T gm = k.hzero;  // ENDS: the group's running maximum (h-space, both halves; the zero score at first)

    for (int r0 = 0; r0 < ncols; r0 += L) {
        const int r = r0 + gl;
        const int myres = r < len ? min((int)ref[start + r], A) : A + 1;  // unknown row A, inert row A+1
        // this lane's column of the boundary row written by the previous
        // chunk (raw packed values; their high halves belong to that chunk's
        // last position), converted once here: its X as a 16-bit value and
        // the F entering (lazy-F: as the pair (F, 0) that starts lane 0's
        // pass; scan-F: as a 16-bit carry).  Packing the two high halves
        // into one word would halve these bytes, but the extra permute per
        // column measured 3-4 % slower on the long-query layouts, and the
        // rows cost no time at these rates.
        uint32_t my_h16 = xinit16, my_f = LAZY ? k.xzero : (uint32_t)LT::BX;
        if (has_prev && r < len) {
            const uint2 raw = reinterpret_cast<const uint2 *>(bnd)[bb + r];
            my_h16 = raw.x >> 16;
            my_f = LAZY ? __byte_perm(raw.y, k.xzero, 0x5432) : raw.y >> 16;
        }
        const int cols = min(L, ncols - r0);
        for (int rr = 0; rr < cols; ++rr) {
            const int rc = r0 + rr;
            int res[1];
            res[0] = __shfl_sync(FULL, myres, rr, L);
            T Pv[V];

            // diagonal: lane l-1's last values (one rotated shuffle); lane 0
            // takes the chunk boundary (low half) and lane L-1's last low
            // half (high half)
            const T v = __shfl_sync(FULL, hlast, rot, L);
            T hd = v;
            T F = k.xzero;
            uint32_t lo_in = xinit16;
            if (has_prev) {
                const uint32_t bh = __shfl_sync(FULL, my_h16, rr, L);
                lo_in = hb16;
                hb16 = bh;
                if (LAZY) {
                    const uint32_t bf = __shfl_sync(FULL, my_f, rr, L);
                    if (gl == 0)
                        F = bf;
                }
            }
            if (gl == 0)
                hd = fadd_u32(v, m16, lo_in);  // (lo_in, low half of v)

            T hpair = k.hzero;
            if constexpr (AC) {
                T d = LT::d0_of(c_prev, k);
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    if (j % V == 0)
                        LT::template load_vec<L, SP>(pbase, res, gl, j / V, Pv);
                    // h = max(Xd + P', E) with the floor carried by the diagonal
                    const T h = LT::addmax(hd, Pv[j % V], E[j]);
                    hd = LT::max3(X[j], d, k.xinit);
                    d = LT::dstep(d, k);
                    const T ho = LT::ho_of(h, k);
                    X[j] = LT::addmax(F, k.negO, ho);
                    E[j] = LT::max3(LT::fadd(E[j], k.negE32, k), d, X[j]);
                    F = LT::addmax(F, k.negE, ho);
                    if (j & 1)
                        mx = LT::max3(mx, hpair, h);
                    else if (j == S - 1)
                        mx = LT::max2(mx, h);
                    else
                        hpair = h;
                }
            } else if (!LAZY && __any_sync(FULL, LT::carry_pos(c_prev, k))) {
                T d = LT::d0_of(c_prev, k);
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    if (j % V == 0)
                        LT::template load_vec<L, SP>(pbase, res, gl, j / V, Pv);
                    T h;
                    if constexpr (D0) {
                        // d_j is dominated by the raised diagonal in h and
                        // enters only the next E: max(E - e, d_j - e, X)
                        h = LT::h_of(hd, Pv[j % V], E[j], k);
                        hd = LT::max2(X[j], d);
                        d = LT::dstep(d, k);
                        const T ho = LT::ho_of(h, k);
                        X[j] = LT::addmax(F, k.negO, ho);
                        E[j] = LT::max3(LT::fadd(E[j], k.negE32, k), d, X[j]);
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
                    if (j & 1) {
                        if constexpr (ENDS)
                            mxb[(j / 2) * ENB / (S / 2)] = LT::max3(mxb[(j / 2) * ENB / (S / 2)], hpair, h);
                        else
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
                    if constexpr (D0)
                        E[j] = LT::addmax(E[j], k.negE, X[j]);  // same space: max(E - e, X)
                    else
                        E[j] = LT::e_next(E[j], X[j], k);
                    F = LT::addmax(F, k.negE, ho);
                    if (j & 1) {
                        if constexpr (ENDS)
                            mxb[(j / 2) * ENB / (S / 2)] = LT::max3(mxb[(j / 2) * ENB / (S / 2)], hpair, h);
                        else
                            mx = LT::max3(mx, hpair, h);
                    } else if (j == S - 1) {
                        mx = LT::max2(mx, h);
                    } else {
                        hpair = h;
                    }
                }
            }
            if constexpr (ENDS) {
                // Only a cell that raises the group's running maximum can be
                // the end cell (a later cell that merely ties it comes after
                // the one that set it), so the halves are looked at only in
                // columns where some half rose above that maximum (gm).  The
                // group maximum g is then re-reduced; if it rose, each half
                // with a block that reached g (in this column, g being new)
                // notes the first cell (smallest j) of its first such block
                // whose X is h - o of g.
                mx = mxb[0];
#pragma unroll
                for (int b = 1; b < ENB; b += 2)
                    mx = b + 1 < ENB ? LT::max3(mx, mxb[b], mxb[b + 1]) : LT::max2(mx, mxb[b]);
                if (__any_sync(FULL, LT::max2(mx, gm) != gm)) {
                    int g = max((int)(mx & 0xffffu), (int)(mx >> 16));
#pragma unroll
                    for (int dd = L / 2; dd >= 1; dd >>= 1)
                        g = max(g, __shfl_xor_sync(FULL, g, dd, L));
                    const bool rose = g > (int)(gm & 0xffffu);
                    gm = (uint32_t)(g & 0xffff) * 0x10001u;
                    int blo = -1, bhi = -1;
#pragma unroll
                    for (int b = ENB - 1; b >= 0; --b) {
                        if ((int)(mxb[b] & 0xffffu) >= g)
                            blo = b;
                        if ((int)(mxb[b] >> 16) >= g)
                            bhi = b;
                    }
                    if (rose && (blo >= 0 || bhi >= 0)) {
                        const T t = LT::ho_of(gm, k);
                        int jlo = 0, jhi = 0;
#pragma unroll
                        for (int b = ENB - 1; b >= 0; --b) {
                            if (b == blo || b == bhi) {
#pragma unroll
                                for (int j = S - 1; j >= 0; --j) {
                                    if ((j / 2) * ENB / (S / 2) != b)
                                        continue;
                                    const uint32_t dx = X[j] ^ t;
                                    if (b == blo && (dx & 0xffffu) == 0u)
                                        jlo = j;
                                    if (b == bhi && (dx >> 16) == 0u)
                                        jhi = j;
                                }
                            }
                        }
                        if (blo >= 0) {
                            br_lo = rc;
                            bj_lo = jlo;
                            bv_lo = g;
                        }
                        if (bhi >= 0) {
                            br_hi = rc;
                            bj_hi = jhi;
                            bv_hi = g;
                        }
                    }
                }
            }
            if constexpr (LAZY) {
                // lazy-F (Alg. 1): shift the F leaving each virtual lane into
                // the next one (lane L-1's low half into lane 0's high half)
                // and correct, for at most 2L rounds; leave every round once
                // no lane's carried F can raise anything (reading R6)
                T fb = F;  // F leaving this lane, corrected as rounds pass
                T Fc = __shfl_sync(FULL, F, rot, L);
                if (gl == 0)
                    Fc = fadd_u32(Fc, m16, (uint32_t)LT::BX);  // (0, low half of lane L-1)
                bool done = false;
                unsigned long long steps = 0;
                for (int kk = 0; kk < 2 * L && !done; ++kk) {
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const T hold = X[j];
                        X[j] = LT::addmax(Fc, k.negO, hold);
                        E[j] = LT::e_raise(E[j], X[j], k);
                        Fc = LT::lazy_step(Fc, k);
                        ++steps;
                        if (__all_sync(FULL, LT::lazy_dominated(Fc, hold, k))) {
                            done = true;
                            break;
                        }
                    }
                    if (!done) {
                        fb = LT::max2(fb, Fc);
                        Fc = __shfl_sync(FULL, Fc, rot, L);
                        if (gl == 0)
                            Fc = fadd_u32(Fc, m16, (uint32_t)LT::BX);
                    }
                }
                if (lazy_steps)
                    *lazy_steps += steps;
                hlast = X[S - 1];
                if (has_next && gl == L - 1 && rc < len)
                    reinterpret_cast<uint2 *>(bnd)[bb + rc] = make_uint2(hlast, fb);
            } else {
                // scan-F: the chunk boundary's F is lane 0's low-half carry
                // (fetched here, after the pass, so that it holds no register
                // during it) and leaves that segment decayed by S*e
                uint32_t bf16 = (uint32_t)LT::BX;  // no carry
                if (has_prev) {
                    bf16 = __shfl_sync(FULL, my_f, rr, L);
                    if (gl == 0)
                        F = LT::addmax(bf16 | 0x80000000u, (uint32_t)((-S * e) & 0xffff), F);
                }
                // scan of both halves at once, then the first half's outgoing
                // F (low half of lane L-1) folded into the second half
                T x = F;
#pragma unroll
                for (int i = 0; i < LOGL; ++i) {
                    const T y = __shfl_up_sync(FULL, x, 1 << i, L);
                    x = LT::addmax(y, negW[i], x);
                }
                const T gb = __shfl_sync(FULL, x, L - 1, L);
                x = LT::addmax(fadd_u32(gb, m16, neg_lo), wfold, x);  // (-32768, low half of gb) + fold
                T cin = __shfl_up_sync(FULL, x, 1, L);
                if (gl == 0)
                    cin = fadd_u32(gb, m16, bf16);  // (boundary F or 0, low half of gb)
                c_prev = cin;
                // AC: the diagonal handed to the next lane carries the floor
                hlast = AC ? LT::max3(X[S - 1], LT::fadd(cin, k.negOS1_32, k), k.xinit)
                           : LT::last_corr(X[S - 1], cin, k);
                // the next chunk reads the high halves (this chunk's last position)
                if (has_next && gl == L - 1 && rc < len)
                    reinterpret_cast<uint2 *>(bnd)[bb + rc] = make_uint2(hlast, x);
            }
        }
    }
    if constexpr (ENDS) {
        // the lane's best note (larger value, then smaller column, then the
        // low half: its positions come first), then the group's best lane.
        // Notes are compared by the value they were made at: a half that
        // only tied the maximum in a later column kept an older, lower note,
        // while the cell that set the alignment's score noted exactly it.
        const int slo = bv_lo, shi = bv_hi;
        const bool hi_wins = shi > slo || (shi == slo && br_hi >= 0 && (br_lo < 0 || br_hi < br_lo));
        int bs = hi_wins ? shi : slo;
        int br = hi_wins ? br_hi : br_lo;
        int bq = hi_wins ? L * S + gl * S + bj_hi : gl * S + bj_lo;
#pragma unroll
        for (int dd = L / 2; dd >= 1; dd >>= 1) {
            const int os = __shfl_xor_sync(FULL, bs, dd, L);
            const int orr = __shfl_xor_sync(FULL, br, dd, L);
            const int oq = __shfl_xor_sync(FULL, bq, dd, L);
            if (os > bs || (os == bs && (orr < br || (orr == br && oq < bq)))) {
                bs = os;
                br = orr;
                bq = oq;
            }
        }
        const bool pos = bs > k.bh;  // above the h-space zero
        *end_r = pos ? br : -1;
        *end_q = pos ? bq : -1;
    }
#pragma unroll
    for (int dd = L / 2; dd >= 1; dd >>= 1)
        mx = LT::max2(mx, __shfl_xor_sync(FULL, mx, dd, L));
    return mx;
}

// CTAs of 256 threads per SM the register budget is held to (48, 64, 80 or
// 128 registers a thread), the most each segment length fits without spills
// (short segments serve short queries, which are latency-bound and want the
// extra warps)
template <int S, bool D0, bool ENDS = false, bool AC = false>
struct SplitMinBlocks {
    static constexpr int value = AC        ? (S <= 20 ? 3 : 2)
                                 : D0 && !ENDS ? (S <= 8 ? 5 : S <= 16 ? 4 : S <= 24 ? 3 : 2)
                                 : ENDS      ? (D0 ? (S <= 8 ? 4 : S <= 20 ? 3 : 2) : (S <= 8 ? 3 : 2))
                                             : (S <= 8 ? 4 : S <= 20 ? 3 : 2);
};

// PIECES: the launch splits long sequences into pieces (scores only, one
// chunk); a separate instantiation so that the others stay as they are.
template <int L, int S, bool D0, bool LAZY = false, bool ENDS = false, bool PIECES = false, bool AC = false>
__global__ void __launch_bounds__(BATCH_THREADS, SplitMinBlocks<S, D0, ENDS, AC>::value) sw_split_kernel(const BatchArgs p)
{
    constexpr int G = 32 / L;
    constexpr int SP = SegPad<S, 4>::value;
    constexpr int QH = L * S;  // positions per half
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *sprof = reinterpret_cast<uint32_t *>(smem_raw);

    // stage the chunk: raw profile of 2L virtual lanes [A][2L][S]; pair
    // virtual lanes l and L + l into one 32-bit element.  Row A: an unknown
    // residue (the smallest matrix entry); row A+1: inert
    const int8_t *gprof = p.prof + (size_t)p.chunk * p.A * 2 * QH;
    const int qbase = p.chunk * 2 * QH;
    const int total = (p.A + 2) * L * SP;
    const int pb = split_pb<D0>(p.o);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int a = idx / (L * SP);
        const int rem = idx - a * (L * SP);
        const int l = rem / SP;
        const int j = rem - l * SP;
        int lo = LaneQ16::PAD, hi = LaneQ16::PAD;
        if (a <= p.A && j < S) {
            const int plo = l * S + j, phi = QH + l * S + j;
            if (qbase + plo < p.qlen)
                lo = (a < p.A ? (int)gprof[(size_t)a * 2 * QH + plo] : (int)p.min_m) + pb;
            if (qbase + phi < p.qlen)
                hi = (a < p.A ? (int)gprof[(size_t)a * 2 * QH + phi] : (int)p.min_m) + pb;
        }
        sprof[((a * (SP / 4) + j / 4) * L + l) * 4 + (j % 4)] = (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    static_assert(!(PIECES && ENDS), "pieces: scores only");
    const int n_pieces = PIECES ? *p.n_pieces : 0;
    const int64_t n_work = (p.n_work_dev ? (int64_t)(*p.n_work_dev) : p.n_work) + n_pieces;
    const bool has_prev = p.chunk > 0;
    const bool has_next = p.chunk + 1 < p.nchunks;
    const LaneQ16::K k = LaneQ16::consts_pb(p.o, p.e, S, p.one, split_pb<D0>(p.o));
    unsigned long long lazy_steps = 0;

    for (;;) {
        unsigned int ubase = 0;
        if (lane == 0)
            ubase = atomicAdd(p.counter, (unsigned int)G);
        ubase = __shfl_sync(FULL, ubase, 0);
        if ((int64_t)ubase >= n_work)
            break;
        const int64_t w = (int64_t)ubase + grp;
        int seq[1];
        int64_t start;
        int len;
        if constexpr (PIECES) {
            const BatchItem it = batch_item(p, w, n_work, n_pieces);
            seq[0] = it.id;
            start = it.start;
            len = it.len;
        } else {
            seq[0] = w < n_work ? (p.order ? p.order[w] : (int)w) : -1;
            start = seq[0] >= 0 ? p.off[seq[0]] : 0;
            len = seq[0] >= 0 ? (int)(p.off[seq[0] + 1] - start) : 0;
        }
        const int ncols = (int)__reduce_max_sync(FULL, (unsigned)len);
        if constexpr (ENDS) {
            int er = -1, eq = -1;
            const uint32_t mx = split_unit<L, S, D0, false, true>(sprof, p.db, start, len, ncols, p.A, p.o, p.e,
                                                                  p.one, has_prev, has_next, p.bnd, gl, nullptr,
                                                                  &er, &eq);
            if (gl == 0 && seq[0] >= 0) {
                // combine with the earlier chunks (smaller query positions)
                int s = LaneQ16::score(mx, 0, k), qe = eq >= 0 ? qbase + eq + 1 : -1, re = er >= 0 ? er + 1 : -1;
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
            const uint32_t mx = split_unit<L, S, D0, LAZY, false, AC>(sprof, p.db, start, len, ncols, p.A, p.o, p.e,
                                                                      p.one, has_prev, has_next, p.bnd, gl,
                                                                      &lazy_steps);
            if (gl == 0) {
                if constexpr (PIECES)
                    write_scores_pieces<LaneQ16>(mx, k, seq, p.flag_thresh, p.scores);
                else
                    write_scores<LaneQ16>(mx, k, seq, has_prev, p.flag_thresh, p.scores);
            }
        }
    }
    // j-steps of the correction loop, counted once per warp
    if (LAZY && p.lazy_steps && lane == 0 && lazy_steps)
        atomicAdd(p.lazy_steps, lazy_steps);
}

}  // namespace swg
