// Lane types of the striped kernels: how one 32-bit register carries the
// cells of 1, 2 or 4 alignments, and the cell update written for them.
//
// Value spaces.  The kernels keep X = H - o (the stored H of Alg. 6), E and
// F, all bounded below by -o, and h = H before F (Alg. 6 takes Max on it).
// A lane type stores X, F and the scan carries in "X-space" (true + BX) and
// h, E and the deferred correction d in "h-space" (true + BH), and stages
// the profile biased by PB (added to every matrix entry):
//     h = max(Xd + P', E, floor)  is exact when  BH = BX + PB - o.
// int32 and s8x4 lanes use BX = BH = 0, PB = o and the relu forms, the
// signed restatement of the paper's saturating arithmetic ("none of the
// vector values can be negative").  s16x2 lanes use BX = 4096 and PB = 128:
// every stored half is then a positive 15-bit number, so a plain 32-bit add
// of a packed constant is an exact add in both halves.
//
// Pure additions go through fadd(): IMAD with a multiplier that is 1 at run
// time, i.e. on the FMA pipe, which leaves the half-rate integer ALU pipe to
// the max-plus DPX steps.  ALU instructions per register-cell of the plain
// pass: h (1), X (1), E (1), F (1) and the running max (1/2, vimax3 over two
// positions); the deferred correction adds 2 (raise E, raise the diagonal),
// or 1 with the D0 lane types at the end of this file.
//
// Packed lanes are exact until H + M leaves the lane range.  The H of the
// first such addition was exact and already folded into the alignment's
// maximum, so alignments whose packed maximum reached the lane's threshold
// are rescored in int32 (sw_batch.cuh).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace swg {

// a + b on the FMA pipe: IMAD with a multiplier the compiler cannot fold
__device__ __forceinline__ uint32_t fadd_u32(uint32_t a, uint32_t one, uint32_t b)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(one), "r"(b));
    return d;
}

// ---------------------------------------------------------------------------
struct LaneI32 {
    using T = int32_t;
    using Elem = int32_t;               // shared-memory profile element
    static constexpr int CELLS = 1;     // alignments per register
    static constexpr int VEC = 4;       // profile elements per 16 bytes
    static constexpr int PAD = -(1 << 24);  // inert staged profile value
    static constexpr bool CROSS = false;    // cells never leak into each other
    static constexpr bool D0 = false;       // see LaneI32D
    __host__ __device__ static constexpr int prof_bias(int o) { return o; }

    struct K {
        uint32_t one;
        T negO, negE, negOS1, xzero, hzero, xinit;
    };
    __device__ __forceinline__ static K consts(int o, int e, int S, uint32_t one)
    {
        K k;
        k.one = one;
        k.negO = -o;
        k.negE = -e;
        k.negOS1 = -o - (S - 1) * e;
        k.xzero = 0;   // inert carry / F
        k.hzero = 0;   // H = 0 in h-space
        k.xinit = -o;  // X of H = 0
        return k;
    }
    __device__ __forceinline__ static T splat(int v) { return v; }
    __device__ __forceinline__ static T fadd(T a, T b, const K &k)
    {
        return (T)fadd_u32((uint32_t)a, k.one, (uint32_t)b);
    }
    __device__ __forceinline__ static T addmax(T a, T b, T c) { return __viaddmax_s32(a, b, c); }
    __device__ __forceinline__ static T max2(T a, T b) { return max(a, b); }
    __device__ __forceinline__ static T max3(T a, T b, T c) { return __vimax3_s32(a, b, c); }

    // h = max(Xd + P', E, 0)
    __device__ __forceinline__ static T h_of(T xd, T P, T E, const K &) { return __viaddmax_s32_relu(xd, P, E); }
    // H' - o in X-space
    __device__ __forceinline__ static T ho_of(T h, const K &k) { return fadd(h, k.negO, k); }
    // E of the next column: max(E - e, X)
    __device__ __forceinline__ static T e_next(T E, T X, const K &k) { return __viaddmax_s32(E, k.negE, X); }
    // correction value of position 0 (h-space) from a carry (X-space)
    __device__ __forceinline__ static T d0_of(T c, const K &k) { return fadd(c, k.negO, k); }
    __device__ __forceinline__ static T dstep(T d, const K &k) { return fadd(d, k.negE, k); }
    // corrected diagonal (X-space) from the stored X and d (h-space)
    __device__ __forceinline__ static T xd_corr(T X, T d, const K &) { return max(X, d); }
    // next E with the correction of the previous column: max(E - e, d_{j+1}, X)
    // (dn = d_j - e; h-space = X-space)
    __device__ __forceinline__ static T e_next_corr(T E, T dn, T X, const K &k)
    {
        return __vimax3_s32(fadd(E, k.negE, k), dn, X);
    }
    __device__ __forceinline__ static bool carry_pos(T c, const K &) { return c > 0; }
    // last position raised by the carry: max(X, c - o - (S-1)e)
    __device__ __forceinline__ static T last_corr(T X, T c, const K &k) { return max(X, fadd(c, k.negOS1, k)); }

    __device__ __forceinline__ static int score(T mx, int, const K &) { return mx; }
    __device__ __forceinline__ static int x_true(T v, int) { return v; }
    __device__ __forceinline__ static T x_pack(const int *v) { return v[0]; }

    // lazy-F loop (Alg. 1): E raised from a corrected X; the carry Fc (after
    // the extend step) is dominated when Fc <= max(X before the raise, 0)
    __device__ __forceinline__ static T e_raise(T E, T X, const K &) { return max(E, X); }
    __device__ __forceinline__ static T lazy_step(T Fc, const K &k) { return Fc + k.negE; }
    __device__ __forceinline__ static bool lazy_dominated(T Fc, T hold, const K &) { return Fc <= max(hold, 0); }

    // Profile rows of residues res[c] for segment positions 0..S-1; base[c]
    // is cell c's staged profile, layout [residue][SP/VEC][lane][VEC].
    // profile vector k (positions VEC*k .. VEC*k+VEC-1) of the residues res[c]
    template <int L, int SP>
    __device__ __forceinline__ static void load_vec(const Elem *const *base, const int *res, int gl, int k, T *P)
    {
        const int4 v = reinterpret_cast<const int4 *>(base[0])[(res[0] * (SP / 4) + k) * L + gl];
        P[0] = v.x;
        P[1] = v.y;
        P[2] = v.z;
        P[3] = v.w;
    }

    template <int L, int S, int SP>
    __device__ __forceinline__ static void load_profile(const Elem *const *base, const int *res, int gl, T *P)
    {
        const int4 *row = reinterpret_cast<const int4 *>(base[0]) + (res[0] * (SP / 4)) * L + gl;
#pragma unroll
        for (int k = 0; k < SP / 4; ++k) {
            const int4 v = row[k * L];
            if (4 * k + 0 < S) P[4 * k + 0] = v.x;
            if (4 * k + 1 < S) P[4 * k + 1] = v.y;
            if (4 * k + 2 < S) P[4 * k + 2] = v.z;
            if (4 * k + 3 < S) P[4 * k + 3] = v.w;
        }
    }
};

// ---------------------------------------------------------------------------
struct LaneI16x2 {
    using T = uint32_t;
    using Elem = int16_t;
    static constexpr int CELLS = 2;
    static constexpr int VEC = 8;
    static constexpr int PB = 128;   // staged profile values M + 128, in [0, 255]
    static constexpr int PAD = 0;    // inert staged value (as if M = -128)
    static constexpr int BX = 4096;  // X-space bias
    // the 32-bit adds are exact only while both halves stay in [0, 0x7fff];
    // once one cell has overflowed the other may be corrupted, so both cells
    // of a register are rescored together
    static constexpr bool CROSS = true;
    static constexpr bool D0 = false;  // see LaneI16x2D
    __host__ __device__ static constexpr int prof_bias(int) { return PB; }

    struct K {
        uint32_t one;
        int bh;
        T negO, negE, delta, negDelta, xzero, hzero, xinit;
        T hshift32, negE32, d0c32, negOS1_32, cpos32;
    };
    // per-half constant for the DPX forms (saturated to 16 bits)
    __device__ __forceinline__ static T splat(int v)
    {
        v = max(-32768, min(32767, v));
        return (uint32_t)(v & 0xffff) * 0x10001u;
    }
    // constant whose 32-bit add adds v to both halves
    __device__ __forceinline__ static T splat32(int v) { return (uint32_t)v * 65537u; }
    __device__ __forceinline__ static K consts(int o, int e, int S, uint32_t one) { return consts_pb(o, e, S, one, PB); }
    // pb: the profile bias actually staged (PB, or o for the split kernel's
    // pass in which h-space and X-space coincide)
    __device__ __forceinline__ static K consts_pb(int o, int e, int S, uint32_t one, int pb)
    {
        K k;
        k.one = one;
        k.bh = BX + pb - o;
        k.negO = splat(-o);
        k.negE = splat(-e);
        k.delta = splat(k.bh - BX);
        k.negDelta = splat(BX - k.bh);
        k.xzero = splat(BX);
        k.hzero = splat(k.bh);
        k.xinit = splat(BX - o);
        k.hshift32 = splat32(-pb);              // h -> H' - o in X-space
        k.negE32 = splat32(-e);
        k.d0c32 = splat32(k.bh - BX - o);       // carry (X) -> d (h): c - o
        k.negOS1_32 = splat32(-o - (S - 1) * e);
        k.cpos32 = splat32(0x7fff - BX);        // half > BX  <=>  bit 15 of half + 0x7fff - BX
        return k;
    }
    __device__ __forceinline__ static T fadd(T a, T b, const K &k) { return fadd_u32(a, k.one, b); }
    __device__ __forceinline__ static T addmax(T a, T b, T c) { return __viaddmax_s16x2(a, b, c); }
    __device__ __forceinline__ static T max2(T a, T b) { return __vmaxs2(a, b); }
    __device__ __forceinline__ static T max3(T a, T b, T c) { return __vimax3_s16x2(a, b, c); }

    __device__ __forceinline__ static T h_of(T xd, T P, T E, const K &k)
    {
        return __vimax3_s16x2(fadd(xd, P, k), E, k.hzero);
    }
    __device__ __forceinline__ static T ho_of(T h, const K &k) { return fadd(h, k.hshift32, k); }
    __device__ __forceinline__ static T e_next(T E, T X, const K &k)
    {
        return __viaddmax_s16x2(X, k.delta, fadd(E, k.negE32, k));
    }
    __device__ __forceinline__ static T d0_of(T c, const K &k) { return fadd(c, k.d0c32, k); }
    __device__ __forceinline__ static T dstep(T d, const K &k) { return fadd(d, k.negE32, k); }
    __device__ __forceinline__ static T xd_corr(T X, T d, const K &k) { return __viaddmax_s16x2(d, k.negDelta, X); }
    // a positive carry in either half (halves are in [0, 0x7fff]; the sum
    // stays below 0x10000, so no carry crosses into the high half)
    __device__ __forceinline__ static bool carry_pos(T c, const K &k)
    {
        return (fadd(c, k.cpos32, k) & 0x80008000u) != 0u;
    }
    __device__ __forceinline__ static T last_corr(T X, T c, const K &k)
    {
        return __vmaxs2(X, fadd(c, k.negOS1_32, k));
    }

    __device__ __forceinline__ static int score(T mx, int c, const K &k)
    {
        return (int)(int16_t)(c ? (mx >> 16) : (mx & 0xffffu)) - k.bh;
    }
    __device__ __forceinline__ static int x_true(T v, int c) { return (int)(int16_t)(c ? (v >> 16) : (v & 0xffffu)) - BX; }
    __device__ __forceinline__ static T x_pack(const int *v)
    {
        return (uint32_t)((v[0] + BX) & 0xffff) | ((uint32_t)((v[1] + BX) & 0xffff) << 16);
    }

    // lazy-F loop: E (h-space) raised from X (X-space); both halves dominated
    __device__ __forceinline__ static T e_raise(T E, T X, const K &k) { return __viaddmax_s16x2(X, k.delta, E); }
    __device__ __forceinline__ static T lazy_step(T Fc, const K &k) { return Fc + k.negE32; }
    __device__ __forceinline__ static bool lazy_dominated(T Fc, T hold, const K &k)
    {
        const T t = __vmaxs2(hold, k.xzero);
        return __vmaxs2(Fc, t) == t;
    }

    template <int L, int SP>
    __device__ __forceinline__ static void load_vec(const Elem *const *base, const int *res, int gl, int k, T *P)
    {
        const int4 a = reinterpret_cast<const int4 *>(base[0])[(res[0] * (SP / 8) + k) * L + gl];
        const int4 b = reinterpret_cast<const int4 *>(base[1])[(res[1] * (SP / 8) + k) * L + gl];
        P[0] = __byte_perm(a.x, b.x, 0x5410);
        P[1] = __byte_perm(a.x, b.x, 0x7632);
        P[2] = __byte_perm(a.y, b.y, 0x5410);
        P[3] = __byte_perm(a.y, b.y, 0x7632);
        P[4] = __byte_perm(a.z, b.z, 0x5410);
        P[5] = __byte_perm(a.z, b.z, 0x7632);
        P[6] = __byte_perm(a.w, b.w, 0x5410);
        P[7] = __byte_perm(a.w, b.w, 0x7632);
    }

    template <int L, int S, int SP>
    __device__ __forceinline__ static void load_profile(const Elem *const *base, const int *res, int gl, T *P)
    {
        const int4 *ra = reinterpret_cast<const int4 *>(base[0]) + (res[0] * (SP / 8)) * L + gl;
        const int4 *rb = reinterpret_cast<const int4 *>(base[1]) + (res[1] * (SP / 8)) * L + gl;
#pragma unroll
        for (int k = 0; k < SP / 8; ++k) {
            const int4 a = ra[k * L];
            const int4 b = rb[k * L];
            const uint32_t aw[4] = {(uint32_t)a.x, (uint32_t)a.y, (uint32_t)a.z, (uint32_t)a.w};
            const uint32_t bw[4] = {(uint32_t)b.x, (uint32_t)b.y, (uint32_t)b.z, (uint32_t)b.w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (8 * k + 2 * w < S) P[8 * k + 2 * w] = __byte_perm(aw[w], bw[w], 0x5410);
                if (8 * k + 2 * w + 1 < S) P[8 * k + 2 * w + 1] = __byte_perm(aw[w], bw[w], 0x7632);
            }
        }
    }
};

// ---------------------------------------------------------------------------
struct LaneI8x4 {
    using T = uint32_t;
    using Elem = int8_t;
    static constexpr int CELLS = 4;
    static constexpr int VEC = 16;
    static constexpr int PAD = -128;
    static constexpr bool CROSS = false;  // saturating bytes never leak
    static constexpr bool D0 = false;
    __host__ __device__ static constexpr int prof_bias(int o) { return o; }

    struct K {
        T negO, negE, negS1, xzero, hzero, xinit;
    };
    // constants saturate to the lane range: a clamped negative constant
    // gives a saturated sum <= max(true sum, -128), which is inert wherever
    // the true sum was (every kept value is >= -o >= -127)
    __device__ __forceinline__ static T splat(int v)
    {
        v = max(-128, min(127, v));
        return (uint32_t)(v & 0xff) * 0x01010101u;
    }
    __device__ __forceinline__ static K consts(int o, int e, int S, uint32_t)
    {
        K k;
        k.negO = splat(-o);
        k.negE = splat(-e);
        k.negS1 = splat(-(S - 1) * e);
        k.xzero = 0u;
        k.hzero = 0u;
        k.xinit = splat(-o);
        return k;
    }
    __device__ __forceinline__ static T fadd(T a, T b, const K &) { return __vaddss4(a, b); }
    __device__ __forceinline__ static T addmax(T a, T b, T c) { return __vmaxs4(__vaddss4(a, b), c); }
    __device__ __forceinline__ static T max2(T a, T b) { return __vmaxs4(a, b); }
    __device__ __forceinline__ static T max3(T a, T b, T c) { return __vmaxs4(__vmaxs4(a, b), c); }

    __device__ __forceinline__ static T h_of(T xd, T P, T E, const K &)
    {
        return __vmaxs4(__vmaxs4(__vaddss4(xd, P), E), 0u);
    }
    __device__ __forceinline__ static T ho_of(T h, const K &k) { return __vaddss4(h, k.negO); }
    __device__ __forceinline__ static T e_next(T E, T X, const K &k) { return __vmaxs4(__vaddss4(E, k.negE), X); }
    __device__ __forceinline__ static T d0_of(T c, const K &k) { return __vaddss4(c, k.negO); }
    __device__ __forceinline__ static T dstep(T d, const K &k) { return __vaddss4(d, k.negE); }
    __device__ __forceinline__ static T xd_corr(T X, T d, const K &) { return __vmaxs4(X, d); }
    __device__ __forceinline__ static bool carry_pos(T c, const K &)
    {
        return (int8_t)c > 0 || (int8_t)(c >> 8) > 0 || (int8_t)(c >> 16) > 0 || (int8_t)(c >> 24) > 0;
    }
    // two saturating adds: each constant stays in range, the result floors at -128
    __device__ __forceinline__ static T last_corr(T X, T c, const K &k)
    {
        return __vmaxs4(X, __vaddss4(__vaddss4(c, k.negO), k.negS1));
    }

    __device__ __forceinline__ static int score(T mx, int c, const K &) { return (int)(int8_t)(mx >> (8 * c)); }
    __device__ __forceinline__ static int x_true(T v, int c) { return (int)(int8_t)(v >> (8 * c)); }
    __device__ __forceinline__ static T x_pack(const int *v)
    {
        return (uint32_t)(v[0] & 0xff) | ((uint32_t)(v[1] & 0xff) << 8) | ((uint32_t)(v[2] & 0xff) << 16) |
               ((uint32_t)(v[3] & 0xff) << 24);
    }

    // 4x4 byte transpose of the four rows' words into per-position registers
    __device__ __forceinline__ static void transpose4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, T *P)
    {
        const uint32_t ab_lo = __byte_perm(a, b, 0x5140);  // a0 b0 a1 b1
        const uint32_t ab_hi = __byte_perm(a, b, 0x7362);  // a2 b2 a3 b3
        const uint32_t cd_lo = __byte_perm(c, d, 0x5140);
        const uint32_t cd_hi = __byte_perm(c, d, 0x7362);
        P[0] = __byte_perm(ab_lo, cd_lo, 0x5410);
        P[1] = __byte_perm(ab_lo, cd_lo, 0x7632);
        P[2] = __byte_perm(ab_hi, cd_hi, 0x5410);
        P[3] = __byte_perm(ab_hi, cd_hi, 0x7632);
    }

    template <int L, int SP>
    __device__ __forceinline__ static void load_vec(const Elem *const *base, const int *res, int gl, int k, T *P)
    {
        const int4 a = reinterpret_cast<const int4 *>(base[0])[(res[0] * (SP / 16) + k) * L + gl];
        const int4 b = reinterpret_cast<const int4 *>(base[1])[(res[1] * (SP / 16) + k) * L + gl];
        const int4 c = reinterpret_cast<const int4 *>(base[2])[(res[2] * (SP / 16) + k) * L + gl];
        const int4 d = reinterpret_cast<const int4 *>(base[3])[(res[3] * (SP / 16) + k) * L + gl];
        transpose4(a.x, b.x, c.x, d.x, P + 0);
        transpose4(a.y, b.y, c.y, d.y, P + 4);
        transpose4(a.z, b.z, c.z, d.z, P + 8);
        transpose4(a.w, b.w, c.w, d.w, P + 12);
    }

    template <int L, int S, int SP>
    __device__ __forceinline__ static void load_profile(const Elem *const *base, const int *res, int gl, T *P)
    {
        const int4 *r0 = reinterpret_cast<const int4 *>(base[0]) + (res[0] * (SP / 16)) * L + gl;
        const int4 *r1 = reinterpret_cast<const int4 *>(base[1]) + (res[1] * (SP / 16)) * L + gl;
        const int4 *r2 = reinterpret_cast<const int4 *>(base[2]) + (res[2] * (SP / 16)) * L + gl;
        const int4 *r3 = reinterpret_cast<const int4 *>(base[3]) + (res[3] * (SP / 16)) * L + gl;
#pragma unroll
        for (int k = 0; k < SP / 16; ++k) {
            const int4 a = r0[k * L], b = r1[k * L], c = r2[k * L], d = r3[k * L];
            T Q[16];
            transpose4(a.x, b.x, c.x, d.x, Q + 0);
            transpose4(a.y, b.y, c.y, d.y, Q + 4);
            transpose4(a.z, b.z, c.z, d.z, Q + 8);
            transpose4(a.w, b.w, c.w, d.w, Q + 12);
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (16 * k + t < S) P[16 * k + t] = Q[t];
        }
    }
};

// ---------------------------------------------------------------------------
// Shorter corrected pass.  The deferred correction d_j = carry - o - j*e
// (the carry's F at position j, less o) raises both E[j] and the diagonal
// of position j+1.  In h it is never needed once every substitution score
// is >= -(o+e): the corrected H of position j-1 is >= carry - (j-1)*e, so
// the raised diagonal already gives h >= carry - (j-1)*e + M >= d_j (for
// j = 0 the diagonal is the previous lane's last position, whose corrected H
// is >= carry + e because e <= o).  d_j then enters only the next E,
// max(E - e, d_j - e, X), which needs h-space = X-space.  Per register-cell
// the corrected pass loses one ALU max.  h itself is unchanged, so scores
// and end cells are the same as with the general pass.
//
// int32: h-space is X-space already; usable when min(M) >= -(o+e).
struct LaneI32D : LaneI32 {
    static constexpr bool D0 = true;
};

// s16x2 with the profile biased by o instead of 128 (h-space = X-space,
// BH = BX): every staged value M + o must stay >= 0 for the packed adds, so
// usable when min(M) >= -o.  The inert value 0 reads as M = -o.
struct LaneI16x2D : LaneI16x2 {
    static constexpr bool D0 = true;
    __host__ __device__ static constexpr int prof_bias(int o) { return o; }
    __device__ __forceinline__ static K consts(int o, int e, int S, uint32_t one)
    {
        return consts_pb(o, e, S, one, o);
    }
    __device__ __forceinline__ static T e_next(T E, T X, const K &k) { return __viaddmax_s16x2(E, k.negE, X); }
    __device__ __forceinline__ static T xd_corr(T X, T d, const K &) { return __vmaxs2(X, d); }
    __device__ __forceinline__ static T e_next_corr(T E, T dn, T X, const K &k)
    {
        return __vimax3_s16x2(fadd(E, k.negE32, k), dn, X);
    }
};

}  // namespace swg
