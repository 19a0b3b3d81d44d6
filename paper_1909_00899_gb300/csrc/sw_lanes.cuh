// Lane types of the striped kernels: how one 32-bit register carries the
// cells of 1, 2 or 4 alignments, and the max-plus primitives on them.
//
// Every value the recurrence keeps is bounded below by -o (E, F and the
// stored H - o are all maxed with a value >= -o), and "+ profile" is floored
// at 0 by the relu forms, which is the signed restatement of the saturating
// unsigned arithmetic of Sec. I ("none of the vector values can be
// negative").  Packed lanes are exact until an addition H + M leaves the
// lane range; such alignments are detected by their maximum (see the
// overflow threshold in sw_internal.h) and rescored in int32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace swg {

struct LaneI32 {
    using T = int32_t;
    using Elem = int32_t;               // shared-memory profile element
    static constexpr int CELLS = 1;     // alignments per register
    static constexpr int VEC = 4;       // profile elements per 16 bytes
    static constexpr int PAD = -(1 << 24);  // inert profile score
    static constexpr int CEIL = 0x3fffffff;

    __device__ __forceinline__ static T splat(int v) { return v; }
    __device__ __forceinline__ static T zero() { return 0; }
    // max(a + b, c, 0)
    __device__ __forceinline__ static T addmax_relu(T a, T b, T c) { return __viaddmax_s32_relu(a, b, c); }
    // max(a + b, c)
    __device__ __forceinline__ static T addmax(T a, T b, T c) { return __viaddmax_s32(a, b, c); }
    __device__ __forceinline__ static T add(T a, T b) { return a + b; }
    __device__ __forceinline__ static T max2(T a, T b) { return max(a, b); }
    __device__ __forceinline__ static T max3(T a, T b, T c) { return __vimax3_s32(a, b, c); }
    __device__ __forceinline__ static bool any_pos(T a) { return a > 0; }
    __device__ __forceinline__ static int get(T a, int) { return a; }
    __device__ __forceinline__ static T shfl_up(T a, int d, int w) { return __shfl_up_sync(0xffffffffu, a, d, w); }
    __device__ __forceinline__ static T shfl_xor(T a, int d, int w) { return __shfl_xor_sync(0xffffffffu, a, d, w); }
    __device__ __forceinline__ static T pack(const int *v) { return v[0]; }

    // Profile rows of the residues res[c] (one per cell) for segment
    // positions 0..S-1.  base[c] is cell c's profile, layout
    // [residue][SP / VEC][lane][VEC] with SP = S rounded up to VEC.
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

struct LaneI16x2 {
    using T = uint32_t;
    using Elem = int16_t;
    static constexpr int CELLS = 2;
    static constexpr int VEC = 8;
    static constexpr int PAD = -16384;
    static constexpr int CEIL = 32767;

    // constants saturate to the lane range
    __device__ __forceinline__ static T splat(int v)
    {
        v = max(-32768, min(32767, v));
        return (uint32_t)(v & 0xffff) * 0x10001u;
    }
    __device__ __forceinline__ static T zero() { return 0u; }
    __device__ __forceinline__ static T addmax_relu(T a, T b, T c) { return __viaddmax_s16x2_relu(a, b, c); }
    __device__ __forceinline__ static T addmax(T a, T b, T c) { return __viaddmax_s16x2(a, b, c); }
    // a + b per half; the floor 0x8000 never binds for the bounded values used here
    __device__ __forceinline__ static T add(T a, T b) { return __viaddmax_s16x2(a, b, 0x80008000u); }
    __device__ __forceinline__ static T max2(T a, T b) { return __vmaxs2(a, b); }
    __device__ __forceinline__ static T max3(T a, T b, T c) { return __vimax3_s16x2(a, b, c); }
    __device__ __forceinline__ static bool any_pos(T a)
    {
        return (int16_t)(a & 0xffffu) > 0 || (int16_t)(a >> 16) > 0;
    }
    __device__ __forceinline__ static int get(T a, int c) { return (int)(int16_t)(c ? (a >> 16) : (a & 0xffffu)); }
    __device__ __forceinline__ static T shfl_up(T a, int d, int w) { return __shfl_up_sync(0xffffffffu, a, d, w); }
    __device__ __forceinline__ static T shfl_xor(T a, int d, int w) { return __shfl_xor_sync(0xffffffffu, a, d, w); }
    __device__ __forceinline__ static T pack(const int *v)
    {
        return (uint32_t)(v[0] & 0xffff) | ((uint32_t)(v[1] & 0xffff) << 16);
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

struct LaneI8x4 {
    using T = uint32_t;
    using Elem = int8_t;
    static constexpr int CELLS = 4;
    static constexpr int VEC = 16;
    static constexpr int PAD = -128;
    static constexpr int CEIL = 127;

    // constants saturate to the lane range: a clamped negative weight gives
    // a saturated sum <= max(true sum, -128), which is inert wherever the
    // true sum was (every kept value is >= -o >= -127)
    __device__ __forceinline__ static T splat(int v)
    {
        v = max(-128, min(127, v));
        return (uint32_t)(v & 0xff) * 0x01010101u;
    }
    __device__ __forceinline__ static T zero() { return 0u; }
    // saturating byte adds: a sum above 127 pins at 127 and flags the alignment
    __device__ __forceinline__ static T addmax_relu(T a, T b, T c)
    {
        return __vmaxs4(__vmaxs4(__vaddss4(a, b), c), 0u);
    }
    __device__ __forceinline__ static T addmax(T a, T b, T c) { return __vmaxs4(__vaddss4(a, b), c); }
    __device__ __forceinline__ static T add(T a, T b) { return __vaddss4(a, b); }
    __device__ __forceinline__ static T max2(T a, T b) { return __vmaxs4(a, b); }
    __device__ __forceinline__ static T max3(T a, T b, T c) { return __vmaxs4(__vmaxs4(a, b), c); }
    __device__ __forceinline__ static bool any_pos(T a)
    {
        return (int8_t)a > 0 || (int8_t)(a >> 8) > 0 || (int8_t)(a >> 16) > 0 || (int8_t)(a >> 24) > 0;
    }
    __device__ __forceinline__ static int get(T a, int c) { return (int)(int8_t)(a >> (8 * c)); }
    __device__ __forceinline__ static T shfl_up(T a, int d, int w) { return __shfl_up_sync(0xffffffffu, a, d, w); }
    __device__ __forceinline__ static T shfl_xor(T a, int d, int w) { return __shfl_xor_sync(0xffffffffu, a, d, w); }
    __device__ __forceinline__ static T pack(const int *v)
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

}  // namespace swg
