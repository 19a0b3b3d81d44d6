// Auxiliary kernels: striped profile build, length-binned work order,
// overflow flagging, and the integer-throughput probe used for the ALU
// roofline.
#include <stdint.h>

#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swg {

// ---------------------------------------------------------------------------
// Striped query profile (Alg. 1 "vprofile"): for chunk c, residue a, lane l,
// segment index j the score M[Q[c*L*S + l*S + j]][a]; 0 past the query end
// (the batch kernel makes those positions inert when it stages the chunk).
// Layout [C][A][L][S] int8.
// ---------------------------------------------------------------------------
__global__ void profile_build_kernel(const uint8_t *__restrict__ query, int32_t qlen, const int8_t *__restrict__ M,
                                     int32_t A, int32_t L, int32_t S, int32_t C, int8_t *__restrict__ prof)
{
    const int64_t QC = (int64_t)L * S;
    const int64_t total = (int64_t)C * A * QC;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / (A * QC);
        const int64_t rem = i - c * A * QC;
        const int a = (int)(rem / QC);
        const int64_t pos = rem - (int64_t)a * QC;  // l*S + j
        const int64_t q = c * QC + pos;
        prof[i] = q < qlen ? M[(int)query[q] * A + a] : (int8_t)0;
    }
}

int launch_profile_build(const uint8_t *d_query, int32_t qlen, const int8_t *d_M, int32_t A, const Plan &pl,
                         int8_t *d_prof, cudaStream_t st)
{
    const int64_t total = (int64_t)pl.C * A * pl.L * pl.S;
    if (total == 0)
        return (int)cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    profile_build_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_query, qlen, d_M, A, pl.L, pl.S, pl.C, d_prof);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Length-binned order, longest bin first.  Key: 0 for empty, else
// 1 + 4*floor(log2 n) + the two bits below the leading one (quarter-octave
// bins).  Within a bin the order is whatever the atomics give; every
// sequence's score is independent of the order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int length_key(int64_t n)
{
    if (n <= 0)
        return 0;
    const unsigned v = (unsigned)min(n, (int64_t)0x7fffffff);
    const int lg = 31 - __clz(v);
    const int frac = lg >= 2 ? (int)((v >> (lg - 2)) & 3u) : 0;
    return 1 + 4 * lg + frac;
}

__global__ void length_hist_kernel(const int64_t *__restrict__ off, int64_t n, int32_t *hist)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[length_key(off[i + 1] - off[i])], 1);
}

// one block of NBINS threads: cursor[k] = number of sequences in bins > k
__global__ void length_scan_kernel(const int32_t *hist, int32_t *cursor)
{
    __shared__ int32_t h[NBINS];
    const int k = threadIdx.x;
    h[k] = hist[k];
    __syncthreads();
    int32_t s = 0;
    for (int b = k + 1; b < NBINS; ++b)
        s += h[b];
    cursor[k] = s;
}

__global__ void length_scatter_kernel(const int64_t *__restrict__ off, int64_t n, int32_t *cursor,
                                      int32_t *__restrict__ order)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&cursor[length_key(off[i + 1] - off[i])], 1);
        order[pos] = (int32_t)i;
    }
}

int launch_length_order(const int64_t *off, int64_t n, int32_t *order, int32_t *bins, cudaStream_t st, int num_sms)
{
    if (n <= 0)
        return (int)cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 8)
        blocks = (int64_t)num_sms * 8;
    length_hist_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n, bins);
    length_scan_kernel<<<1, NBINS, 0, st>>>(bins, bins + NBINS);
    length_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n, bins + NBINS, order);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Overflow flagging of packed-lane results (the paper does not cover lane
// overflow).  A packed lane is exact until some H + M exceeds the lane
// ceiling; that H was an exact value already folded into the alignment's
// maximum, so any alignment whose lane result reached ceiling - max(M) is
// listed for an int32 rescore.
// ---------------------------------------------------------------------------
__global__ void flag_overflow_kernel(const int32_t *__restrict__ scores, int64_t n, int32_t thresh, int32_t *list,
                                     int32_t *count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (scores[i] >= thresh)
            list[atomicAdd(count, 1)] = (int32_t)i;
}

int launch_flag_overflow(const int32_t *scores, int64_t n, int32_t thresh, int32_t *list, int32_t *count,
                         cudaStream_t st, int num_sms)
{
    if (n <= 0)
        return (int)cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 8)
        blocks = (int64_t)num_sms * 8;
    flag_overflow_kernel<<<(unsigned)blocks, 256, 0, st>>>(scores, n, thresh, list, count);
    return (int)cudaGetLastError();
}

// Pieces of the long sequences.  The reservation of a sequence's k slots
// retries a bounded number of times under contention; a sequence that does
// not get its slots (the cap is reached) is aligned whole.
__global__ void piece_plan_kernel(const int64_t *__restrict__ off, int64_t n, int32_t piece_len, int32_t stride,
                                  int32_t cap, Piece *pieces, int32_t *n_pieces, uint8_t *split, int32_t *scores)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t start = off[i];
        const int64_t len = off[i + 1] - start;
        uint8_t s = 0;
        if (len > piece_len) {
            const int64_t k = 1 + (len - piece_len + stride - 1) / stride;
            int32_t base = -1;
            if (k <= cap) {
                int32_t old = *((volatile int32_t *)n_pieces);
                for (int tries = 0; tries < (1 << 16) && old + k <= cap; ++tries) {
                    const int32_t prev = atomicCAS(n_pieces, old, old + (int32_t)k);
                    if (prev == old) {
                        base = old;
                        break;
                    }
                    old = prev;
                }
            }
            if (base >= 0) {
                for (int64_t j = 0; j < k; ++j) {
                    const int64_t c0 = j * stride;
                    Piece pc;
                    pc.start = start + c0;
                    pc.seq = (int32_t)i;
                    pc.len = (int32_t)(len - c0 < piece_len ? len - c0 : piece_len);
                    pieces[base + j] = pc;
                }
                scores[i] = 0;
                s = 1;
            }
        }
        split[i] = s;
    }
}

int launch_piece_plan(const int64_t *off, int64_t n, int32_t piece_len, int32_t stride, int32_t cap,
                      Piece *pieces, int32_t *n_pieces, uint8_t *split, int32_t *scores, cudaStream_t st,
                      int num_sms)
{
    if (n <= 0)
        return (int)cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 8)
        blocks = (int64_t)num_sms * 8;
    piece_plan_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n, piece_len, stride, cap, pieces, n_pieces, split,
                                                         scores);
    return (int)cudaGetLastError();
}

__global__ void flag_overflow_list_kernel(const int32_t *__restrict__ scores, const int32_t *__restrict__ list,
                                          int64_t n, int32_t thresh, int32_t *out, int32_t *out_count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = list[i];
        if (scores[id] >= thresh)
            out[atomicAdd(out_count, 1)] = id;
    }
}

int launch_flag_overflow_list(const int32_t *scores, const int32_t *list, int64_t n, int32_t thresh, int32_t *out,
                              int32_t *out_count, cudaStream_t st, int num_sms)
{
    if (n <= 0)
        return (int)cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 8)
        blocks = (int64_t)num_sms * 8;
    flag_overflow_list_kernel<<<(unsigned)blocks, 256, 0, st>>>(scores, list, n, thresh, out, out_count);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Query-length classes of the pair kernel (counting sort by class).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pair_class(int64_t qlen, const ClassTable &t)
{
    for (int k = 0; k < t.n; ++k)
        if (qlen <= t.q[k])
            return k;
    return t.n;
}

__global__ void pair_class_hist_kernel(const int64_t *__restrict__ q_off, int64_t n, const ClassTable t,
                                       int32_t *hist)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[pair_class(q_off[i + 1] - q_off[i], t)], 1);
}

__global__ void pair_class_scan_kernel(const int32_t *hist, int32_t *cursor, int ncls)
{
    if (threadIdx.x == 0) {
        int32_t s = 0;
        for (int k = 0; k <= ncls; ++k) {
            cursor[k] = s;
            s += hist[k];
        }
    }
}

__global__ void pair_class_scatter_kernel(const int64_t *__restrict__ q_off, int64_t n, const ClassTable t,
                                          int32_t *cursor, int32_t *__restrict__ order)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&cursor[pair_class(q_off[i + 1] - q_off[i], t)], 1);
        order[pos] = (int32_t)i;
    }
}

int launch_pair_classes(const int64_t *q_off, int64_t n_pairs, const ClassTable &t, int32_t *hist, int32_t *cursor,
                        int32_t *order, cudaStream_t st, int num_sms)
{
    if (n_pairs <= 0)
        return (int)cudaSuccess;
    int64_t blocks = (n_pairs + 255) / 256;
    if (blocks > (int64_t)num_sms * 8)
        blocks = (int64_t)num_sms * 8;
    pair_class_hist_kernel<<<(unsigned)blocks, 256, 0, st>>>(q_off, n_pairs, t, hist);
    pair_class_scan_kernel<<<1, 32, 0, st>>>(hist, cursor, t.n);
    pair_class_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(q_off, n_pairs, t, cursor, order);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cell-rate probe.  Each thread updates K positions per column with the
// exact instruction sequence of a scan-F pass (no loads, shuffles or scan),
// so the measured rate is the ceiling of that sequence on this GPU.  CORR:
// the shorter corrected pass (every substitution score >= -o), which raises
// the diagonal and E by the decaying carry d; AC: the always-corrected pass
// of the long-query split kernels (the floor of H on the diagonal, h one DPX
// add-max); else the plain general pass.
// op 0: int32 cells, 1: s16x2, 2: s8x4 (plain only).
// ---------------------------------------------------------------------------
template <class LT, bool CORR = false, bool AC = false>
__global__ void __launch_bounds__(256) cell_peak_kernel(int iters, int seed, uint32_t one, int *sink)
{
    using T = typename LT::T;
    constexpr int K = 16;
    const typename LT::K k = LT::consts(11, 1, K, one);
    T X[K], E[K];
    T P0 = LT::splat(((seed + threadIdx.x) & 7) + 11), P1 = LT::splat((((seed >> 3) + threadIdx.x) & 7) + 11);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        X[j] = k.xinit;
        E[j] = k.hzero;
    }
    T mx = k.hzero;
    for (int it = 0; it < iters; ++it) {
        T hd = X[K - 1];
        T F = k.xzero;
        T hpair = k.hzero;
        T d = LT::d0_of(X[K / 2], k);  // a carry that changes every column
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const T h = AC ? LT::addmax(hd, (j & 1) ? P1 : P0, E[j]) : LT::h_of(hd, (j & 1) ? P1 : P0, E[j], k);
            const T ho = LT::ho_of(h, k);
            if constexpr (AC) {
                hd = LT::max3(X[j], d, k.xinit);
                d = LT::dstep(d, k);
                X[j] = LT::addmax(F, k.negO, ho);
                E[j] = LT::max3(LT::fadd(E[j], k.negE32, k), d, X[j]);
            } else if constexpr (CORR) {
                hd = LT::xd_corr(X[j], d, k);
                d = LT::dstep(d, k);
                X[j] = LT::addmax(F, k.negO, ho);
                E[j] = LT::e_next_corr(E[j], d, X[j], k);
            } else {
                hd = X[j];
                X[j] = LT::addmax(F, k.negO, ho);
                E[j] = LT::e_next(E[j], X[j], k);
            }
            F = LT::addmax(F, k.negE, ho);
            if (j & 1)
                mx = LT::max3(mx, hpair, h);
            else
                hpair = h;
        }
        const T t = P0;
        P0 = P1;
        P1 = t;
    }
    int acc = 0;
#pragma unroll
    for (int j = 0; j < K; ++j)
        acc ^= (int)X[j] ^ (int)E[j];
    acc ^= (int)mx;
    if (acc == 0x7fffffff)
        sink[0] = acc;
}

int run_int_peak(int op, bool corrected, bool always, int blocks, int threads, int iters, double *cells, float *ms,
                 cudaStream_t st)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int *sink = nullptr;
    cudaError_t err = cudaMallocAsync((void **)&sink, sizeof(int), st);
    if (err != cudaSuccess)
        return (int)err;
    const uint32_t one = 1;
    auto go = [&](void) {
        if (op == 1 && always)
            cell_peak_kernel<LaneI16x2D, true, true><<<blocks, threads, 0, st>>>(iters, 12345, one, sink);
        else if (op == 0 && corrected)
            cell_peak_kernel<LaneI32D, true><<<blocks, threads, 0, st>>>(iters, 12345, one, sink);
        else if (op == 0)
            cell_peak_kernel<LaneI32><<<blocks, threads, 0, st>>>(iters, 12345, one, sink);
        else if (op == 1 && corrected)
            cell_peak_kernel<LaneI16x2D, true><<<blocks, threads, 0, st>>>(iters, 12345, one, sink);
        else if (op == 1)
            cell_peak_kernel<LaneI16x2><<<blocks, threads, 0, st>>>(iters, 12345, one, sink);
        else
            cell_peak_kernel<LaneI8x4><<<blocks, threads, 0, st>>>(iters, 12345, one, sink);
    };
    go();  // warm-up
    cudaEventRecord(a, st);
    go();
    cudaEventRecord(b, st);
    err = cudaEventSynchronize(b);
    float t = 0.f;
    if (err == cudaSuccess)
        err = cudaEventElapsedTime(&t, a, b);
    cudaFreeAsync(sink, st);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (err != cudaSuccess)
        return (int)err;
    const int cells_per_reg = op == 0 ? 1 : (op == 1 ? 2 : 4);
    *cells = 16.0 * (double)iters * (double)blocks * (double)threads * cells_per_reg;
    *ms = t;
    return (int)cudaGetLastError();
}

}  // namespace swg
