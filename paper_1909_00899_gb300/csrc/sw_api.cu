// C ABI of the library (declared in include/sw_gb300.h): argument checks,
// plans, library-owned scratch, launches.  Every compute step runs in the
// kernels of this directory; there is no host fallback.
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>

#include "sw_gb300.h"
#include "sw_internal.h"

namespace swg {
int launch_batch_i32(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_i16(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_i8(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_q16(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_i32_ends(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_q16_ends(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st);
// launches that split long sequences into pieces (layouts of <= 1024 positions)
int launch_batch_i32_pieces(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_i16_pieces(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_i8_pieces(const Plan &pl, const BatchArgs &a, int num_sms, cudaStream_t st);
int launch_batch_q16_pieces(const Plan &pl, bool lazy, const BatchArgs &a, int num_sms, cudaStream_t st);
}  // namespace swg

using swg::Plan;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(int err, const char *what)
{
    return fail(err == (int)cudaErrorMemoryAllocation ? SW_ERR_NOMEM : SW_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString((cudaError_t)err));
}

int num_sms_of(int dev)
{
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64)
        return 1;
    if (!cache[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

// Keep freed scratch in the device's default pool instead of returning it
// at every synchronisation (set once per device).
void keep_pool_warm(int dev)
{
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || done[dev])
        return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

struct Choice {
    int L, S;
};

// Lanes per alignment and segment length per lane type, smallest chunk that
// holds the query first; longer queries use the last entry in chunks.
// (measured on GB300: the widest segment that keeps padding low wins,
// 32 lanes x 32 positions for long queries)
const Choice kI32[] = {{4, 8}, {8, 8}, {16, 8}, {32, 8}, {32, 16}, {32, 32}};
const Choice kI16[] = {{8, 8}, {16, 8}, {32, 8}, {32, 16}, {32, 32}};
const Choice kI8[] = {{8, 16}, {16, 16}, {32, 16}};
// split-query s16x2: virtual lanes (two per thread)
const Choice kQ16[] = {{16, 8}, {32, 8}, {64, 8}, {64, 16}, {64, 32}};
// every (lanes, segment length) the batch kernels are instantiated for
const Choice kAllI32[] = {{1, 16}, {1, 32}, {4, 8},   {4, 32},  {8, 8},  {8, 16}, {16, 8},
                          {16, 16}, {32, 8}, {32, 12}, {32, 16}, {8, 32}, {16, 32}, {32, 32}};
const Choice kAllI16[] = {{8, 8}, {8, 16}, {16, 8}, {16, 16}, {32, 8}, {32, 12}, {32, 16}, {16, 32}, {32, 24}, {32, 32}};
const Choice kAllI8[] = {{8, 16}, {16, 16}, {32, 16}};
const Choice kAllQ16[] = {{2, 16}, {2, 32}, {16, 8},  {16, 32}, {32, 8},  {32, 12}, {32, 16}, {32, 20}, {32, 24},
                          {32, 32}, {32, 40}, {64, 8}, {64, 16}, {64, 20}, {64, 24}, {64, 28}, {64, 32}, {64, 40}};

bool plan_supported(int lane, int L, int S)
{
    const Choice *t = lane == SW_LANE_I32     ? kAllI32
                      : lane == SW_LANE_I16X2 ? kAllI16
                      : lane == SW_LANE_I8X4  ? kAllI8
                                              : kAllQ16;
    const int n = lane == SW_LANE_I32 ? 14 : (lane == SW_LANE_I16X2 ? 10 : lane == SW_LANE_I8X4 ? 3 : 18);
    for (int i = 0; i < n; ++i)
        if (t[i].L == L && t[i].S == S)
            return true;
    return false;
}

// query-length classes of the pair kernel (one query per pair, <= 512)
const Choice kPairI32[] = {{4, 8}, {8, 8}, {16, 8}, {16, 10}, {32, 8}, {32, 16}};
const Choice kPairI16[] = {{8, 8}, {16, 8}, {16, 10}, {32, 8}, {32, 16}};
const Choice kPairI8[] = {{8, 16}, {16, 10}, {16, 16}, {32, 16}};
const Choice kPairQ16[] = {{16, 8}, {16, 10}, {32, 8}, {32, 12}, {32, 16}};  // virtual lanes
const int kPairI32N = 6, kPairI16N = 5, kPairI8N = 4, kPairQ16N = 5;

// Automatic choice of lane type and layout: the layout maximising
// its measured single-chunk rate on GB300 (GCUPS per processed cell, 100k
// log-normal protein sequences, the query as long as one chunk; the
// split layouts with the always-corrected pass where it runs; 32 x 40 and
// 64 x 40 from their multi-chunk runs at m = 5000; refined per workload by
// the autotuner) x (useful positions / chunk positions) / (1 + 1.5 % per
// extra chunk: each chunk launch re-streams the database, hands boundary
// rows on and drains its own tail).
struct AutoChoice {
    int lane, L, S;
    double gcups;
};
const AutoChoice kAuto[] = {
    {SW_LANE_I16X2Q, 16, 8, 2894},  {SW_LANE_I16X2Q, 16, 32, 4491}, {SW_LANE_I16X2Q, 32, 8, 4290},
    {SW_LANE_I16X2Q, 32, 16, 4340},
    {SW_LANE_I16X2Q, 32, 12, 4157}, {SW_LANE_I16X2Q, 32, 20, 4680}, {SW_LANE_I16X2Q, 32, 24, 5109},
    {SW_LANE_I16X2Q, 32, 32, 5127}, {SW_LANE_I16X2Q, 32, 40, 5523}, {SW_LANE_I16X2Q, 64, 8, 4388},
    {SW_LANE_I16X2Q, 64, 16, 4932}, {SW_LANE_I16X2Q, 64, 20, 5110}, {SW_LANE_I16X2Q, 64, 24, 5340},
    {SW_LANE_I16X2Q, 64, 28, 5218}, {SW_LANE_I16X2Q, 64, 32, 5547}, {SW_LANE_I16X2Q, 64, 40, 5245},
    {SW_LANE_I16X2, 32, 16, 3865},  {SW_LANE_I16X2, 32, 32, 4578},
};
constexpr double kChunkCost = 0.015;

Plan choose_auto(int32_t qlen)
{
    Plan best;
    double best_rate = -1.0;
    for (const AutoChoice &c : kAuto) {
        const int QC = c.L * c.S;
        const int C = qlen > 0 ? (qlen + QC - 1) / QC : 1;
        const double rate =
            c.gcups * (double)std::max(qlen, 1) / ((double)C * QC) / (1.0 + kChunkCost * (double)(C - 1));
        if (rate > best_rate) {
            best_rate = rate;
            best.lane = c.lane;
            best.L = c.L;
            best.S = c.S;
            best.C = qlen > 0 ? C : 0;
        }
    }
    return best;
}

Plan choose_plan(int32_t qlen, int lane)
{
    const Choice *tab = kI32;
    int n = 6;
    if (lane == SW_LANE_I16X2) {
        tab = kI16;
        n = 5;
    } else if (lane == SW_LANE_I8X4) {
        tab = kI8;
        n = 3;
    } else if (lane == SW_LANE_I16X2Q) {
        tab = kQ16;
        n = 5;
    }
    Plan p;
    p.lane = lane;
    int k = 0;
    while (k + 1 < n && tab[k].L * tab[k].S < qlen)
        ++k;
    p.L = tab[k].L;
    p.S = tab[k].S;
    const int QC = p.L * p.S;
    p.C = qlen > 0 ? (qlen + QC - 1) / QC : 0;
    return p;
}

// Largest score bias and scan weights a lane type must hold.
bool lane_fits(int lane, const sw_profile *pf, int32_t o, int32_t e, const Plan &pl)
{
    if (lane == SW_LANE_I32)
        return true;
    const int64_t ceil = lane == SW_LANE_I8X4 ? 127 : 32767;
    if (lane == SW_LANE_I8X4 && (int64_t)pf->maxM + o > ceil)
        return false;
    if (o > 127)
        return false;
    if (lane == SW_LANE_I16X2 || lane == SW_LANE_I16X2Q) {
        // biased halves stay positive: 2o + S*e below the X-space bias (4096),
        // the deepest scan hop (and the split lane's fold of the first half,
        // up to L*S*e over its L = plan lanes / 2 threads) above -32768
        if (2LL * o + (int64_t)pl.S * e + 256 > 4096)
            return false;
        if (4096LL - o - (int64_t)pl.L * pl.S * e < -32000)
            return false;
    } else {
        // the last-position correction subtracts (S-1)*e in one saturating add
        if ((int64_t)(pl.S - 1) * e > 127)
            return false;
    }
    return true;
}

// True score from which a packed lane's result is rescored in int32: the
// first addition H + M that can leave the lane range needs H above it.
int32_t flag_threshold(int lane, int32_t o, int32_t maxM)
{
    const int32_t m = std::max(maxM, 0);
    if (lane == SW_LANE_I16X2 || lane == SW_LANE_I16X2Q)
        return 32767 - (4096 + 128 - o) - m;  // s16x2: h-space bias 4096 + 128 - o
    if (lane == SW_LANE_I8X4)
        return 127 - m;
    return INT32_MAX;
}

struct Scratch {
    void *base = nullptr;
    cudaStream_t st = nullptr;
    ~Scratch()
    {
        if (base)
            cudaFreeAsync(base, st);
    }
};

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

int check_align_args(const sw_profile *prof, const uint8_t *db, const int64_t *off, int64_t n_db, int32_t o,
                     int32_t e, int32_t *scores)
{
    if (!prof)
        return fail(SW_ERR_INVALID, "profile is NULL");
    if (n_db < 0)
        return fail(SW_ERR_INVALID, "n_db < 0 (%lld)", (long long)n_db);
    if (n_db > INT32_MAX - 1024)
        return fail(SW_ERR_INVALID, "n_db too large (%lld)", (long long)n_db);
    if (n_db > 0 && (!db || !off || !scores))
        return fail(SW_ERR_INVALID, "null device pointer");
    if (o < 1)
        return fail(SW_ERR_INVALID, "gap_open must be >= 1 (got %d)", o);
    if (e < 0 || e > o)
        return fail(SW_ERR_INVALID, "gap_extend must satisfy 0 <= e <= gap_open (got e=%d, o=%d)", e, o);
    if (o > (1 << 20))
        return fail(SW_ERR_RANGE, "gap_open too large for int32 accumulation (%d)", o);
    if ((int64_t)prof->qlen * std::max(prof->maxM, 0) >= (1LL << 24))
        return fail(SW_ERR_RANGE, "query length x largest score exceeds the int32 working range");
    return SW_OK;
}

int launch_plan(const Plan &pl, bool lazy, const swg::BatchArgs &a, int sms, cudaStream_t st)
{
    if (a.pieces) {
        if (pl.lane == SW_LANE_I32)
            return swg::launch_batch_i32_pieces(pl, lazy, a, sms, st);
        if (pl.lane == SW_LANE_I16X2)
            return swg::launch_batch_i16_pieces(pl, lazy, a, sms, st);
        if (pl.lane == SW_LANE_I16X2Q)
            return swg::launch_batch_q16_pieces(pl, lazy, a, sms, st);
        return swg::launch_batch_i8_pieces(pl, a, sms, st);
    }
    if (pl.lane == SW_LANE_I32)
        return swg::launch_batch_i32(pl, lazy, a, sms, st);
    if (pl.lane == SW_LANE_I16X2)
        return swg::launch_batch_i16(pl, lazy, a, sms, st);
    if (pl.lane == SW_LANE_I16X2Q)
        return swg::launch_batch_q16(pl, lazy, a, sms, st);
    return swg::launch_batch_i8(pl, a, sms, st);
}

// Splitting of long sequences: pieces of at least this many columns (a
// short query keeps a few thousand columns of serial work per item), and no
// splitting when pieces would be longer than the cap (the span grows with
// m x max M / e; beyond the cap hardly any database sequence is longer than
// a piece, and the splitting kernels would only add their per-item cost).
constexpr int64_t kMinPieceLen = 2048;
constexpr int64_t kMaxPieceLen = 8192;
// layouts instantiated for splitting launches: at most this many positions
// per chunk (longer queries have spans beyond any usual database sequence)
constexpr int kPieceMaxChunk = 1024;

// pre_order / pre_total: a database handle's persistent length order and
// residue count (then no order kernels run and nothing is read back).
// q_end / r_end: end cells wanted (ENDS kernels: split s16x2 lanes for split
// profiles, int32 lanes otherwise and for the rescore)
int align_impl(const sw_profile *prof, const uint8_t *db, const int64_t *off, int64_t n_db, int32_t o, int32_t e,
               int32_t *scores, void *stream, bool lazy, const int32_t *pre_order = nullptr,
               int64_t pre_total = -1, unsigned long long *lazy_steps = nullptr, int32_t *q_end = nullptr,
               int32_t *r_end = nullptr)
{
    int rc = check_align_args(prof, db, off, n_db, o, e, scores);
    if (rc)
        return rc;
    const bool ends = q_end != nullptr;
    if (ends && (!r_end || lazy))
        return fail(SW_ERR_INVALID, "end cells need q_end and r_end (scan-F only)");
    if (n_db == 0)
        return SW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (prof->qlen == 0) {
        cudaError_t err = cudaMemsetAsync(scores, 0, sizeof(int32_t) * (size_t)n_db, st);
        if (err == cudaSuccess && ends)
            err = cudaMemsetAsync(q_end, 0xff, sizeof(int32_t) * (size_t)n_db, st);
        if (err == cudaSuccess && ends)
            err = cudaMemsetAsync(r_end, 0xff, sizeof(int32_t) * (size_t)n_db, st);
        return err == cudaSuccess ? SW_OK : cuda_fail(err, "cudaMemsetAsync");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != prof->device)
        return fail(SW_ERR_INVALID, "profile built on device %d, current device is %d", prof->device, dev);
    keep_pool_warm(dev);
    const int sms = num_sms_of(dev);

    // lazy-F runs on the profile's own layout (int32, two-alignment or split
    // s16x2; s8x4 profiles fall back to int32)
    int lane = prof->lane;
    if ((lazy && lane == SW_LANE_I8X4) || (ends && lane != SW_LANE_I16X2Q))
        lane = SW_LANE_I32;
    if (lane != SW_LANE_I32 && !lane_fits(lane, prof, o, e, prof->plan))
        lane = SW_LANE_I32;  // values do not fit the packed lanes: exact int32 throughout
    const Plan main = lane == SW_LANE_I32 ? prof->plan32 : prof->plan;
    const int8_t *main_prof = lane == SW_LANE_I32 ? prof->d_prof32 : prof->d_prof;
    const bool packed = lane != SW_LANE_I32;
    const int C32 = prof->plan32.C;

    // total residues, needed only to size the boundary rows of long queries
    int64_t total = pre_total > 0 ? pre_total : 0;
    const bool chunked = main.C > 1 || (packed && C32 > 1);
    if (chunked && pre_total < 0) {
        cudaError_t err = cudaMemcpyAsync(&total, off + n_db, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaStreamSynchronize(st);
        if (err != cudaSuccess)
            return cuda_fail(err, "reading db_offsets[n_db]");
        if (total < 0)
            return fail(SW_ERR_INVALID, "db_offsets[n_db] < 0");
    }

    // Long sequences against a short single-chunk query: split into pieces
    // that overlap by the widest span a positive-scoring local alignment can
    // have (m aligned pairs at most, and each column of horizontal gap costs
    // at least e, so it spans at most m + (m * max M - 1) / e columns).  Every
    // optimal alignment then lies inside one piece, so the best piece score is
    // the sequence's score, while the longest work item shrinks to the piece
    // length: a single short query no longer waits on one warp that walks the
    // longest sequence alone.  Scores only (end cells and the lazy-F
    // statistics keep whole sequences).
    int32_t piece_len = 0, piece_stride = 0;
    if (!ends && !lazy_steps && main.C == 1 && (!packed || C32 == 1) && e >= 1 && prof->maxM >= 1 &&
        main.L * main.S <= kPieceMaxChunk && n_db < (int64_t)swg::PIECE_BIT) {
        const int64_t span = (int64_t)prof->qlen + ((int64_t)prof->qlen * prof->maxM - 1) / e;
        const int64_t plen = std::max<int64_t>(2 * span, kMinPieceLen);
        if (plen <= kMaxPieceLen) {
            piece_len = (int32_t)plen;
            piece_stride = (int32_t)(plen - span + 1);
        }
    }
    const bool pieces = piece_len > 0;

    const size_t n = (size_t)n_db;
    const int ncount = main.C + (packed ? C32 : 0) + 3;
    const size_t sz_order = pre_order ? 0 : align_up(n * 4);
    const size_t sz_zero = align_up((2 * swg::NBINS + ncount) * 4);
    const size_t sz_list = packed ? align_up(n * 4) : 0;
    const size_t sz_bnd = chunked ? align_up((size_t)total * sizeof(int2) + 16) : 0;
    const size_t sz_pieces = pieces ? align_up(n * sizeof(swg::Piece)) + align_up(n) : 0;
    Scratch sc;
    sc.st = st;
    cudaError_t err = cudaMallocAsync(&sc.base, sz_order + sz_zero + sz_list + sz_bnd + sz_pieces, st);
    if (err != cudaSuccess) {
        sc.base = nullptr;
        return cuda_fail(err, "cudaMallocAsync(scratch)");
    }
    char *p = (char *)sc.base;
    int32_t *order = pre_order ? const_cast<int32_t *>(pre_order) : (int32_t *)p;
    int32_t *zero = (int32_t *)(p + sz_order);
    int32_t *bins = zero;
    uint32_t *counters = (uint32_t *)(zero + 2 * swg::NBINS);
    int32_t *list_count = (int32_t *)(counters + main.C + (packed ? C32 : 0));
    int32_t *n_pieces = list_count + 1;
    int32_t *list = (int32_t *)(p + sz_order + sz_zero);
    int2 *bnd = chunked ? (int2 *)(p + sz_order + sz_zero + sz_list) : nullptr;
    swg::Piece *piece_arr = pieces ? (swg::Piece *)(p + sz_order + sz_zero + sz_list + sz_bnd) : nullptr;
    uint8_t *split = pieces ? (uint8_t *)piece_arr + align_up(n * sizeof(swg::Piece)) : nullptr;

    err = cudaMemsetAsync(zero, 0, sz_zero, st);
    if (err != cudaSuccess)
        return cuda_fail(err, "cudaMemsetAsync(scratch)");
    int kr = 0;
    if (!pre_order) {
        kr = swg::launch_length_order(off, n_db, order, bins, st, sms);
        if (kr)
            return cuda_fail(kr, "length order kernels");
    }

    swg::BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.A = prof->A;
    a.qlen = prof->qlen;
    a.db = db;
    a.off = off;
    a.order = order;
    a.n_work = n_db;
    a.o = o;
    a.e = e;
    a.bnd = bnd;
    a.scores = scores;
    a.one = 1;
    a.lazy_steps = lazy_steps;
    a.q_end = q_end;
    a.r_end = r_end;
    a.flag_thresh = flag_threshold(lane, o, prof->maxM);
    a.min_m = prof->minM;
    a.prof = main_prof;
    a.nchunks = main.C;
    if (pieces) {
        kr = swg::launch_piece_plan(off, n_db, piece_len, piece_stride, (int32_t)std::min<int64_t>(n_db, INT32_MAX),
                                    piece_arr, n_pieces, split, scores, st, sms);
        if (kr)
            return cuda_fail(kr, "piece plan kernel");
        a.pieces = piece_arr;
        a.n_pieces = n_pieces;
        a.split = split;
    }
    for (int c = 0; c < main.C; ++c) {
        a.chunk = c;
        a.counter = counters + c;
        kr = !ends                    ? launch_plan(main, lazy, a, sms, st)
             : lane == SW_LANE_I32    ? swg::launch_batch_i32_ends(main, a, sms, st)
                                      : swg::launch_batch_q16_ends(main, a, sms, st);
        if (kr)
            return cuda_fail(kr, "batch kernel launch");
    }
    if (packed) {
        kr = swg::launch_flag_overflow(scores, n_db, a.flag_thresh, list, list_count, st, sms);
        if (kr)
            return cuda_fail(kr, "overflow flag kernel");
        a.prof = prof->d_prof32;
        a.flag_thresh = INT32_MAX;
        a.nchunks = C32;
        a.pieces = nullptr;  // flagged sequences are rescored whole
        a.n_pieces = nullptr;
        a.split = nullptr;
        a.order = list;
        a.n_work = n_db;
        a.n_work_dev = list_count;
        for (int c = 0; c < C32; ++c) {
            a.chunk = c;
            a.counter = counters + main.C + c;
            kr = ends ? swg::launch_batch_i32_ends(prof->plan32, a, sms, st)
                      : launch_plan(prof->plan32, false, a, sms, st);
            if (kr)
                return cuda_fail(kr, "rescore kernel launch");
        }
    }
    return SW_OK;
}

}  // namespace

// Helpers shared with the other host translation units (sw_noalloc.cu).
namespace swg {
int api_fail(int code, const char *msg) { return fail(code, "%s", msg); }
int api_cuda_fail(int err, const char *what) { return cuda_fail(err, what); }
int api_num_sms(int dev) { return num_sms_of(dev); }
bool api_lane_fits(int lane, const sw_profile *pf, int32_t o, int32_t e, const Plan &pl)
{
    return lane_fits(lane, pf, o, e, pl);
}
int32_t api_flag_threshold(int lane, int32_t o, int32_t maxM) { return flag_threshold(lane, o, maxM); }
int api_check_align_args(const sw_profile *prof, const uint8_t *db, const int64_t *off, int64_t n_db, int32_t o,
                         int32_t e, int32_t *scores)
{
    return check_align_args(prof, db, off, n_db, o, e, scores);
}
int api_launch_plan(const Plan &pl, bool lazy, const BatchArgs &a, int sms, cudaStream_t st)
{
    return launch_plan(pl, lazy, a, sms, st);
}
}  // namespace swg

extern "C" {

const char *sw_last_error(void) { return g_err.c_str(); }

const char *sw_version(void) { return "0.1.0"; }

int sw_profile_build(const uint8_t *query, int32_t qlen, const int8_t *subst_matrix, int32_t alphabet,
                     int32_t lane_type, void *cuda_stream, sw_profile **out)
{
    return sw_profile_build_ex(query, qlen, subst_matrix, alphabet, lane_type, 0, 0, cuda_stream, out);
}

int sw_profile_build_ex(const uint8_t *query, int32_t qlen, const int8_t *subst_matrix, int32_t alphabet,
                        int32_t lane_type, int32_t lanes, int32_t seg_len, void *cuda_stream, sw_profile **out)
{
    if (!out)
        return fail(SW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (qlen < 0)
        return fail(SW_ERR_INVALID, "qlen < 0 (%d)", qlen);
    if (qlen > 0 && !query)
        return fail(SW_ERR_INVALID, "query is NULL");
    if (alphabet < 1 || alphabet > 32)
        return fail(SW_ERR_INVALID, "alphabet must be in 1..32 (got %d)", alphabet);
    if (!subst_matrix)
        return fail(SW_ERR_INVALID, "subst_matrix is NULL");
    if (lane_type < SW_LANE_AUTO || lane_type > SW_LANE_I16X2Q)
        return fail(SW_ERR_INVALID, "unknown lane_type %d", lane_type);
    for (int32_t i = 0; i < qlen; ++i)
        if (query[i] >= alphabet)
            return fail(SW_ERR_INVALID, "query residue %d at %d is >= alphabet %d", query[i], i, alphabet);

    sw_profile *pf = new sw_profile();
    pf->qlen = qlen;
    pf->A = alphabet;
    pf->maxM = -128;
    pf->minM = 127;
    for (int i = 0; i < alphabet * alphabet; ++i) {
        pf->maxM = std::max<int32_t>(pf->maxM, subst_matrix[i]);
        pf->minM = std::min<int32_t>(pf->minM, subst_matrix[i]);
    }
    int lane = lane_type;
    if (lane_type == SW_LANE_AUTO)
        lane = lanes ? SW_LANE_I16X2 : choose_auto(qlen).lane;
    if ((lanes == 0) != (seg_len == 0) || (lanes && !plan_supported(lane, lanes, seg_len))) {
        delete pf;
        return fail(SW_ERR_INVALID, "no kernel for lane type %d with %d lanes x %d positions", lane, lanes, seg_len);
    }
    pf->lane = lane;
    pf->plan = lane_type == SW_LANE_AUTO && !lanes ? choose_auto(qlen) : choose_plan(qlen, lane);
    if (lanes) {
        pf->plan.L = lanes;
        pf->plan.S = seg_len;
        pf->plan.C = qlen > 0 ? (qlen + lanes * seg_len - 1) / (lanes * seg_len) : 0;
    }
    // int32 profiles serve lazy-F and the rescore with their own layout
    pf->plan32 = lane == SW_LANE_I32 ? pf->plan : choose_plan(qlen, SW_LANE_I32);
    cudaGetDevice(&pf->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    pf->stream = st;
    keep_pool_warm(pf->device);

    const size_t qbytes = align_up((size_t)std::max(qlen, 1));
    const size_t mbytes = align_up((size_t)alphabet * alphabet);
    const size_t pbytes = align_up((size_t)pf->plan.C * alphabet * pf->plan.L * pf->plan.S);
    const size_t p32bytes =
        lane == SW_LANE_I32 ? 0 : align_up((size_t)pf->plan32.C * alphabet * pf->plan32.L * pf->plan32.S);
    cudaError_t err = cudaMallocAsync(&pf->block, qbytes + mbytes + pbytes + p32bytes, st);
    if (err != cudaSuccess) {
        pf->block = nullptr;
        delete pf;
        return cuda_fail(err, "cudaMallocAsync(profile)");
    }
    char *base = (char *)pf->block;
    pf->d_query = (uint8_t *)base;
    pf->d_M = (int8_t *)(base + qbytes);
    pf->d_prof = (int8_t *)(base + qbytes + mbytes);
    pf->d_prof32 = lane == SW_LANE_I32 ? pf->d_prof : (int8_t *)(base + qbytes + mbytes + pbytes);
    auto cleanup = [&](int code) {
        sw_profile_free_async(pf, st);
        return code;
    };
    if (qlen > 0)
        err = cudaMemcpyAsync(pf->d_query, query, (size_t)qlen, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(pf->d_M, subst_matrix, (size_t)alphabet * alphabet, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "profile upload"));
    if (qlen > 0) {
        int kr = swg::launch_profile_build(pf->d_query, qlen, pf->d_M, alphabet, pf->plan, pf->d_prof, st);
        if (!kr && lane != SW_LANE_I32)
            kr = swg::launch_profile_build(pf->d_query, qlen, pf->d_M, alphabet, pf->plan32, pf->d_prof32, st);
        if (kr)
            return cleanup(cuda_fail(kr, "profile build kernel"));
    }
    *out = pf;
    return SW_OK;
}

int sw_profile_free(sw_profile *prof)
{
    if (!prof)
        return SW_OK;
    // the profile may be in use on any stream: wait for the device first
    cudaError_t err = cudaDeviceSynchronize();
    if (prof->block)
        cudaFreeAsync(prof->block, prof->stream);
    cudaStreamSynchronize(prof->stream);
    delete prof;
    return err == cudaSuccess ? SW_OK : cuda_fail(err, "sw_profile_free");
}

int sw_profile_free_async(sw_profile *prof, void *cuda_stream)
{
    if (!prof)
        return SW_OK;
    cudaError_t err = cudaSuccess;
    if (prof->block)
        err = cudaFreeAsync(prof->block, (cudaStream_t)cuda_stream);
    delete prof;
    return err == cudaSuccess ? SW_OK : cuda_fail(err, "cudaFreeAsync(profile)");
}

int sw_profile_plan(const sw_profile *prof, int32_t *lanes, int32_t *seg_len, int32_t *chunks, int32_t *lane_type)
{
    if (!prof)
        return fail(SW_ERR_INVALID, "profile is NULL");
    if (lanes)
        *lanes = prof->plan.L;
    if (seg_len)
        *seg_len = prof->plan.S;
    if (chunks)
        *chunks = prof->plan.C;
    if (lane_type)
        *lane_type = prof->lane;
    return SW_OK;
}

int sw_plan_query(int32_t qlen, int32_t lane_type, int32_t *lanes, int32_t *seg_len, int32_t *chunks,
                  int32_t *lane_out)
{
    if (qlen < 0)
        return fail(SW_ERR_INVALID, "qlen < 0 (%d)", qlen);
    if (lane_type < SW_LANE_AUTO || lane_type > SW_LANE_I16X2Q)
        return fail(SW_ERR_INVALID, "unknown lane type %d", lane_type);
    const Plan pl = lane_type == SW_LANE_AUTO ? choose_auto(qlen) : choose_plan(qlen, lane_type);
    if (lanes)
        *lanes = pl.L;
    if (seg_len)
        *seg_len = pl.S;
    if (chunks)
        *chunks = pl.C;
    if (lane_out)
        *lane_out = pl.lane;
    return SW_OK;
}

int sw_align_batch(const sw_profile *prof, const uint8_t *db_residues, const int64_t *db_offsets, int64_t n_db,
                   int32_t gap_open, int32_t gap_extend, int32_t *scores_out, void *cuda_stream)
{
    return align_impl(prof, db_residues, db_offsets, n_db, gap_open, gap_extend, scores_out, cuda_stream, false);
}

int sw_align_batch_ends(const sw_profile *prof, const uint8_t *db_residues, const int64_t *db_offsets,
                        int64_t n_db, int32_t gap_open, int32_t gap_extend, int32_t *scores_out,
                        int32_t *q_end_out, int32_t *r_end_out, void *cuda_stream)
{
    if (n_db > 0 && (!q_end_out || !r_end_out))
        return fail(SW_ERR_INVALID, "q_end_out / r_end_out is NULL");
    return align_impl(prof, db_residues, db_offsets, n_db, gap_open, gap_extend, scores_out, cuda_stream, false,
                      nullptr, -1, nullptr, n_db > 0 ? q_end_out : nullptr, r_end_out);
}

int sw_align_lazyf_batch(const sw_profile *prof, const uint8_t *db_residues, const int64_t *db_offsets,
                         int64_t n_db, int32_t gap_open, int32_t gap_extend, int32_t *scores_out,
                         void *cuda_stream)
{
    return align_impl(prof, db_residues, db_offsets, n_db, gap_open, gap_extend, scores_out, cuda_stream, true);
}

int sw_db_create(const uint8_t *db_residues, const int64_t *db_offsets, int64_t n_db, void *cuda_stream,
                 sw_db **out)
{
    if (!out)
        return fail(SW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n_db < 0 || n_db > INT32_MAX - 1024)
        return fail(SW_ERR_INVALID, "n_db out of range (%lld)", (long long)n_db);
    if (n_db > 0 && (!db_residues || !db_offsets))
        return fail(SW_ERR_INVALID, "null device pointer");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    sw_db *d = new sw_db();
    cudaGetDevice(&d->device);
    d->res = db_residues;
    d->off = db_offsets;
    d->n = n_db;
    if (n_db == 0) {
        *out = d;
        return SW_OK;
    }
    int32_t *bins = nullptr;
    cudaError_t err = cudaMalloc(&d->order, sizeof(int32_t) * (size_t)n_db);
    if (err == cudaSuccess)
        err = cudaMalloc(&bins, sizeof(int32_t) * 2 * swg::NBINS);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(bins, 0, sizeof(int32_t) * 2 * swg::NBINS, st);
    if (err != cudaSuccess) {
        if (bins)
            cudaFree(bins);
        sw_db_free(d);
        return cuda_fail(err, "sw_db_create allocation");
    }
    int kr = swg::launch_length_order(db_offsets, n_db, d->order, bins, st, num_sms_of(d->device));
    if (!kr)
        kr = (int)cudaMemcpyAsync(&d->total, db_offsets + n_db, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (!kr)
        kr = (int)cudaStreamSynchronize(st);
    cudaFree(bins);
    if (kr) {
        sw_db_free(d);
        return cuda_fail(kr, "sw_db_create");
    }
    if (d->total < 0) {
        sw_db_free(d);
        return fail(SW_ERR_INVALID, "db_offsets[n_db] < 0");
    }
    *out = d;
    return SW_OK;
}

int sw_db_free(sw_db *db)
{
    if (!db)
        return SW_OK;
    if (db->order)
        cudaFree(db->order);
    delete db;
    return SW_OK;
}

int sw_align_db(const sw_profile *prof, const sw_db *db, int32_t gap_open, int32_t gap_extend, int32_t *scores_out,
                void *cuda_stream)
{
    if (!db)
        return fail(SW_ERR_INVALID, "db is NULL");
    return align_impl(prof, db->res, db->off, db->n, gap_open, gap_extend, scores_out, cuda_stream, false,
                      db->order, db->total);
}

int sw_align_db_ends(const sw_profile *prof, const sw_db *db, int32_t gap_open, int32_t gap_extend,
                     int32_t *scores_out, int32_t *q_end_out, int32_t *r_end_out, void *cuda_stream)
{
    if (!db)
        return fail(SW_ERR_INVALID, "db is NULL");
    if (db->n > 0 && (!q_end_out || !r_end_out))
        return fail(SW_ERR_INVALID, "q_end_out / r_end_out is NULL");
    return align_impl(prof, db->res, db->off, db->n, gap_open, gap_extend, scores_out, cuda_stream, false,
                      db->order, db->total, nullptr, db->n > 0 ? q_end_out : nullptr, r_end_out);
}

int sw_align_lazyf_db(const sw_profile *prof, const sw_db *db, int32_t gap_open, int32_t gap_extend,
                      int32_t *scores_out, void *cuda_stream)
{
    return sw_align_lazyf_db_stats(prof, db, gap_open, gap_extend, scores_out, nullptr, cuda_stream);
}

int sw_align_lazyf_db_stats(const sw_profile *prof, const sw_db *db, int32_t gap_open, int32_t gap_extend,
                            int32_t *scores_out, unsigned long long *lazy_steps, void *cuda_stream)
{
    if (!db)
        return fail(SW_ERR_INVALID, "db is NULL");
    return align_impl(prof, db->res, db->off, db->n, gap_open, gap_extend, scores_out, cuda_stream, true,
                      db->order, db->total, lazy_steps);
}

// q_end / r_end: end cells wanted (scan-F; split s16x2 or int32 pair kernels)
static int pairs_impl(const uint8_t *q, const int64_t *q_off, const uint8_t *r, const int64_t *r_off, int64_t n_pairs,
               const int8_t *subst_matrix, int32_t alphabet, int32_t gap_open, int32_t gap_extend,
               int32_t lane_type, int32_t *scores_out, void *cuda_stream, bool lazy,
               unsigned long long *lazy_steps, int32_t *q_end = nullptr, int32_t *r_end = nullptr)
{
    const bool ends = q_end != nullptr;
    if (n_pairs < 0)
        return fail(SW_ERR_INVALID, "n_pairs < 0 (%lld)", (long long)n_pairs);
    if (n_pairs > INT32_MAX - 1024)
        return fail(SW_ERR_INVALID, "n_pairs too large (%lld)", (long long)n_pairs);
    if (n_pairs > 0 && (!q || !q_off || !r || !r_off || !scores_out || (ends && !r_end)))
        return fail(SW_ERR_INVALID, "null device pointer");
    if (!subst_matrix)
        return fail(SW_ERR_INVALID, "subst_matrix is NULL");
    if (alphabet < 1 || alphabet > 32)
        return fail(SW_ERR_INVALID, "alphabet must be in 1..32 (got %d)", alphabet);
    if (lane_type < SW_LANE_AUTO || lane_type > SW_LANE_I16X2Q)
        return fail(SW_ERR_INVALID, "pairs take lane types AUTO, I32, I16X2, I8X4 or I16X2Q (got %d)", lane_type);
    if (gap_open < 1)
        return fail(SW_ERR_INVALID, "gap_open must be >= 1 (got %d)", gap_open);
    if (gap_extend < 0 || gap_extend > gap_open)
        return fail(SW_ERR_INVALID, "gap_extend must satisfy 0 <= e <= gap_open (got e=%d, o=%d)", gap_extend,
                    gap_open);
    if (gap_open > (1 << 20))
        return fail(SW_ERR_RANGE, "gap_open too large for int32 accumulation (%d)", gap_open);
    if (n_pairs == 0)
        return SW_OK;

    swg::PairArgs a;
    memset(&a, 0, sizeof(a));
    int32_t maxM = -128, minM = 127;
    for (int i = 0; i < alphabet * alphabet; ++i) {
        a.M[i] = subst_matrix[i];
        maxM = std::max<int32_t>(maxM, subst_matrix[i]);
        minM = std::min<int32_t>(minM, subst_matrix[i]);
    }
    a.min_m = minM;
    sw_profile shape;  // only the matrix range is read by lane_fits
    shape.maxM = maxM;
    // automatic: split s16x2 (one pair per group, no byte permutes), measured
    // fastest on reads vs windows
    // lazy-F: int32 lanes, or the split s16x2 layout when asked for
    int lane = lazy ? (lane_type == SW_LANE_I16X2Q ? SW_LANE_I16X2Q : SW_LANE_I32)
                    : (lane_type == SW_LANE_AUTO ? SW_LANE_I16X2Q : lane_type);
    if (ends && lane != SW_LANE_I16X2Q)
        lane = SW_LANE_I32;  // end cells: split s16x2 or int32 kernels
    // query-length classes of the lane type; the packed classes must fit
    const Choice *tab = kPairI32;
    int ncls = kPairI32N;
    if (lane == SW_LANE_I16X2) {
        tab = kPairI16;
        ncls = kPairI16N;
    } else if (lane == SW_LANE_I8X4) {
        tab = kPairI8;
        ncls = kPairI8N;
    } else if (lane == SW_LANE_I16X2Q) {
        tab = kPairQ16;
        ncls = kPairQ16N;
    }
    if (lane != SW_LANE_I32) {
        Plan widest;
        widest.L = tab[ncls - 1].L;
        widest.S = tab[ncls - 1].S;
        if (!lane_fits(lane, &shape, gap_open, gap_extend, widest)) {
            lane = SW_LANE_I32;
            tab = kPairI32;
            ncls = kPairI32N;
        }
    }
    swg::ClassTable ct;
    ct.n = ncls;
    for (int k = 0; k < ncls; ++k)
        ct.q[k] = tab[k].L * tab[k].S;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_warm(dev);
    const int sms = num_sms_of(dev);
    const size_t n = (size_t)n_pairs;
    // hist, cursor (ncls + 1 each), 2 work counters and 1 list count per class
    const size_t sz_small = align_up((size_t)(2 * (ncls + 1) + 3 * ncls) * 4);
    const size_t sz_order = align_up(n * 4);
    const size_t sz_list = lane != SW_LANE_I32 ? align_up(n * 4) : 0;
    Scratch sc;
    sc.st = st;
    cudaError_t err = cudaMallocAsync(&sc.base, sz_small + sz_order + sz_list, st);
    if (err != cudaSuccess) {
        sc.base = nullptr;
        return cuda_fail(err, "cudaMallocAsync(scratch)");
    }
    char *p = (char *)sc.base;
    int32_t *hist = (int32_t *)p;
    int32_t *cursor = hist + (ncls + 1);
    uint32_t *counters = (uint32_t *)(cursor + (ncls + 1));  // 2 per class
    int32_t *order = (int32_t *)(p + sz_small);
    int32_t *list = sz_list ? (int32_t *)(p + sz_small + sz_order) : nullptr;
    int32_t *list_count = (int32_t *)(counters + 2 * ncls);  // 1 per class
    err = cudaMemsetAsync(p, 0, sz_small, st);
    if (err != cudaSuccess)
        return cuda_fail(err, "cudaMemsetAsync(scratch)");
    int kr = swg::launch_pair_classes(q_off, n_pairs, ct, hist, cursor, order, st, sms);
    if (kr)
        return cuda_fail(kr, "pair class kernels");
    // class sizes decide the launches: one small synchronous read
    int32_t h_hist[16] = {0};
    err = cudaMemcpyAsync(h_hist, hist, sizeof(int32_t) * (ncls + 1), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(st);
    if (err != cudaSuccess)
        return cuda_fail(err, "reading pair classes");
    if (h_hist[ncls] > 0)
        return fail(SW_ERR_RANGE, "%d pairs have a query longer than %d residues", h_hist[ncls], ct.q[ncls - 1]);

    a.q = q;
    a.q_off = q_off;
    a.r = r;
    a.r_off = r_off;
    a.n_pairs = n_pairs;
    a.A = alphabet;
    a.o = gap_open;
    a.e = gap_extend;
    a.scores = scores_out;
    a.one = 1;
    a.lazy_steps = lazy_steps;
    a.q_end = q_end;
    a.r_end = r_end;
    const int32_t thresh = flag_threshold(lane, gap_open, maxM);
    int64_t begin = 0;
    for (int k = 0; k < ncls; ++k) {
        const int64_t cnt = h_hist[k];
        if (cnt == 0)
            continue;
        const int32_t *cls = order + begin;
        a.counter = counters + 2 * k;
        const int lk = lane == SW_LANE_I32     ? swg::LK_I32
                       : lane == SW_LANE_I16X2 ? swg::LK_I16X2
                       : lane == SW_LANE_I8X4  ? swg::LK_I8X4
                                               : swg::LK_I16X2Q;
        a.flag_thresh = thresh;
        kr = ends ? swg::launch_pairs_ends(lk, tab[k].L, tab[k].S, a, cls, nullptr, cnt, sms, st)
                  : swg::launch_pairs(lk, tab[k].L, tab[k].S, lazy, a, cls, nullptr, cnt, sms, st);
        if (kr)
            return cuda_fail(kr, "pair kernel launch");
        if (lane != SW_LANE_I32) {
            int32_t *cl = list + begin;
            kr = swg::launch_flag_overflow_list(scores_out, cls, cnt, thresh, cl, list_count + k, st, sms);
            if (kr)
                return cuda_fail(kr, "overflow flag kernel");
            // int32 class covering the same query lengths
            int j = 0;
            while (j + 1 < kPairI32N && kPairI32[j].L * kPairI32[j].S < ct.q[k])
                ++j;
            a.counter = counters + 2 * k + 1;
            a.flag_thresh = INT32_MAX;
            kr = ends ? swg::launch_pairs_ends(swg::LK_I32, kPairI32[j].L, kPairI32[j].S, a, cl, list_count + k,
                                               cnt, sms, st)
                      : swg::launch_pairs(swg::LK_I32, kPairI32[j].L, kPairI32[j].S, false, a, cl, list_count + k,
                                          cnt, sms, st);
            if (kr)
                return cuda_fail(kr, "rescore kernel launch");
        }
        begin += cnt;
    }
    return SW_OK;
}

int sw_align_pairs(const uint8_t *q, const int64_t *q_off, const uint8_t *r, const int64_t *r_off,
                   int64_t n_pairs, const int8_t *subst_matrix, int32_t alphabet, int32_t gap_open,
                   int32_t gap_extend, int32_t lane_type, int32_t *scores_out, void *cuda_stream)
{
    return pairs_impl(q, q_off, r, r_off, n_pairs, subst_matrix, alphabet, gap_open, gap_extend, lane_type,
                      scores_out, cuda_stream, false, nullptr);
}

int sw_align_pairs_ends(const uint8_t *q, const int64_t *q_off, const uint8_t *r, const int64_t *r_off,
                        int64_t n_pairs, const int8_t *subst_matrix, int32_t alphabet, int32_t gap_open,
                        int32_t gap_extend, int32_t lane_type, int32_t *scores_out, int32_t *q_end_out,
                        int32_t *r_end_out, void *cuda_stream)
{
    if (n_pairs > 0 && (!q_end_out || !r_end_out))
        return fail(SW_ERR_INVALID, "q_end_out / r_end_out is NULL");
    return pairs_impl(q, q_off, r, r_off, n_pairs, subst_matrix, alphabet, gap_open, gap_extend, lane_type,
                      scores_out, cuda_stream, false, nullptr, n_pairs > 0 ? q_end_out : nullptr, r_end_out);
}

int sw_align_lazyf_pairs(const uint8_t *q, const int64_t *q_off, const uint8_t *r, const int64_t *r_off,
                         int64_t n_pairs, const int8_t *subst_matrix, int32_t alphabet, int32_t gap_open,
                         int32_t gap_extend, int32_t *scores_out, unsigned long long *lazy_steps,
                         void *cuda_stream)
{
    return pairs_impl(q, q_off, r, r_off, n_pairs, subst_matrix, alphabet, gap_open, gap_extend, SW_LANE_I32,
                      scores_out, cuda_stream, true, lazy_steps);
}

int sw_align_lazyf_pairs_lane(const uint8_t *q, const int64_t *q_off, const uint8_t *r, const int64_t *r_off,
                              int64_t n_pairs, const int8_t *subst_matrix, int32_t alphabet, int32_t gap_open,
                              int32_t gap_extend, int32_t lane_type, int32_t *scores_out,
                              unsigned long long *lazy_steps, void *cuda_stream)
{
    return pairs_impl(q, q_off, r, r_off, n_pairs, subst_matrix, alphabet, gap_open, gap_extend, lane_type,
                      scores_out, cuda_stream, true, lazy_steps);
}

int sw_stream_sync(void *cuda_stream, int64_t timeout_ms)
{
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t err = cudaStreamQuery(st);
        if (err == cudaSuccess)
            return SW_OK;
        if (err != cudaErrorNotReady)
            return cuda_fail(err, "cudaStreamQuery");
        const auto ms =
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= timeout_ms)
            return fail(SW_ERR_TIMEOUT, "stream still busy after %lld ms", (long long)timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int sw_mem_available(int64_t *bytes)
{
    if (!bytes)
        return fail(SW_ERR_INVALID, "bytes is NULL");
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    size_t free_b = 0, total_b = 0;
    if (err == cudaSuccess)
        err = cudaMemGetInfo(&free_b, &total_b);
    if (err != cudaSuccess)
        return cuda_fail(err, "cudaMemGetInfo");
    // the library's scratch comes from the device's default stream-ordered
    // pool, which keeps freed blocks: those are available to the next call
    uint64_t reserved = 0, used = 0;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    }
    *bytes = (int64_t)free_b + (int64_t)(reserved > used ? reserved - used : 0);
    return SW_OK;
}

int sw_probe_cell_rate(int32_t lane_type, int32_t iters, double *cells_per_second, void *cuda_stream)
{
    return sw_probe_cell_rate_pass(lane_type, 0, iters, cells_per_second, cuda_stream);
}

int sw_probe_cell_rate_pass(int32_t lane_type, int32_t corrected, int32_t iters, double *cells_per_second,
                            void *cuda_stream)
{
    if (!cells_per_second)
        return fail(SW_ERR_INVALID, "cells_per_second is NULL");
    if (lane_type < SW_LANE_I32 || lane_type > SW_LANE_I16X2Q)
        return fail(SW_ERR_INVALID, "lane_type must be I32, I16X2, I8X4 or I16X2Q");
    if (corrected < 0 || corrected > 2)
        return fail(SW_ERR_INVALID, "corrected must be 0, 1 or 2");
    if (corrected && lane_type == SW_LANE_I8X4)
        return fail(SW_ERR_INVALID, "the s8x4 lanes have no corrected pass");
    if (corrected == 2 && lane_type != SW_LANE_I16X2 && lane_type != SW_LANE_I16X2Q)
        return fail(SW_ERR_INVALID, "the always-corrected pass runs on s16x2 lanes only");
    if (lane_type == SW_LANE_I16X2Q)
        lane_type = SW_LANE_I16X2;  // the same cell sequence on the same lane type
    if (iters < 1)
        return fail(SW_ERR_INVALID, "iters must be >= 1");
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = num_sms_of(dev);
    double cells = 0;
    float ms = 0;
    const int op = lane_type - 1;
    int kr = swg::run_int_peak(op, corrected == 1, corrected == 2, sms * 8, 256, iters, &cells, &ms,
                               (cudaStream_t)cuda_stream);
    if (kr)
        return cuda_fail(kr, "cell-rate probe");
    *cells_per_second = ms > 0 ? cells / (ms * 1e-3) : 0.0;
    return SW_OK;
}

}  // extern "C"
