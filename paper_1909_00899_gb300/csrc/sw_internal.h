// Internal declarations shared by the host API (sw_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace swg {

enum LaneKind { LK_I32 = 1, LK_I16X2 = 2, LK_I8X4 = 3, LK_I16X2Q = 4 };

// One layout of the striped query: L lanes per alignment, S positions per
// lane (the paper's p and segLen), C query chunks of L*S positions each.
struct Plan {
    int L = 0, S = 0, C = 0, lane = 0;
};

// Parameters of one launch of the batch kernel (one query chunk).
// One piece of a long database sequence (a window of its columns), aligned
// as if it were a sequence of its own; the pieces of one sequence overlap by
// at least the number of columns a positive-scoring local alignment of the
// query can span, so the largest piece score is the sequence's score.
struct Piece {
    int64_t start;  // first residue (index into the concatenated database)
    int32_t seq;    // the sequence it belongs to
    int32_t len;    // columns
};
// In the batch kernels a work item's sequence id with this bit set is a
// piece of a long sequence (its score is combined by atomicMax); calls that
// split long sequences keep their ids below 2^30.
constexpr int PIECE_BIT = 1 << 30;

struct BatchArgs {
    const int8_t *prof;       // raw striped profile of this plan: [C][A][L][S] int8 (M values)
    int32_t A;                // alphabet size; profile row A is the inert "no residue" row
    int32_t qlen;
    int32_t chunk, nchunks;
    const uint8_t *db;
    const int64_t *off;       // db offsets, n+1
    const int32_t *order;     // sequence ids in processing order (may be null: identity)
    int64_t n_work;           // entries of order to process
    const int32_t *n_work_dev;  // if set, the number of entries is read here instead
    int32_t o, e;
    int2 *bnd;                // boundary rows between chunks: per sequence, index off[seq]+r
    int32_t *scores;          // per sequence
    uint32_t *counter;        // work counter, zero at launch
    unsigned long long *lazy_steps;  // optional statistics of the lazy-F loop
    uint32_t one;             // 1 (a run-time multiplier for FMA-pipe additions)
    int32_t flag_thresh;      // packed lanes: true score at which a cell is rescored
    int32_t *q_end;           // end cells (1-based query / reference position), ENDS kernels
    int32_t *r_end;
    int32_t min_m;            // smallest substitution score of the profile (the split
                              // kernels' shorter corrected pass needs min_m >= -o)
    // long sequences split into overlapping pieces (single-chunk scores
    // only; null otherwise): work items [0, *n_pieces) are pieces, whose
    // scores are combined by atomicMax, then the entries of order, skipping
    // the sequences whose split flag is set
    const Piece *pieces;
    const int32_t *n_pieces;
    const uint8_t *split;
};

// Parameters of the pair kernel (each pair has its own query).
struct PairArgs {
    const uint8_t *q;
    const int64_t *q_off;
    const uint8_t *r;
    const int64_t *r_off;
    int64_t n_pairs;
    const int32_t *order;       // optional pair ids to process (rescore list)
    const int32_t *n_work_dev;  // optional device count of order entries
    int32_t A, o, e;
    int8_t M[32 * 32];          // substitution matrix [query][reference]
    int32_t *scores;
    uint32_t *counter;
    uint32_t one;             // 1 (a run-time multiplier for FMA-pipe additions)
    int32_t flag_thresh;      // packed lanes: true score at which a cell is rescored
    unsigned long long *lazy_steps;  // optional statistics of the lazy-F loop
    int32_t min_m;            // smallest substitution score (shorter corrected pass: see sw_lanes.cuh)
    int32_t *q_end;           // end cells (1-based query / reference position), ENDS pair kernels
    int32_t *r_end;
};

// batch launchers (sw_k_i32.cu, sw_k_i16.cu, sw_k_i8.cu), declared in
// sw_api.cu; every launcher returns a cudaError_t value.
// pair launchers (sw_k_pairs.cu): one query-length class (L, S) per launch
// over list[0 .. n_hint), or list[0 .. *count_dev) when count_dev is set
// (*count_dev <= n_hint).
int launch_pairs(int lane, int L, int S, bool lazy, const PairArgs &a, const int32_t *list, const int32_t *count_dev,
                 int64_t n_hint, int num_sms, cudaStream_t st);
// the same with end cells (scan-F; lane LK_I16X2Q or LK_I32, sw_k_pairs_e.cu)
int launch_pairs_ends(int lane, int L, int S, const PairArgs &a, const int32_t *list, const int32_t *count_dev,
                      int64_t n_hint, int num_sms, cudaStream_t st);

// Query-length classes of the pair kernel: class k holds pairs with
// qlen <= q[k] (and > q[k-1]); class n holds longer queries.
struct ClassTable {
    int n;
    int q[8];
};
// hist[n + 1] and cursor[n + 1] zeroed; order grouped by class, ascending.
int launch_pair_classes(const int64_t *q_off, int64_t n_pairs, const ClassTable &t, int32_t *hist,
                        int32_t *cursor, int32_t *order, cudaStream_t st, int num_sms);
// flag list entries whose score reached thresh into out (count in *out_count)
int launch_flag_overflow_list(const int32_t *scores, const int32_t *list, int64_t n, int32_t thresh, int32_t *out,
                              int32_t *out_count, cudaStream_t st, int num_sms);

// aux kernels (sw_aux.cu)
int launch_profile_build(const uint8_t *d_query, int32_t qlen, const int8_t *d_M, int32_t A, const Plan &pl,
                         int8_t *d_prof, cudaStream_t st);
// Length-binned processing order, longest first: order[n] of sequence ids.
// scratch: 2*NBINS int32 of zeroed scratch (histogram, cursors).
constexpr int NBINS = 128;
int launch_length_order(const int64_t *off, int64_t n, int32_t *order, int32_t *bins, cudaStream_t st,
                        int num_sms);
// Sequences whose score reached thresh -> list (count in *count, zero at launch).
int launch_flag_overflow(const int32_t *scores, int64_t n, int32_t thresh, int32_t *list, int32_t *count,
                         cudaStream_t st, int num_sms);
// Long sequences (more than piece_len residues) -> overlapping pieces of
// piece_len columns every stride columns, at most cap pieces in all (a
// sequence that no longer fits stays whole); split[i] tells which, and a
// split sequence's score is zeroed for the pieces' atomicMax.
// *n_pieces zero at launch.
int launch_piece_plan(const int64_t *off, int64_t n, int32_t piece_len, int32_t stride, int32_t cap,
                      Piece *pieces, int32_t *n_pieces, uint8_t *split, int32_t *scores, cudaStream_t st,
                      int num_sms);

}  // namespace swg

// A built query profile (opaque in the public header).
struct sw_profile {
    int device = 0;
    int32_t qlen = 0, A = 0, lane = 0;
    swg::Plan plan;    // plan of the requested lane type
    swg::Plan plan32;  // int32 plan: lazy-F and the rescore of flagged alignments
    void *block = nullptr;          // one stream-ordered allocation for all parts
    cudaStream_t stream = nullptr;  // stream the profile was built on
    uint8_t *d_query = nullptr;
    int8_t *d_M = nullptr;
    int8_t *d_prof = nullptr;
    int8_t *d_prof32 = nullptr;
    int32_t maxM = 0, minM = 0;
};

// A device-resident database handle (opaque in the public header).
struct sw_db {
    int device = 0;
    const uint8_t *res = nullptr;
    const int64_t *off = nullptr;
    int64_t n = 0;
    int64_t total = 0;
    int32_t *order = nullptr;  // length-binned order, longest first (owned)
};

namespace swg {

// Host helpers of sw_api.cu shared with other host translation units.
int api_fail(int code, const char *msg);
int api_cuda_fail(int err, const char *what);
int api_num_sms(int dev);
bool api_lane_fits(int lane, const sw_profile *pf, int32_t o, int32_t e, const Plan &pl);
int32_t api_flag_threshold(int lane, int32_t o, int32_t maxM);
int api_check_align_args(const sw_profile *prof, const uint8_t *db, const int64_t *off, int64_t n_db, int32_t o,
                         int32_t e, int32_t *scores);
int api_launch_plan(const Plan &pl, bool lazy, const BatchArgs &a, int sms, cudaStream_t st);

// Cell-rate probe of the plain pass for the roofline: 'op' selects the
// lane type (0 int32, 1 s16x2, 2 s8x4); corrected: the shorter corrected
// pass; always: the always-corrected pass (s16x2 only); returns cells
// updated and ms.
int run_int_peak(int op, bool corrected, bool always, int blocks, int threads, int iters, double *cells, float *ms,
                 cudaStream_t st);

}  // namespace swg

namespace swg {

// One query of a batched multi-query launch (device table entry).
struct MultiQuery {
    const int8_t *prof;    // raw profile of its layout: [C][A][L*S] int8
    int32_t qlen;
    int32_t C;             // chunks of its layout
    int64_t row;           // its score row (the query's index in the batch)
};

// Parameters of one multi-query launch: every pair of queries[0 ..
// n_queries) x the first n_items entries of the length order (the phase
// kernel and the chunk walk pull them query by query, or chunk by chunk;
// the fused-chunk kernel in (query, tile of sequences) units).
struct MultiArgs {
    const MultiQuery *queries;
    int32_t n_queries;
    int32_t A, o, e, min_m;
    uint32_t one;
    const uint8_t *db;
    const int64_t *off;
    const int32_t *order;   // sequence ids by length, longest first
    int64_t n_items;        // entries of order covered
    int32_t skip_len;       // pairs with min(query length, sequence length) >= skip_len: the
                            // int32 launch's candidates (only they can overflow the packed lanes)
    int32_t flag_thresh;    // the int32 launch rescores candidates whose packed score reached it
    int32_t *scores;        // row-major [query][row_stride]
    int64_t row_stride;
    int32_t k_items;        // fused-chunk kernel: sequences per lane group per unit (a tile is k_items x groups per CTA)
    unsigned long long *counter;  // work counters, zero at launch: one per query (phase kernel), one per
                                  // (query, chunk) phase (chunk walk), one per launch (fused-chunk)
    uint32_t *bnd;          // per-group boundary-row slots (32-bit words), null when C == 1 throughout
    int64_t bnd_stride;     // words per group slot
    // the chunk-phase kernel: boundary rows of every database residue
    // (int2, indexed offsets[seq] + r), the last phase each sequence of the
    // order finished (-1 at launch), and a status word set when a bounded
    // wait gave up (0 at launch)
    int2 *rows;
    int32_t *done;
    int32_t *status;
    int32_t wait_limit;     // polls (about 256 ns each) before a wait gives up
    int32_t wait_skew;      // added to the awaited mark: 0, or past every phase (a test of the bound)
};

// multi-query launchers (sw_k_multi*.cu): split s16x2 layouts (virtual lanes
// x segment length; kind: the phase kernel of single-chunk queries, the
// (query, chunk) walk or the fused-chunk kernel of longer ones) and the int32
// layouts 32 x {8, 16, 32} of the pairs that could overflow the packed
// lanes; grid is fixed by the caller (its boundary slots are sized for it).
constexpr int MULTI_FUSED = 0, MULTI_PHASE = 1, MULTI_CHUNKS = 2;
int launch_multi_split(int VL, int S, int kind, const MultiArgs &a, int grid, cudaStream_t st);
int launch_multi_i32(int S, const MultiArgs &a, int grid, cudaStream_t st);
// CTAs per SM the launch runs with (0 for a layout without a kernel)
int multi_split_blocks_per_sm(int VL, int S, int kind, bool d0, int A);
int multi_i32_blocks_per_sm(int S, bool d0, int A);
// groups (one item each) per CTA of a layout of `lanes` virtual lanes (the
// int32 kernels' 32 lanes per alignment count as 64: one group per warp)
int multi_groups_per_cta(int lanes);

}  // namespace swg
