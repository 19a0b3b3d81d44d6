/*
 * sw_gb300.h — C ABI of the GB300 (sm_103a) score-only Smith-Waterman/Gotoh
 * library: striped query layout with the F dependency between segments
 * resolved by a max-plus prefix scan (arXiv:1909.00899, Alg. 6), plus the
 * lazy-F correction loop (Alg. 1) as the plain-method comparison.
 *
 * What is computed (Sec. I): for a query Q (length m) and each reference
 * sequence R (length n), the optimal local alignment score with affine gaps,
 *   E(q,r) = max(H(q,r-1) - o, E(q,r-1) - e)
 *   F(q,r) = max(H(q-1,r) - o, F(q-1,r) - e)
 *   H(q,r) = max(0, H(q-1,r-1) + M[Q_q][R_r], E(q,r), F(q,r))
 *   score  = max over q,r of H(q,r)   (0 when m == 0 or n == 0)
 * so a gap run of k residues costs o + (k-1)*e (Alg. 1 charges GapOpen for
 * the first residue and GapExtend for each further one).  M is indexed
 * [query residue][reference residue] (the query profile of Alg. 1 is built
 * from the query).  Scores are exact int32 whatever lane type computes them.
 *
 * Conventions for every call
 *  - Residues are codes 0..A-1 in uint8.  A code >= A (in a database
 *    sequence, or in a query of sw_align_pairs) is an unknown residue: it
 *    scores the smallest entry of the substitution matrix against anything,
 *    on every lane type.  sw_profile_build rejects query codes >= A.
 *  - "device" pointers are CUDA device memory on the current device, owned
 *    by the caller; "host" pointers are host memory owned by the caller and
 *    only read during the call.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Align
 *    calls are asynchronous on that stream: they return after enqueueing
 *    work; results are valid once the stream reaches that point.
 *  - Return value: SW_OK (0) or a negative SW_ERR_* code; sw_last_error()
 *    then returns a message (thread-local, valid until the next call on the
 *    same thread).  Invalid arguments are rejected before any CUDA call.
 *  - Library scratch (length-sorted work order, boundary rows of long
 *    queries, overflow lists) is allocated with cudaMallocAsync on the call's
 *    stream from the device's default memory pool and released on that
 *    stream; the library raises that pool's release threshold once per
 *    device so freed scratch stays cached between calls.
 */
#ifndef SW_GB300_H
#define SW_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SW_OK 0
#define SW_ERR_INVALID (-1)  /* bad argument (null pointer, range, shape)  */
#define SW_ERR_CUDA (-2)     /* a CUDA runtime call or a launch failed      */
#define SW_ERR_NOMEM (-3)    /* device or host allocation failed            */
#define SW_ERR_TIMEOUT (-4)  /* sw_stream_sync gave up waiting              */
#define SW_ERR_RANGE (-5)    /* matrix/gap values do not fit the lane type  */

/* lane types: how many cells one 32-bit register carries */
#define SW_LANE_AUTO 0   /* library picks lane type and layout per query
                            length (packed lanes + exact rescore)         */
#define SW_LANE_I32 1    /* one int32 cell per register                    */
#define SW_LANE_I16X2 2  /* two int16 cells per register, DPX s16x2 ops    */
#define SW_LANE_I8X4 3   /* four int8 cells per register, saturating SIMD  */
#define SW_LANE_I16X2Q 4 /* two int16 cells per register: the two halves of
                            one alignment's query (no byte permutes);
                            plans count virtual lanes, two per thread     */

typedef struct sw_profile sw_profile; /* opaque, owned by the library */

/*
 * sw_profile_build — striped query profile (Alg. 1/6 "vprofile": for each
 * residue c, the score M[Q_q][c] of every query position q, laid out so that
 * lane l of an alignment holds positions l*segLen .. l*segLen+segLen-1).
 *   query         host, qlen codes in 0..alphabet-1 (may be NULL if qlen 0)
 *   qlen          >= 0
 *   subst_matrix  host, alphabet*alphabet int8, row-major [query][reference]
 *   alphabet      1..32
 *   lane_type     SW_LANE_*; the layout (lanes per alignment, segment
 *                 length, query chunks) is chosen from qlen and lane_type
 *   cuda_stream   stream for the upload and the profile-build kernel
 *   out           receives the profile; free with sw_profile_free
 * Device memory for the profile is one stream-ordered allocation
 * (cudaMallocAsync on cuda_stream, current device); work on other streams
 * that uses the profile must be ordered after the build (an event, or a
 * synchronisation).  The host buffers are read before the call returns.
 * Errors: SW_ERR_INVALID (qlen < 0, alphabet out of range, null pointers,
 * query code >= alphabet), SW_ERR_NOMEM, SW_ERR_CUDA.
 */
int sw_profile_build(const uint8_t *query, int32_t qlen,
                     const int8_t *subst_matrix, int32_t alphabet,
                     int32_t lane_type, void *cuda_stream, sw_profile **out);

/*
 * sw_profile_build_ex — as sw_profile_build with an explicit layout: lanes
 * per alignment (the paper's p, a power of two up to 32) and seg_len query
 * positions per lane (segLen); both 0 selects the built-in table.  Only the
 * shapes the kernels are compiled for are accepted (SW_ERR_INVALID
 * otherwise): int32 {1x16, 1x32, 4x8, 4x32, 8x8, 8x16, 16x8, 16x16, 32x8,
 * 32x12, 32x16, 8x32, 16x32, 32x32} (1 lane: one thread per alignment, no
 * scan), s16x2 {8x8, 8x16, 16x8, 16x16, 32x8, 32x12, 32x16, 16x32,
 * 32x24, 32x32}, s8x4 {8x16, 16x16, 32x16}, split s16x2 (virtual lanes)
 * {2x16, 2x32, 16x8, 32x8, 32x12, 32x16, 32x20, 32x24, 32x32, 64x8, 64x16,
 * 64x20, 64x24, 64x28, 64x32} (2
 * virtual lanes: one thread per alignment).  Used by the autotuner.
 */
int sw_profile_build_ex(const uint8_t *query, int32_t qlen,
                        const int8_t *subst_matrix, int32_t alphabet,
                        int32_t lane_type, int32_t lanes, int32_t seg_len,
                        void *cuda_stream, sw_profile **out);

/* Releases a profile after waiting for the whole device to finish (safe
 * whatever stream used it).  NULL ok. */
int sw_profile_free(sw_profile *prof);

/* Releases a profile in stream order on cuda_stream, without waiting: every
 * use of the profile must already be ordered before this point of that
 * stream.  The handle is invalid on return.  NULL ok. */
int sw_profile_free_async(sw_profile *prof, void *cuda_stream);

/* Describes a profile's plan: lanes per alignment, segment length per lane,
 * query chunks, lane type actually used.  Any out pointer may be NULL. */
int sw_profile_plan(const sw_profile *prof, int32_t *lanes, int32_t *seg_len,
                    int32_t *chunks, int32_t *lane_type);

/* The plan sw_profile_build would choose for a query of qlen residues and
 * lane_type (SW_LANE_AUTO: the layout maximising the measured single-chunk
 * rate x useful positions / chunk positions, less 1.5 % per extra chunk),
 * without building anything: host only, no CUDA call.  Any out pointer may
 * be NULL.  SW_ERR_INVALID for qlen < 0 or an unknown lane type. */
int sw_plan_query(int32_t qlen, int32_t lane_type, int32_t *lanes,
                  int32_t *seg_len, int32_t *chunks, int32_t *lane_out);

/*
 * sw_align_batch — scores of one profiled query against n_db database
 * sequences with the scan-F method (Alg. 6): per reference column each lane
 * runs its segment with a zero F carry, the carry between segments is the
 * max-plus prefix scan over lanes with weight segLen*e per hop, and the
 * correction of H (and of E) is deferred into the next column's pass.
 * When the query fits one chunk of at most 1024 positions and
 * P = max(2*span, 2048) <= 8192, span = m + (m*maxM - 1)/e, database
 * sequences longer than P columns are aligned as windows of P columns
 * overlapping by span columns (every positive-scoring alignment spans at
 * most that many) and the largest window score is kept: the same scores,
 * without one warp walking the longest sequence alone (e >= 1 and maxM >= 1
 * only; scratch grows by 17 bytes per sequence).
 * Synchronisation: when the query spans more than one chunk (of the
 * profile's layout, or of the int32 layout a packed profile rescores with:
 * above 1024 positions), the chunk boundary rows are sized by the residue
 * count, so the call reads db_offsets[n_db] back and synchronises
 * cuda_stream first; such a call cannot be captured into a CUDA graph.
 * sw_db_create caches that count once: sw_align_db on the handle never
 * synchronises and can be captured for any query length.
 *   db_residues  device, concatenated residue codes
 *   db_offsets   device, int64[n_db + 1], offsets[0] = 0, non-decreasing;
 *                sequence k is db_residues[offsets[k] .. offsets[k+1])
 *   n_db         >= 0 (0 is a no-op)
 *   gap_open     o >= 1;  gap_extend  0 <= e <= o  (the carry of Alg. 4-6
 *                only extends gaps, exact only when e <= o)
 *   scores_out   device, int32[n_db]
 * Errors: SW_ERR_INVALID (null pointers, n_db < 0, gap costs out of range),
 * SW_ERR_RANGE (values too large even for int32 accumulation),
 * SW_ERR_NOMEM, SW_ERR_CUDA.  Offsets are not validated on the device.
 */
int sw_align_batch(const sw_profile *prof, const uint8_t *db_residues,
                   const int64_t *db_offsets, int64_t n_db, int32_t gap_open,
                   int32_t gap_extend, int32_t *scores_out, void *cuda_stream);

/*
 * sw_align_batch_ends — sw_align_batch plus where each best local alignment
 * ends (what a mate-rescue caller places reads by; Alg. 1's Max only keeps
 * the score): q_end_out[k], r_end_out[k] = the 1-based query and reference
 * positions of the first cell, in column order (smallest reference position,
 * then smallest query position), whose H equals the score; -1, -1 when the
 * score is 0.  Runs on the profile's layout when it is split s16x2 (the
 * automatic choice; about 1.2x the cost of the score-only call, flagged
 * alignments rescored with int32 end cells), on its int32 layout otherwise
 * (about 1.6x the cost of the int32 score-only call).
 * q_end_out, r_end_out: device int32[n_db].
 */
int sw_align_batch_ends(const sw_profile *prof, const uint8_t *db_residues,
                        const int64_t *db_offsets, int64_t n_db,
                        int32_t gap_open, int32_t gap_extend,
                        int32_t *scores_out, int32_t *q_end_out,
                        int32_t *r_end_out, void *cuda_stream);

/*
 * sw_align_lazyf_batch — same inputs, outputs and errors as sw_align_batch,
 * computed with the lazy-F correction loop of Alg. 1 (up to p rounds of
 * shift-and-correct per column, leaving as soon as no lane's carried F can
 * raise anything).  Runs on the profile's own layout: int32, two-alignment
 * s16x2 or split s16x2 (the latter with up to 2p rounds over its 2p virtual
 * lanes; flagged s16x2 alignments are rescored with the scan-F int32
 * kernel); an s8x4 profile runs on the int32 layout.  The comparison.
 */
int sw_align_lazyf_batch(const sw_profile *prof, const uint8_t *db_residues,
                         const int64_t *db_offsets, int64_t n_db,
                         int32_t gap_open, int32_t gap_extend,
                         int32_t *scores_out, void *cuda_stream);

/*
 * sw_db — a database kept resident on the device: the caller's residue and
 * offset buffers (which must outlive the handle) plus, computed once by
 * sw_db_create, the length-binned processing order (longest first) and the
 * total residue count.  sw_db_create synchronises cuda_stream once;
 * sw_align_db / sw_align_lazyf_db then read nothing back and allocate their
 * scratch with cudaMallocAsync on the call's stream, so they can be captured
 * into a CUDA graph, and calls on different streams may overlap.
 * Errors as sw_align_batch; sw_db_free releases the handle (NULL ok).
 */
typedef struct sw_db sw_db; /* opaque, owned by the library */
int sw_db_create(const uint8_t *db_residues, const int64_t *db_offsets,
                 int64_t n_db, void *cuda_stream, sw_db **out);
int sw_db_free(sw_db *db);
int sw_align_db(const sw_profile *prof, const sw_db *db, int32_t gap_open,
                int32_t gap_extend, int32_t *scores_out, void *cuda_stream);
int sw_align_lazyf_db(const sw_profile *prof, const sw_db *db,
                      int32_t gap_open, int32_t gap_extend,
                      int32_t *scores_out, void *cuda_stream);
/* sw_align_db_ends — sw_align_batch_ends against a resident database (same
 * outputs: q_end_out, r_end_out device int32[n], -1 where the score is 0). */
int sw_align_db_ends(const sw_profile *prof, const sw_db *db, int32_t gap_open,
                     int32_t gap_extend, int32_t *scores_out, int32_t *q_end_out,
                     int32_t *r_end_out, void *cuda_stream);

/*
 * sw_align_pairs — n_pairs independent alignments, pair k aligning query
 * q[q_off[k] .. q_off[k+1]) against reference r[r_off[k] .. r_off[k+1])
 * with the scan-F method (read-vs-window batches; each pair's profile is
 * built inside the kernel from its own query).
 *   q, r            device residue codes;  q_off, r_off  device int64[n+1]
 *   subst_matrix    host, alphabet*alphabet int8 [query][reference]
 *                   (copied into the launch parameters)
 *   lane_type       SW_LANE_* (SW_LANE_I16X2Q: one pair per group, the two
 *                   query halves in the two halves of each register);
 *                   packed types flag pairs whose score may have left the
 *                   lane range and rescore them in int32
 *   scores_out      device int32[n_pairs]
 * Query lengths up to 512 per pair (SW_ERR_RANGE otherwise).  Pairs are
 * sorted into query-length classes on the device; the class sizes are read
 * back once (a synchronous 64-byte copy), so this call synchronises
 * cuda_stream once and cannot be captured into a CUDA graph.  Errors as
 * sw_align_batch.
 */
int sw_align_pairs(const uint8_t *q, const int64_t *q_off, const uint8_t *r,
                   const int64_t *r_off, int64_t n_pairs,
                   const int8_t *subst_matrix, int32_t alphabet,
                   int32_t gap_open, int32_t gap_extend, int32_t lane_type,
                   int32_t *scores_out, void *cuda_stream);

/*
 * sw_align_pairs_ends — sw_align_pairs plus where each pair's best local
 * alignment ends, as sw_align_batch_ends defines it: q_end_out[k],
 * r_end_out[k] = the 1-based query and reference positions of the first
 * cell in column order (smallest reference position, then smallest query
 * position) whose H equals the score; -1, -1 when the score is 0.  This is
 * what a mate-rescue caller places a read by.  Split s16x2 kernels for
 * SW_LANE_AUTO and SW_LANE_I16X2Q (flagged pairs rescored with int32 end
 * cells), int32 kernels for the other lane types.  q_end_out, r_end_out:
 * device int32[n_pairs].  Errors and synchronisation as sw_align_pairs.
 */
int sw_align_pairs_ends(const uint8_t *q, const int64_t *q_off, const uint8_t *r,
                        const int64_t *r_off, int64_t n_pairs,
                        const int8_t *subst_matrix, int32_t alphabet,
                        int32_t gap_open, int32_t gap_extend, int32_t lane_type,
                        int32_t *scores_out, int32_t *q_end_out,
                        int32_t *r_end_out, void *cuda_stream);

/*
 * sw_align_lazyf_pairs — as sw_align_pairs with the lazy-F correction loop
 * of Alg. 1 (int32 lanes), the plain-method comparison for read-vs-window
 * batches.  lazy_steps: optional device counter (caller zeroes it) to which
 * every warp adds the j-steps its correction loop ran; divided by the
 * main-pass j-steps (cells / 32) it is the paper's corrective factor C
 * (Sec. I, cost O((1+C) n/p)).  NULL: not counted.
 */
int sw_align_lazyf_pairs(const uint8_t *q, const int64_t *q_off,
                         const uint8_t *r, const int64_t *r_off,
                         int64_t n_pairs, const int8_t *subst_matrix,
                         int32_t alphabet, int32_t gap_open,
                         int32_t gap_extend, int32_t *scores_out,
                         unsigned long long *lazy_steps, void *cuda_stream);

/* sw_align_lazyf_pairs on a chosen layout: SW_LANE_I16X2Q runs the
 * correction loop on the split s16x2 pair kernel (the layout of the
 * automatic sw_align_pairs; flagged pairs are rescored with the scan-F
 * int32 kernel), any other lane type on int32 lanes.  lazy_steps as above,
 * counted per warp (a split warp step covers twice the cells of an int32
 * one). */
int sw_align_lazyf_pairs_lane(const uint8_t *q, const int64_t *q_off,
                              const uint8_t *r, const int64_t *r_off,
                              int64_t n_pairs, const int8_t *subst_matrix,
                              int32_t alphabet, int32_t gap_open,
                              int32_t gap_extend, int32_t lane_type,
                              int32_t *scores_out,
                              unsigned long long *lazy_steps, void *cuda_stream);

/* sw_align_lazyf_db with the same optional lazy-F step counter. */
int sw_align_lazyf_db_stats(const sw_profile *prof, const sw_db *db,
                            int32_t gap_open, int32_t gap_extend,
                            int32_t *scores_out,
                            unsigned long long *lazy_steps, void *cuda_stream);

/*
 * sw_multi — many profiled queries against one resident database in one
 * persistent launch per layout (the ragged batch; every (query, sequence)
 * alignment is independent, Sec. III).  sw_multi_create groups the queries
 * by their layout, reads the database's offsets back once to order its
 * sequences exactly by length, uploads the tables and that order and sizes
 * the per-group boundary slots (it synchronises cuda_stream and allocates
 * about 4 bytes per sequence, plus 8 bytes per residue when some query has
 * several chunks, or the slots of the fused-chunk tiles); sw_align_multi
 * then issues a few memsets (work counters, the walk's marks) and one
 * launch per layout (two when a layout holds both one- and
 * several-chunk queries), plus one int32 launch per int32 layout when some
 * pairs could overflow the packed lanes, with no host
 * synchronisation: it can be captured into a CUDA graph.
 *  - Queries of one chunk (per layout, one launch): every CTA walks the
 *    queries in order, stages each one's profile once and pulls its
 *    sequences, longest first, from the query's own counter, as the
 *    per-query kernel does.
 *  - Queries of several chunks (per layout, one launch): every CTA walks
 *    the (query, chunk) phases in order, staging each chunk's profile once
 *    and pulling the phase's sequences from its own counter, with one
 *    chunk boundary row per database residue (8 bytes each, allocated by
 *    sw_multi_create) reused by every query; a sequence is aligned in a
 *    phase only after the previous phase finished it (a per-sequence mark;
 *    the wait is bounded, see sw_multi_status).
 *  - items_per_group (1..64; 0: the phase walk above) asks instead for
 *    the fused-chunk kernel on queries of several chunks: units of (query,
 *    tile of that many sequences per lane group), each running all chunks
 *    of its query inside one CTA with every group's boundary row in its
 *    own slot of max_len columns (no residue-sized rows).
 *  - Overflow: the packed launches score every pair; only pairs with
 *    min(m, n) * max(M) >= the s16x2 rescore threshold can overflow, and
 *    the int32 launch walks those and rescores the ones whose packed score
 *    reached the threshold (none, on random protein data).
 *  - profiles: host array of n_queries profiles, all built with the same
 *    substitution matrix on SW_LANE_I16X2Q (or SW_LANE_AUTO, which chooses
 *    it) with layouts of 16 or more virtual lanes; they and the database
 *    handle must outlive the batch handle (SW_ERR_INVALID otherwise).
 *  - scores_out: device int32, row-major [n_queries][row_stride],
 *    row_stride >= the database's sequence count; row q holds query q's
 *    scores in the database's order.
 *  - gap_open <= 127 and the packed lanes' range check of sw_align_batch
 *    (SW_ERR_RANGE otherwise: align such queries one by one).
 *  - Calls on one handle share its counters and slots: do not overlap them.
 */
typedef struct sw_multi sw_multi; /* opaque, owned by the library */
int sw_multi_create(const sw_profile *const *profiles, int32_t n_queries,
                    const sw_db *db, int32_t items_per_group,
                    void *cuda_stream, sw_multi **out);
int sw_align_multi(const sw_multi *batch, int32_t gap_open, int32_t gap_extend,
                   int32_t *scores_out, int64_t row_stride, void *cuda_stream);
int sw_multi_free(sw_multi *batch);
/* The batch handle's status word, then cleared: 0, or 1 when a bounded
 * wait of the (query, chunk) phase walk gave up (about a second) since the
 * last read, in which case some scores of those calls may be wrong.  Once
 * the word is set, later waits give up at their first poll until it is
 * read, so a launch that lost a mark still ends.  Synchronises cuda_stream. */
int sw_multi_status(const sw_multi *batch, int32_t *status_out, void *cuda_stream);
/* The bound of the phase walk's waits for the handle's later calls:
 * max_polls polls of about 256 ns (0: the default, 2^22, about a second).
 * unreachable != 0 is for testing the bound: every wait then awaits a mark
 * no phase writes, runs out and sets the status word; the scores of such
 * calls are undefined (but every access stays inside the handle's buffers
 * and the caller's score matrix).  SW_ERR_INVALID for a NULL handle or
 * max_polls < 0.  Host only, no CUDA call. */
int sw_multi_set_wait(sw_multi *batch, int32_t max_polls, int32_t unreachable);

/*
 * sw_align_batch_noalloc — sw_align_batch (same arguments, results and
 * errors) for callers that cannot let a library allocate device memory, for
 * example an application whose own allocator has reserved the device's
 * memory, or a host framework that forbids its plug-ins to allocate.  This
 * call allocates nothing: its scratch (work order, counters, overflow list,
 * chunk boundary rows) lives in one fixed device array of
 * SW_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  The paper has no counterpart; it is a deployment
 * variant of the batch path.
 *  - The profile still comes from sw_profile_build (which allocates), so
 *    build profiles up front.
 *  - A call whose scratch would exceed the array (about 8 bytes per
 *    sequence, plus 8 bytes per residue for queries longer than one chunk)
 *    returns SW_ERR_RANGE before launching anything.
 *  - Every call shares the one array: calls whose work overlaps on the GPU
 *    (other streams, other host threads) race; serialise them.  Each call
 *    clears the counters it needs on its stream.
 *  - The first call on a device looks the array's address up
 *    (cudaGetSymbolAddress) with that device current; make it before any
 *    stream capture.  The address is kept for the process: after
 *    cudaDeviceReset (or a release of the device's primary context) the
 *    module, and with it the array, moves, so the call must not be used on
 *    that device again.
 *  - A query longer than one chunk synchronises cuda_stream on every call
 *    (as sw_align_batch does: the boundary rows are sized by reading
 *    db_offsets[n_db] back), so such calls can never be captured.
 *  - Long database sequences are not split into overlapping windows (the
 *    window plan would need scratch per sequence), so a short query against
 *    a few very long sequences can take longer than with sw_align_batch:
 *    one warp walks each of them whole.  Scores are the same.
 */
#define SW_NOALLOC_SCRATCH_BYTES (32u << 20)
int sw_align_batch_noalloc(const sw_profile *prof, const uint8_t *db_residues,
                           const int64_t *db_offsets, int64_t n_db,
                           int32_t gap_open, int32_t gap_extend,
                           int32_t *scores_out, void *cuda_stream);

/* Waits for cuda_stream with a bound: SW_OK when the stream is idle,
 * SW_ERR_TIMEOUT after timeout_ms milliseconds (the work keeps running and
 * the context stays usable), SW_ERR_CUDA if the stream reported an error. */
int sw_stream_sync(void *cuda_stream, int64_t timeout_ms);

/* Message for the last failing call on this thread ("" if none). */
const char *sw_last_error(void);

/*
 * sw_probe_cell_rate — measures the ALU ceiling of the cell update: every
 * thread of a full-device grid updates independent cells with exactly the
 * per-cell instruction sequence of the scan-F pass (no loads, no
 * shuffles, no scan).  Writes cells per second (host double) for the lane
 * type (SW_LANE_I32, _I16X2, _I8X4, or _I16X2Q which runs the s16x2
 * sequence).  Synchronises cuda_stream.  Used as
 * the measured denominator of the integer roofline.
 */
int sw_probe_cell_rate(int32_t lane_type, int32_t iters, double *cells_per_second,
                       void *cuda_stream);

/*
 * sw_probe_cell_rate_pass — as sw_probe_cell_rate, for one pass of the
 * scan-F column loop: corrected = 0 is the plain pass above; corrected = 1
 * is the shorter corrected pass the kernels run in columns that receive a
 * carry when every substitution score is >= -gap_open (the deferred
 * correction of Alg. 6: the diagonal and E raised by the carry, decaying by
 * gap_extend per position); corrected = 2 (SW_LANE_I16X2 / _I16X2Q only)
 * is the always-corrected pass of the long-query split kernels (no carry
 * vote, the zero floor of H taken on the corrected diagonal).
 * SW_LANE_I8X4 has no corrected pass (SW_ERR_INVALID), as has any other
 * value of corrected.
 */
int sw_probe_cell_rate_pass(int32_t lane_type, int32_t corrected, int32_t iters,
                            double *cells_per_second, void *cuda_stream);

/*
 * sw_mem_available — device memory a new call could use now on the current
 * device: the free memory (cudaMemGetInfo) plus the blocks the device's
 * default stream-ordered pool holds unused (the library's scratch and
 * profiles come from that pool, which keeps freed blocks).  Host query, no
 * stream work; the serving loop admits requests against it.
 */
int sw_mem_available(int64_t *bytes);

/* Library version, e.g. "0.1.0". */
const char *sw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SW_GB300_H */
