// sw_multi_create / sw_align_multi / sw_multi_free: many profiled queries
// against one resident database in one persistent launch per layout (the
// kernels are in sw_multi.cuh).  Creation groups the queries by layout,
// reads the database's offsets back once to order its sequences exactly by
// length (a unit's groups then finish together at the CTA's barriers),
// uploads the tables and that order, and sizes the per-group boundary
// slots; a call is then a memset and a few launches with no host
// synchronisation, so it can be captured in a CUDA graph.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "sw_gb300.h"
#include "sw_internal.h"

namespace {

struct MultiBin {
    int VL = 0, S = 0;   // split layout: virtual lanes x positions
    bool phase = false;  // single-chunk queries (the phase kernel), else several chunks
    int kind = 0;        // MULTI_PHASE, MULTI_CHUNKS or MULTI_FUSED
    int nq = 0;          // queries of the bin
    int64_t chunks = 0;  // chunks of all its queries
    int64_t cnt = 0;     // first of its counters (phase: one per query; chunks: one per chunk)
    int64_t tbl = 0;     // first entry in the device table
    int maxC = 0;        // most chunks of a query of the bin
    int grid[2] = {0, 0};  // CTAs of the general [0] / D0 [1] kernel
};

struct MultiI32 {
    int S = 0;                      // int32 layout 32 x S
    int nq = 0;
    int64_t tbl = 0;
    std::vector<int32_t> qlen_desc;  // its queries' lengths, longest first (the table's order)
    int maxC = 0;
    int grid[2] = {0, 0};
};

}  // namespace

// sequences per lane group per unit when the caller leaves it to the library
// (the rate on GB300 rose from 1 to 4; the autotuner can pick per batch)
constexpr int32_t kDefaultItems = 4;
// polls of about 256 ns before a wait of the chunk walk gives up (a second)
constexpr int32_t kDefaultWaitPolls = 1 << 22;

struct sw_multi {
    int device = 0;
    int32_t k_items = kDefaultItems;
    int32_t nq = 0, A = 0, maxM = 0, minM = 0;
    const uint8_t *res = nullptr;
    const int64_t *off = nullptr;
    const int32_t *order = nullptr;
    int64_t n = 0;
    int64_t total = 0;   // residues of the database
    int64_t max_len = 0;
    std::vector<int64_t> len_desc;  // sequence lengths in the order's order (longest first)
    std::vector<MultiBin> bins;
    MultiI32 i32[3];  // S = 8, 16, 32
    std::vector<int32_t> empty_q;  // queries of length 0 (their rows are zeroed)
    int64_t n_counters = 0;        // work counters of one call
    int32_t qlen_no_i32 = 0;       // longest query without a 32-lane int32 layout
    void *block = nullptr;
    swg::MultiQuery *d_tables = nullptr;
    unsigned long long *d_counters = nullptr;
    uint32_t *d_bnd = nullptr;
    uint32_t *d_bnd32 = nullptr;
    int64_t bnd_stride = 0, bnd32_stride = 0;
    int2 *d_rows = nullptr;       // chunk-phase boundary rows (one per residue)
    int32_t *d_done = nullptr;    // last phase each sequence of the order finished
    int32_t *d_status = nullptr;  // set by a bounded wait that gave up
    int32_t wait_limit = kDefaultWaitPolls;
    int32_t wait_skew = 0;
};

extern "C" {

int sw_multi_create(const sw_profile *const *profiles, int32_t n_queries, const sw_db *db, int32_t items_per_group,
                    void *cuda_stream, sw_multi **out)
{
    using namespace swg;
    if (!out)
        return api_fail(SW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!db)
        return api_fail(SW_ERR_INVALID, "db is NULL");
    if (n_queries < 0 || (n_queries > 0 && !profiles))
        return api_fail(SW_ERR_INVALID, "n_queries < 0 or profiles is NULL");
    if (items_per_group < 0 || items_per_group > 64)
        return api_fail(SW_ERR_INVALID, "items_per_group must be in 0..64 (0: the default)");
    int dev = 0;
    cudaGetDevice(&dev);
    if (db->device != dev)
        return api_fail(SW_ERR_INVALID, "database handle built on another device than the current one");
    for (int32_t q = 0; q < n_queries; ++q) {
        const sw_profile *p = profiles[q];
        if (!p)
            return api_fail(SW_ERR_INVALID, "a profile is NULL");
        if (p->device != dev)
            return api_fail(SW_ERR_INVALID, "a profile was built on another device than the current one");
        if (p->lane != SW_LANE_I16X2Q)
            return api_fail(SW_ERR_INVALID,
                            "the batched launch runs split s16x2 profiles (SW_LANE_I16X2Q, the automatic choice)");
        if (p->qlen > 0 && p->plan.L < 16)
            return api_fail(SW_ERR_INVALID, "the batched launch needs layouts of 16 or more virtual lanes");
        const sw_profile *p0 = profiles[0];
        if (p->A != p0->A || p->maxM != p0->maxM || p->minM != p0->minM)
            return api_fail(SW_ERR_INVALID, "profiles of one batch must share the substitution matrix");
        if ((int64_t)p->qlen * std::max(p->maxM, 0) >= (1LL << 24))
            return api_fail(SW_ERR_RANGE, "query length x largest score exceeds the int32 working range");
    }
    sw_multi *m = new sw_multi();
    m->device = dev;
    m->nq = n_queries;
    m->res = db->res;
    m->off = db->off;
    m->n = db->n;
    m->k_items = items_per_group ? items_per_group : kDefaultItems;
    if (n_queries > 0) {
        m->A = profiles[0]->A;
        m->maxM = profiles[0]->maxM;
        m->minM = profiles[0]->minM;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int sms = api_num_sms(dev);

    // layout bins of the packed launch, and the int32 sets (32-lane int32
    // layouts) of the pairs that could overflow it
    std::vector<MultiQuery> table;
    for (int32_t q = 0; q < n_queries; ++q) {
        const sw_profile *p = profiles[q];
        if (p->qlen == 0) {
            m->empty_q.push_back(q);
            continue;
        }
        if (p->plan32.L != 32)
            m->qlen_no_i32 = std::max(m->qlen_no_i32, p->qlen);
        MultiBin *b = nullptr;
        const bool phase = p->plan.C == 1;
        for (auto &x : m->bins)
            if (x.VL == p->plan.L && x.S == p->plan.S && x.phase == phase)
                b = &x;
        if (!b) {
            m->bins.push_back(MultiBin());
            b = &m->bins.back();
            b->VL = p->plan.L;
            b->S = p->plan.S;
            b->phase = phase;
        }
        b->nq++;
        b->chunks += p->plan.C;
        b->maxC = std::max(b->maxC, p->plan.C);
    }
    int64_t pos = 0;
    for (auto &b : m->bins) {
        // several chunks: the (query, chunk) phase walk, or the fused-chunk
        // tiles when the caller asked for a tile shape
        b.kind = b.phase ? MULTI_PHASE : items_per_group ? MULTI_FUSED : MULTI_CHUNKS;
        b.tbl = pos;
        pos += b.nq;
        b.cnt = m->n_counters;
        m->n_counters += b.kind == MULTI_PHASE ? b.nq : b.kind == MULTI_CHUNKS ? b.chunks : 1;
    }
    m->n_counters += 3;  // the int32 launches
    table.resize((size_t)pos);
    std::vector<int64_t> fill(m->bins.size(), 0);
    for (int32_t q = 0; q < n_queries; ++q) {
        const sw_profile *p = profiles[q];
        if (p->qlen == 0)
            continue;
        for (size_t k = 0; k < m->bins.size(); ++k) {
            MultiBin &b = m->bins[k];
            if (b.VL == p->plan.L && b.S == p->plan.S && b.phase == (p->plan.C == 1)) {
                MultiQuery &e = table[(size_t)(b.tbl + fill[k]++)];
                e.prof = p->d_prof;
                e.qlen = p->qlen;
                e.C = p->plan.C;
                e.row = q;  // times the row stride at call time: stored as the query index
                break;
            }
        }
    }
    const int i32S[3] = {8, 16, 32};
    for (int k = 0; k < 3; ++k) {
        MultiI32 &s = m->i32[k];
        s.S = i32S[k];
        std::vector<std::pair<int32_t, int32_t>> qs;  // (qlen, query index)
        for (int32_t q = 0; q < n_queries; ++q) {
            const sw_profile *p = profiles[q];
            if (p->qlen > 0 && p->plan32.L == 32 && p->plan32.S == s.S)
                qs.push_back({p->qlen, q});
        }
        std::sort(qs.begin(), qs.end(), [](auto &a, auto &b) { return a.first > b.first || (a.first == b.first && a.second < b.second); });
        s.nq = (int)qs.size();
        s.tbl = (int64_t)table.size();
        for (auto &x : qs) {
            const sw_profile *p = profiles[x.second];
            MultiQuery e;
            e.prof = p->d_prof32;
            e.qlen = p->qlen;
            e.C = p->plan32.C;
            e.row = x.second;
            table.push_back(e);
            s.qlen_desc.push_back(x.first);
            s.maxC = std::max(s.maxC, p->plan32.C);
        }
    }

    // the database's order, exactly by length (longest first, then by id):
    // consecutive entries, a unit's tile, have the same work
    std::vector<int32_t> order;
    cudaError_t err = cudaSuccess;
    if (m->n > 0) {
        std::vector<int64_t> off((size_t)m->n + 1);
        err = cudaMemcpyAsync(off.data(), m->off, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess)
            err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) {
            delete m;
            return api_cuda_fail((int)err, "sw_multi_create (reading db_offsets)");
        }
        order.resize((size_t)m->n);
        for (int64_t i = 0; i < m->n; ++i)
            order[(size_t)i] = (int32_t)i;
        std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            const int64_t la = off[(size_t)a + 1] - off[(size_t)a], lb = off[(size_t)b + 1] - off[(size_t)b];
            return la > lb || (la == lb && a < b);
        });
        m->len_desc.resize((size_t)m->n);
        for (int64_t i = 0; i < m->n; ++i) {
            const int32_t k = order[(size_t)i];
            m->len_desc[(size_t)i] = off[(size_t)k + 1] - off[(size_t)k];
        }
        m->max_len = m->len_desc[0];
        m->total = off[(size_t)m->n];
        if (m->max_len < 0 || m->len_desc.back() < 0) {
            delete m;
            return api_fail(SW_ERR_INVALID, "db_offsets must be non-decreasing");
        }
    }

    // grids (both passes) and boundary slots: one slot of max_len words per
    // resident group, for layouts whose queries have more than one chunk
    int64_t bnd_words = 0, bnd32_words = 0;
    for (auto &b : m->bins) {
        for (int d0 = 0; d0 < 2; ++d0) {
            const int per_sm = multi_split_blocks_per_sm(b.VL, b.S, b.kind, d0 == 1, m->A);
            if (per_sm <= 0) {
                delete m;
                return api_fail(SW_ERR_INVALID, "no batched kernel for a profile's layout");
            }
            b.grid[d0] = sms * per_sm;
            if (b.kind == MULTI_FUSED && b.maxC > 1)  // int2 per column
                bnd_words = std::max(bnd_words, (int64_t)b.grid[d0] * multi_groups_per_cta(b.VL) * m->max_len * 2);
        }
    }
    for (auto &s : m->i32) {
        if (!s.nq)
            continue;
        for (int d0 = 0; d0 < 2; ++d0) {
            const int per_sm = multi_i32_blocks_per_sm(s.S, d0 == 1, m->A);
            if (per_sm <= 0) {
                delete m;
                return api_fail(SW_ERR_INVALID, "no batched int32 kernel");
            }
            s.grid[d0] = sms * per_sm;
            if (s.maxC > 1)  // int2 per column
                bnd32_words = std::max(bnd32_words, (int64_t)s.grid[d0] * multi_groups_per_cta(64) * m->max_len * 2);
        }
    }
    m->bnd_stride = m->max_len * 2;
    m->bnd32_stride = m->max_len * 2;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t sz_tab = up(sizeof(MultiQuery) * std::max<size_t>(table.size(), 1));
    const size_t sz_cnt = up(sizeof(unsigned long long) * (size_t)m->n_counters);
    const size_t sz_bnd = up(sizeof(uint32_t) * (size_t)bnd_words);
    const size_t sz_bnd32 = up(sizeof(uint32_t) * (size_t)bnd32_words);
    const size_t sz_order = up(sizeof(int32_t) * (size_t)std::max<int64_t>(m->n, 1));
    bool chunk_walk = false;
    for (const auto &b : m->bins)
        chunk_walk |= b.kind == MULTI_CHUNKS;
    // the chunk-phase walk: boundary rows of every residue and a mark per sequence
    const size_t sz_rows = chunk_walk ? up(sizeof(int2) * (size_t)m->total + 16) : 0;
    const size_t sz_done = chunk_walk ? up(sizeof(int32_t) * (size_t)m->n) : 0;
    const size_t sz_status = up(sizeof(int32_t));
    err = cudaMalloc(&m->block, sz_tab + sz_cnt + sz_bnd + sz_bnd32 + sz_order + sz_rows + sz_done + sz_status);
    if (err != cudaSuccess) {
        m->block = nullptr;
        delete m;
        return api_cuda_fail((int)err, "sw_multi_create allocation");
    }
    char *base = (char *)m->block;
    m->d_tables = (MultiQuery *)base;
    m->d_counters = (unsigned long long *)(base + sz_tab);
    m->d_bnd = bnd_words ? (uint32_t *)(base + sz_tab + sz_cnt) : nullptr;
    m->d_bnd32 = bnd32_words ? (uint32_t *)(base + sz_tab + sz_cnt + sz_bnd) : nullptr;
    int32_t *d_order = (int32_t *)(base + sz_tab + sz_cnt + sz_bnd + sz_bnd32);
    m->order = d_order;
    char *tail = base + sz_tab + sz_cnt + sz_bnd + sz_bnd32 + sz_order;
    m->d_rows = chunk_walk ? (int2 *)tail : nullptr;
    m->d_done = chunk_walk ? (int32_t *)(tail + sz_rows) : nullptr;
    m->d_status = (int32_t *)(tail + sz_rows + sz_done);
    err = cudaMemsetAsync(m->d_status, 0, sizeof(int32_t), st);
    if (err == cudaSuccess && !table.empty())
        err = cudaMemcpyAsync(m->d_tables, table.data(), sizeof(MultiQuery) * table.size(), cudaMemcpyHostToDevice,
                              st);
    if (err == cudaSuccess && m->n > 0)
        err = cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(st);  // the host copies go out of scope
    if (err != cudaSuccess) {
        sw_multi_free(m);
        return api_cuda_fail((int)err, "sw_multi_create upload");
    }
    *out = m;
    return SW_OK;
}

int sw_multi_free(sw_multi *m)
{
    if (!m)
        return SW_OK;
    cudaError_t err = cudaSuccess;
    if (m->block) {
        err = cudaDeviceSynchronize();  // a launch may still read the tables
        cudaFree(m->block);
    }
    delete m;
    return err == cudaSuccess ? SW_OK : swg::api_cuda_fail((int)err, "sw_multi_free");
}

int sw_multi_status(const sw_multi *m, int32_t *status_out, void *cuda_stream)
{
    if (!m || !status_out)
        return swg::api_fail(SW_ERR_INVALID, "batch handle or status_out is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int32_t v = 0;
    cudaError_t err = cudaMemcpyAsync(&v, m->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(m->d_status, 0, sizeof(int32_t), st);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(st);
    if (err != cudaSuccess)
        return swg::api_cuda_fail((int)err, "sw_multi_status");
    *status_out = v;
    return SW_OK;
}

int sw_multi_set_wait(sw_multi *m, int32_t max_polls, int32_t unreachable)
{
    if (!m)
        return swg::api_fail(SW_ERR_INVALID, "batch handle is NULL");
    if (max_polls < 0)
        return swg::api_fail(SW_ERR_INVALID, "max_polls must be >= 0");
    m->wait_limit = max_polls ? max_polls : kDefaultWaitPolls;
    // past every phase number a walk reaches (phases < 2^30 by the chunk and
    // query counts the handle accepts)
    m->wait_skew = unreachable ? (1 << 30) : 0;
    return SW_OK;
}

int sw_align_multi(const sw_multi *m, int32_t gap_open, int32_t gap_extend, int32_t *scores_out, int64_t row_stride,
                   void *cuda_stream)
{
    using namespace swg;
    if (!m)
        return api_fail(SW_ERR_INVALID, "batch handle is NULL");
    if (gap_open < 1)
        return api_fail(SW_ERR_INVALID, "gap_open must be >= 1");
    if (gap_extend < 0 || gap_extend > gap_open)
        return api_fail(SW_ERR_INVALID, "gap_extend must satisfy 0 <= e <= gap_open");
    if (gap_open > 127)
        return api_fail(SW_ERR_RANGE, "the batched launch runs packed lanes: gap_open must be <= 127");
    if (m->nq == 0 || m->n == 0)
        return SW_OK;
    if (!scores_out)
        return api_fail(SW_ERR_INVALID, "scores_out is NULL");
    if (row_stride < m->n)
        return api_fail(SW_ERR_INVALID, "row_stride is smaller than the number of database sequences");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != m->device)
        return api_fail(SW_ERR_INVALID, "batch handle built on another device than the current one");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    sw_profile shape;  // the matrix range is all lane_fits reads
    shape.maxM = m->maxM;
    shape.minM = m->minM;
    for (const auto &b : m->bins) {
        Plan pl;
        pl.L = b.VL;
        pl.S = b.S;
        if (!api_lane_fits(SW_LANE_I16X2Q, &shape, gap_open, gap_extend, pl))
            return api_fail(SW_ERR_RANGE, "gap costs too large for the packed lanes of the batched launch; "
                                          "align these queries one by one");
    }
    // only pairs with min(m, n) >= skip_len can reach the packed lanes'
    // rescore threshold (score <= max(M) * min(m, n)): the int32 launch
    // walks them, the prefix of the length order, and rescores the ones
    // whose packed score reached the threshold
    const int32_t thresh = api_flag_threshold(SW_LANE_I16X2Q, gap_open, m->maxM);
    const int32_t skip_len = m->maxM > 0 ? (int32_t)((thresh + m->maxM - 1) / m->maxM) : INT32_MAX;
    if (m->qlen_no_i32 >= skip_len)  // cannot happen for matrix entries <= 127: skip_len >= 224 > 128
        return api_fail(SW_ERR_RANGE, "a short query could overflow the packed lanes of the batched launch");
    // the sequences of at least skip_len residues: a prefix of the order
    const int64_t n_prefix =
        skip_len == INT32_MAX ? 0
                              : (int64_t)(std::lower_bound(m->len_desc.begin(), m->len_desc.end(), (int64_t)skip_len,
                                                           [](int64_t x, int64_t v) { return x >= v; }) -
                                          m->len_desc.begin());

    cudaError_t err = cudaMemsetAsync(m->d_counters, 0, sizeof(unsigned long long) * (size_t)m->n_counters, st);
    // the rows of empty queries score 0
    for (size_t k = 0; k < m->empty_q.size() && err == cudaSuccess; ++k)
        err = cudaMemsetAsync(scores_out + (int64_t)m->empty_q[k] * row_stride, 0, sizeof(int32_t) * (size_t)m->n,
                              st);
    if (err != cudaSuccess)
        return api_cuda_fail((int)err, "cudaMemsetAsync");
    MultiArgs a;
    memset(&a, 0, sizeof(a));
    a.A = m->A;
    a.o = gap_open;
    a.e = gap_extend;
    a.min_m = m->minM;
    a.one = 1;
    a.db = m->res;
    a.off = m->off;
    a.order = m->order;
    a.skip_len = skip_len;
    a.flag_thresh = thresh;
    a.k_items = m->k_items;
    a.scores = scores_out;
    a.row_stride = row_stride;  // MultiQuery.row is the query's index
    a.rows = m->d_rows;
    a.done = m->d_done;
    a.status = m->d_status;
    a.wait_limit = m->wait_limit;
    a.wait_skew = m->wait_skew;
    const bool d0 = m->minM >= -gap_open;
    for (size_t k = 0; k < m->bins.size(); ++k) {
        const MultiBin &b = m->bins[k];
        a.queries = m->d_tables + b.tbl;
        a.n_queries = b.nq;
        a.n_items = m->n;
        a.counter = m->d_counters + b.cnt;
        a.bnd = b.kind == MULTI_FUSED && b.maxC > 1 ? m->d_bnd : nullptr;
        a.bnd_stride = m->bnd_stride;
        if (b.kind == MULTI_CHUNKS) {
            // every sequence starts before the bin's first phase (marks of
            // an earlier bin's walk would skip its waits)
            err = cudaMemsetAsync(m->d_done, 0xff, sizeof(int32_t) * (size_t)m->n, st);
            if (err != cudaSuccess)
                return api_cuda_fail((int)err, "cudaMemsetAsync(marks)");
        }
        const int kr = launch_multi_split(b.VL, b.S, b.kind, a, b.grid[d0 ? 1 : 0], st);
        if (kr)
            return api_cuda_fail(kr, "batched kernel launch");
    }
    const bool d032 = m->minM >= -(gap_open + gap_extend);
    for (int k = 0; k < 3; ++k) {
        const MultiI32 &s = m->i32[k];
        if (!s.nq || n_prefix == 0)
            continue;
        // its queries longest first: the long ones are a prefix of the table
        const int n_long = (int)(std::lower_bound(s.qlen_desc.begin(), s.qlen_desc.end(), skip_len,
                                                  [](int32_t x, int32_t v) { return x >= v; }) -
                                 s.qlen_desc.begin());
        if (n_long == 0)
            continue;
        a.queries = m->d_tables + s.tbl;
        a.n_queries = n_long;
        a.k_items = 1;
        a.n_items = n_prefix;
        a.counter = m->d_counters + m->n_counters - 3 + k;
        a.bnd = s.maxC > 1 ? m->d_bnd32 : nullptr;
        a.bnd_stride = m->bnd32_stride;
        const int kr = launch_multi_i32(s.S, a, s.grid[d032 ? 1 : 0], st);
        if (kr)
            return api_cuda_fail(kr, "batched int32 kernel launch");
    }
    return SW_OK;
}

}  // extern "C"
