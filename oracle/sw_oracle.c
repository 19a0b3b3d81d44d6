/*
 * Oracle for score-only Smith-Waterman/Gotoh local alignment (affine gaps).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Contents
 *   oracle_gotoh          plain int32 textbook recurrence (Section I: the
 *                         optimal local alignment score of two sequences in
 *                         O(mn); gap of length k costs o + (k-1)e as charged
 *                         by "H - GapOpen" then "- GapExtend" in Alg. 1/6).
 *   oracle_brute          enumeration of every local alignment (tiny inputs);
 *                         pins oracle_gotoh.
 *   oracle_gotoh_end,     the end cell of the best alignment (first in column
 *   oracle_brute_end      order) by the recurrence and by enumeration.
 *   oracle_striped_lazyf  Alg. 1 (striped layout, lazy-F correction loop) in
 *                         the paper's step order, with the readings listed
 *                         in its comment.
 *   oracle_striped_scan   Alg. 6 (striped layout, max-plus scan of F), in the
 *                         paper's step order, with the readings listed in
 *                         its comment.
 *   oracle_*_batch/pairs  the scalar recurrence over many pairs on host
 *                         threads (the timed CPU baseline).
 *
 * Domain: 0 <= gap_extend <= gap_open.  For gap_extend > gap_open the
 * recurrence would re-open a run instead of extending it and no longer
 * equals "one run of k costs o + (k-1)e"; the GPU boundary rejects it too.
 *
 * Conventions: residues are codes 0..A-1; the substitution matrix M is A*A,
 * row-major, indexed M[query residue][reference residue] (the query profile
 * of Alg. 1 is built from the query, so the query picks the row).  A code
 * >= A on either side is an unknown residue and scores the smallest entry of
 * M against anything (the paper has no such residues; this is the library's
 * convention, the same for every lane type).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define NEG_INF (INT32_MIN / 4)

static inline int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

/* smallest entry of M: the score of an unknown residue (code >= A) */
static int32_t min_entry(const int8_t *M, int32_t A)
{
    int32_t v = 127;
    for (int32_t i = 0; i < A * A; ++i)
        if (M[i] < v)
            v = M[i];
    return v;
}

/* M[qc][rc], or the smallest entry when either code is outside 0..A-1 */
static inline int32_t subst(const int8_t *M, int32_t A, int32_t minM, int32_t qc, int32_t rc)
{
    return (qc < A && rc < A) ? (int32_t)M[qc * A + rc] : minM;
}

/* ------------------------------------------------------------------------ */
/* Textbook Gotoh, int32.  Rows are query positions q = 1..m, columns are    */
/* reference positions r = 1..n:                                             */
/*   E(q,r) = max(H(q,r-1) - o, E(q,r-1) - e)     horizontal gap             */
/*   F(q,r) = max(H(q-1,r) - o, F(q-1,r) - e)     vertical gap               */
/*   H(q,r) = max(0, H(q-1,r-1) + M[Q_q][R_r], E(q,r), F(q,r))               */
/*   H(0,.) = H(.,0) = 0, E(.,0) = F(0,.) = -inf, score = max H (0 if empty) */
/* ------------------------------------------------------------------------ */
int32_t oracle_gotoh(const uint8_t *query, int32_t m, const uint8_t *ref,
                     int32_t n, const int8_t *M, int32_t A, int32_t o,
                     int32_t e)
{
    if (m <= 0 || n <= 0)
        return 0;
    const int32_t minM = min_entry(M, A);
    int32_t *Hcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t *Ecol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    for (int32_t q = 0; q <= m; ++q) {
        Hcol[q] = 0;       /* H(q, 0) */
        Ecol[q] = NEG_INF; /* E(q, 0) */
    }
    int32_t best = 0;
    for (int32_t r = 1; r <= n; ++r) {
        const int32_t rc = ref[r - 1];
        int32_t diag = 0;    /* H(q-1, r-1), starts at H(0, r-1) */
        int32_t up = 0;      /* H(q-1, r),   starts at H(0, r)   */
        int32_t F = NEG_INF; /* F(q-1, r),   starts at F(0, r)   */
        for (int32_t q = 1; q <= m; ++q) {
            const int32_t Eq = imax(Hcol[q] - o, Ecol[q] - e);
            const int32_t Fq = imax(up - o, F - e);
            int32_t H = diag + subst(M, A, minM, query[q - 1], rc);
            H = imax(H, Eq);
            H = imax(H, Fq);
            H = imax(H, 0);
            diag = Hcol[q];
            Hcol[q] = H;
            Ecol[q] = Eq;
            F = Fq;
            up = H;
            best = imax(best, H);
        }
    }
    free(Hcol);
    free(Ecol);
    return best;
}

/* ------------------------------------------------------------------------ */
/* End coordinates of the best local alignment: the first cell, in column-  */
/* major order (smallest reference position r, then smallest query position */
/* q, both 1-based), whose H equals the score; (-1, -1) when the score is 0. */
/* Same recurrence as oracle_gotoh.                                          */
/* ------------------------------------------------------------------------ */
int32_t oracle_gotoh_end(const uint8_t *query, int32_t m, const uint8_t *ref,
                         int32_t n, const int8_t *M, int32_t A, int32_t o,
                         int32_t e, int32_t *q_end, int32_t *r_end)
{
    *q_end = -1;
    *r_end = -1;
    if (m <= 0 || n <= 0)
        return 0;
    const int32_t minM = min_entry(M, A);
    int32_t *Hcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t *Ecol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    for (int32_t q = 0; q <= m; ++q) {
        Hcol[q] = 0;
        Ecol[q] = NEG_INF;
    }
    int32_t best = 0;
    for (int32_t r = 1; r <= n; ++r) {
        const int32_t rc = ref[r - 1];
        int32_t diag = 0, up = 0, F = NEG_INF;
        for (int32_t q = 1; q <= m; ++q) {
            const int32_t Eq = imax(Hcol[q] - o, Ecol[q] - e);
            const int32_t Fq = imax(up - o, F - e);
            int32_t H = diag + subst(M, A, minM, query[q - 1], rc);
            H = imax(imax(imax(H, Eq), Fq), 0);
            diag = Hcol[q];
            Hcol[q] = H;
            Ecol[q] = Eq;
            F = Fq;
            up = H;
            if (H > best) { /* strictly: keeps the first cell in column order */
                best = H;
                *q_end = q;
                *r_end = r;
            }
        }
    }
    free(Hcol);
    free(Ecol);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Brute force: every alignment of every pair of substrings.  An alignment  */
/* is a path of steps: match (one query and one reference residue, scored   */
/* M), query-only (I) or reference-only (D).  A maximal run of k steps of   */
/* one gap kind costs o + (k-1)e.  The empty alignment scores 0.  Paths may  */
/* start at any (i0, j0) and end anywhere, so every prefix is scored.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint8_t *q, *r;
    int32_t m, n, A, o, e;
    const int8_t *M;
    int32_t minM;
    int32_t best;
    int32_t best_q, best_r; /* end cell of the best path (1-based), first in column order */
} brute_ctx;

static void brute_walk(brute_ctx *c, int32_t i, int32_t j, int32_t last,
                       int32_t score)
{
    /* last: 0 = match or start, 1 = query-only gap, 2 = reference-only gap.
     * A path that has consumed query residues up to i and reference residues
     * up to j ends in cell (i, j); only paths whose last step is a match end
     * a maximal alignment (a trailing gap only lowers the score). */
    if (score > c->best) {
        c->best = score;
        c->best_q = i;
        c->best_r = j;
    } else if (score == c->best && score > 0 && last == 0 && i > 0 && j > 0 &&
               (j < c->best_r || (j == c->best_r && i < c->best_q))) {
        c->best_q = i;
        c->best_r = j;
    }
    if (i < c->m && j < c->n)
        brute_walk(c, i + 1, j + 1, 0, score + subst(c->M, c->A, c->minM, c->q[i], c->r[j]));
    if (i < c->m)
        brute_walk(c, i + 1, j, 1, score - (last == 1 ? c->e : c->o));
    if (j < c->n)
        brute_walk(c, i, j + 1, 2, score - (last == 2 ? c->e : c->o));
}

static int32_t brute_run(brute_ctx *c)
{
    if (c->m > 9 || c->n > 9)
        return -1; /* refuse: exponential */
    for (int32_t i0 = 0; i0 < c->m; ++i0)
        for (int32_t j0 = 0; j0 < c->n; ++j0)
            brute_walk(c, i0, j0, 0, 0);
    return c->best;
}

int32_t oracle_brute(const uint8_t *query, int32_t m, const uint8_t *ref,
                     int32_t n, const int8_t *M, int32_t A, int32_t o,
                     int32_t e)
{
    brute_ctx c = {query, ref, m, n, A, o, e, M, min_entry(M, A), 0, -1, -1};
    return brute_run(&c);
}

/* end cell of the best alignment by enumeration (-1, -1 when the score is 0) */
int32_t oracle_brute_end(const uint8_t *query, int32_t m, const uint8_t *ref,
                         int32_t n, const int8_t *M, int32_t A, int32_t o,
                         int32_t e, int32_t *q_end, int32_t *r_end)
{
    brute_ctx c = {query, ref, m, n, A, o, e, M, min_entry(M, A), 0, -1, -1};
    const int32_t s = brute_run(&c);
    *q_end = s > 0 ? c.best_q : -1;
    *r_end = s > 0 ? c.best_r : -1;
    return s;
}

/* ------------------------------------------------------------------------ */
/* Shared pieces of the two striped CPU variants.  A "vector" is p int32    */
/* lanes; lane l, segment index j holds query position l*segLen + j         */
/* (Alg. 1: segLen = (length(query) + p - 1) / p).  Values never go below   */
/* zero: "-" is subtraction floored at 0 (Section I) and "+ vprofile" is    */
/* floored at 0 too (local alignment).                                      */
/* ------------------------------------------------------------------------ */
static inline int32_t sat_sub(int32_t a, int32_t b) { return imax(a - b, 0); }

/* vprofile[c][j][lane]: score of query position lane*segLen+j against      */
/* residue c, c = 0..A (row A: an unknown residue).  Positions past the     */
/* query end get a score that keeps them at 0 after flooring (they can      */
/* never raise Max).                                                        */
static int32_t *build_vprofile(const uint8_t *query, int32_t m, const int8_t *M,
                               int32_t A, int32_t p, int32_t segLen)
{
    const int32_t minM = min_entry(M, A);
    int32_t *vp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A + 1) * segLen * p);
    for (int32_t c = 0; c <= A; ++c)
        for (int32_t j = 0; j < segLen; ++j)
            for (int32_t l = 0; l < p; ++l) {
                const int32_t pos = l * segLen + j;
                vp[((size_t)c * segLen + j) * p + l] =
                    pos < m ? subst(M, A, minM, query[pos], c) : NEG_INF;
            }
    return vp;
}

/* shift toward higher lanes by one, 0 into lane 0 (the paper's "<<< 1"). */
static inline void vshift(int32_t *dst, const int32_t *src, int32_t p)
{
    for (int32_t l = p - 1; l >= 1; --l)
        dst[l] = src[l - 1];
    dst[0] = 0;
}

/*
 * Alg. 1, striped Smith-Waterman with the lazy-F correction loop.
 * Readings where the listing is silent or ambiguous:
 *  - E is raised from the corrected H inside the correction loop, so a
 *    vertical gap carried in from an earlier segment may be followed by a
 *    horizontal gap exactly as within a segment (textbook Gotoh).
 *  - The exit test "(F - H) == 0" reads: every lane's carried F, after the
 *    extend step, is <= (H before this correction) - GapOpen.  Then the
 *    carry is dominated by the F the main pass already propagated.
 *  - "break" leaves the whole correction (all k rounds), not only the j loop.
 *  - Requires gap_extend <= gap_open (the carry only extends).
 * *lazy_steps (if non-NULL) accumulates the j-steps executed by the
 * correction loop (the corrective factor C of Section I times n/p).
 */
int32_t oracle_striped_lazyf(const uint8_t *query, int32_t m,
                             const uint8_t *ref, int32_t n, const int8_t *M,
                             int32_t A, int32_t o, int32_t e, int32_t p,
                             int64_t *lazy_steps)
{
    if (m <= 0 || n <= 0 || p <= 0)
        return 0;
    const int32_t segLen = (m + p - 1) / p;
    int32_t *vprofile = build_vprofile(query, m, M, A, p, segLen);
    const size_t vecs = (size_t)segLen * p;
    int32_t *HStore = (int32_t *)calloc(vecs, sizeof(int32_t));
    int32_t *HLoad = (int32_t *)calloc(vecs, sizeof(int32_t));
    int32_t *Earr = (int32_t *)calloc(vecs, sizeof(int32_t));
    int32_t *H = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *F = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *T = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t Max = 0;
    int64_t steps = 0;

    for (int32_t i = 0; i < n; ++i) {
        const int32_t *vp = vprofile + (size_t)(ref[i] < A ? ref[i] : A) * segLen * p;
        for (int32_t l = 0; l < p; ++l)
            F[l] = 0;
        vshift(H, HStore + (size_t)(segLen - 1) * p, p);
        int32_t *tmp = HLoad;
        HLoad = HStore;
        HStore = tmp;
        for (int32_t j = 0; j < segLen; ++j) {
            int32_t *Ej = Earr + (size_t)j * p;
            int32_t *HSj = HStore + (size_t)j * p;
            const int32_t *HLj = HLoad + (size_t)j * p;
            for (int32_t l = 0; l < p; ++l) {
                int32_t h = imax(H[l] + vp[(size_t)j * p + l], 0);
                Max = imax(Max, h);
                h = imax(h, Ej[l]);
                h = imax(h, F[l]);
                HSj[l] = h;
                h = sat_sub(h, o);
                Ej[l] = imax(sat_sub(Ej[l], e), h);
                F[l] = imax(sat_sub(F[l], e), h);
                H[l] = HLj[l];
            }
        }
        /* lazy-F correction */
        int done = 0;
        for (int32_t k = 1; k <= p && !done; ++k) {
            vshift(T, F, p);
            memcpy(F, T, sizeof(int32_t) * p);
            for (int32_t j = 0; j < segLen; ++j) {
                int32_t *HSj = HStore + (size_t)j * p;
                int32_t *Ej = Earr + (size_t)j * p;
                int all_dominated = 1;
                ++steps;
                for (int32_t l = 0; l < p; ++l) {
                    const int32_t hold = HSj[l];
                    HSj[l] = imax(hold, F[l]);
                    Ej[l] = imax(Ej[l], sat_sub(HSj[l], o));
                    F[l] = sat_sub(F[l], e);
                    if (F[l] > sat_sub(hold, o))
                        all_dominated = 0;
                }
                if (all_dominated) {
                    done = 1;
                    break;
                }
            }
        }
    }
    if (lazy_steps)
        *lazy_steps += steps;
    free(vprofile);
    free(HStore);
    free(HLoad);
    free(Earr);
    free(H);
    free(F);
    free(T);
    return Max;
}

/*
 * Alg. 6, striped Smith-Waterman with the max-plus scan of F.
 * Readings where the listing is garbled or silent:
 *  - Two carries: carryPrev is the scan result of the previous column and
 *    feeds the deferred corrections of this column (the "Fj" read before the
 *    loop and inside it); carryNew starts at 0 and is filled by this
 *    column's scan.  The listing's single Fj (reset to 0 at the top) cannot
 *    serve both.
 *  - E is raised from the corrected H as well: before E[j] is used in
 *    column i it is maxed with (carryPrev - j*GapExtend) - GapOpen, the
 *    correction the previous column's H at position j received.
 *  - The scan is the paper's p-step loop (the GPU replaces it by a log p
 *    shuffle scan computing the same values).
 *  - Requires gap_extend <= gap_open (the carry only extends).
 */
int32_t oracle_striped_scan(const uint8_t *query, int32_t m, const uint8_t *ref,
                            int32_t n, const int8_t *M, int32_t A, int32_t o,
                            int32_t e, int32_t p)
{
    if (m <= 0 || n <= 0 || p <= 0)
        return 0;
    const int32_t segLen = (m + p - 1) / p;
    int32_t *vprofile = build_vprofile(query, m, M, A, p, segLen);
    const size_t vecs = (size_t)segLen * p;
    int32_t *HStore = (int32_t *)calloc(vecs, sizeof(int32_t));
    int32_t *HLoad = (int32_t *)calloc(vecs, sizeof(int32_t));
    int32_t *Earr = (int32_t *)calloc(vecs, sizeof(int32_t));
    int32_t *H = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *F = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *T = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *Fj = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *carryPrev = (int32_t *)calloc((size_t)p, sizeof(int32_t));
    int32_t *carryNew = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t Max = 0;

    for (int32_t i = 0; i < n; ++i) {
        const int32_t *vp = vprofile + (size_t)(ref[i] < A ? ref[i] : A) * segLen * p;
        for (int32_t l = 0; l < p; ++l) {
            F[l] = 0;
            carryNew[l] = 0;
            /* deferred correction of the last element before the shift */
            T[l] = imax(HStore[(size_t)(segLen - 1) * p + l],
                        sat_sub(carryPrev[l], (segLen - 1) * e));
        }
        vshift(H, T, p);
        int32_t *tmp = HLoad;
        HLoad = HStore;
        HStore = tmp;
        for (int32_t l = 0; l < p; ++l)
            Fj[l] = carryPrev[l];
        for (int32_t j = 0; j < segLen; ++j) {
            int32_t *Ej = Earr + (size_t)j * p;
            int32_t *HSj = HStore + (size_t)j * p;
            const int32_t *HLj = HLoad + (size_t)j * p;
            for (int32_t l = 0; l < p; ++l) {
                /* E(i) from the corrected H(i-1) at this position */
                Ej[l] = imax(Ej[l], sat_sub(Fj[l], o));
                int32_t h = imax(H[l] + vp[(size_t)j * p + l], 0);
                Max = imax(Max, h);
                h = imax(h, Ej[l]);
                h = imax(h, F[l]);
                HSj[l] = h;
                h = sat_sub(h, o);
                Ej[l] = imax(sat_sub(Ej[l], e), h);
                F[l] = imax(sat_sub(F[l], e), h);
                /* previous column's H at j, corrected, is the next diagonal */
                H[l] = imax(HLj[l], Fj[l]);
                Fj[l] = sat_sub(Fj[l], e);
            }
        }
        /* scan: carry into lane l = max_k (Fout[l-k] - (k-1)*segLen*e) */
        for (int32_t k = 1; k <= p; ++k) {
            vshift(T, F, p);
            for (int32_t l = 0; l < p; ++l) {
                carryNew[l] = imax(carryNew[l], T[l]);
                F[l] = sat_sub(T[l], segLen * e);
            }
        }
        memcpy(carryPrev, carryNew, sizeof(int32_t) * p);
    }
    free(vprofile);
    free(HStore);
    free(HLoad);
    free(Earr);
    free(H);
    free(F);
    free(T);
    free(Fj);
    free(carryPrev);
    free(carryNew);
    return Max;
}

/* ------------------------------------------------------------------------ */
/* Many pairs on host threads (scalar recurrence per pair).                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint8_t *q;
    const int64_t *qoff; /* NULL: one query of length m for every pair */
    int32_t m;
    const uint8_t *r;
    const int64_t *roff;
    int64_t npairs;
    const int8_t *M;
    int32_t A, o, e;
    int32_t *out;
    int64_t next;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *b = (batch_job *)arg;
    for (;;) {
        const int64_t start = __atomic_fetch_add(&b->next, 16, __ATOMIC_RELAXED);
        if (start >= b->npairs)
            break;
        const int64_t stop = start + 16 < b->npairs ? start + 16 : b->npairs;
        for (int64_t k = start; k < stop; ++k) {
            const uint8_t *q = b->q;
            int32_t m = b->m;
            if (b->qoff) {
                q = b->q + b->qoff[k];
                m = (int32_t)(b->qoff[k + 1] - b->qoff[k]);
            }
            b->out[k] = oracle_gotoh(q, m, b->r + b->roff[k],
                                     (int32_t)(b->roff[k + 1] - b->roff[k]),
                                     b->M, b->A, b->o, b->e);
        }
    }
    return NULL;
}

static void run_batch(batch_job *b, int32_t nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    b->next = 0;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int32_t t = 0; t < nthreads; ++t)
        pthread_create(&th[t], NULL, batch_worker, b);
    for (int32_t t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    free(th);
}

typedef struct {
    const uint8_t *q;
    int32_t m;
    const uint8_t *r;
    const int64_t *roff;
    int64_t n;
    const int8_t *M;
    int32_t A, o, e;
    int32_t *out, *qe, *re;
    int64_t next;
} ends_job;

static void *ends_worker(void *arg)
{
    ends_job *b = (ends_job *)arg;
    for (;;) {
        const int64_t start = __atomic_fetch_add(&b->next, 16, __ATOMIC_RELAXED);
        if (start >= b->n)
            break;
        const int64_t stop = start + 16 < b->n ? start + 16 : b->n;
        for (int64_t k = start; k < stop; ++k)
            b->out[k] = oracle_gotoh_end(b->q, b->m, b->r + b->roff[k], (int32_t)(b->roff[k + 1] - b->roff[k]),
                                         b->M, b->A, b->o, b->e, &b->qe[k], &b->re[k]);
    }
    return NULL;
}

/* scores and end cells of one query against n_db sequences */
void oracle_gotoh_end_batch(const uint8_t *query, int32_t m, const uint8_t *db,
                            const int64_t *db_off, int64_t n_db, const int8_t *M,
                            int32_t A, int32_t o, int32_t e, int32_t *out,
                            int32_t *q_end, int32_t *r_end, int32_t nthreads)
{
    ends_job b = {query, m, db, db_off, n_db, M, A, o, e, out, q_end, r_end, 0};
    if (nthreads < 1)
        nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int32_t t = 0; t < nthreads; ++t)
        pthread_create(&th[t], NULL, ends_worker, &b);
    for (int32_t t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    free(th);
}

/* one query against n_db reference sequences (concatenated, offsets n+1) */
void oracle_gotoh_batch(const uint8_t *query, int32_t m, const uint8_t *db,
                        const int64_t *db_off, int64_t n_db, const int8_t *M,
                        int32_t A, int32_t o, int32_t e, int32_t *out,
                        int32_t nthreads)
{
    batch_job b = {query, NULL, m, db, db_off, n_db, M, A, o, e, out, 0};
    run_batch(&b, nthreads);
}

/* pair k: query q[qoff[k]..qoff[k+1]) against r[roff[k]..roff[k+1]) */
void oracle_gotoh_pairs(const uint8_t *q, const int64_t *qoff,
                        const uint8_t *r, const int64_t *roff, int64_t npairs,
                        const int8_t *M, int32_t A, int32_t o, int32_t e,
                        int32_t *out, int32_t nthreads)
{
    batch_job b = {q, qoff, 0, r, roff, npairs, M, A, o, e, out, 0};
    run_batch(&b, nthreads);
}
