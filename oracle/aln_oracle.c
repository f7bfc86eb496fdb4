/*
 * aln_oracle.c -- plain, slow, obviously-correct CPU oracle for the BWA-aln
 * inexact search over an FM-index, as used by BarraCUDA.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into its own shared library
 * and is loaded by the tests, by the smoke check and by the benchmark's
 * CPU-baseline leg.  The product library never links, includes or calls it, and
 * it shares no code, header or table with the CUDA path.
 *
 * What it follows (paper: "Genetically Improved BarraCUDA", Sec. 2 "NextGen DNA
 * Sequence Alignment"):
 *  - the index groups all suffixes that share a prefix into one contiguous
 *    range, so that extending the prefix by a base maps a range to a sub-range
 *    (index principle, Sec. 2);
 *  - lookup keeps a lower and an upper pointer that every processed base
 *    updates from index data; their distance is the number of matching
 *    positions, and crossed pointers mean no match (backward search, Sec. 2);
 *  - for non-exact matches the search backs up and tries alternatives
 *    (bounded backtracking, Sec. 2).
 * The paper gives no finer detail.  The D lower-bound array, the gap limits, the
 * seed rule, the strata and the counts follow BWA's short-read method as read in
 * the project's design notes; each rule is stated where it is implemented.
 *
 * Conventions.  Text X over codes A0 C1 G2 T3 (N is replaced before indexing);
 * Xr = X reversed.  For a text Y, SA and B (the BWT) are over Y$ ($ smallest),
 * C[c] = number of symbols < c in Y, Occ(c, r) = number of c in B[0..r].
 * Extending the closed interval [k, l] by c gives
 *     k' = C[c] + Occ(c, k-1) + 1,   l' = C[c] + Occ(c, l),
 * empty iff k' > l'.  The empty string has the interval [0, n].
 *
 * Parity status: every function here is pinned by tests (brute force over all
 * alignments on tiny texts, exact-match counts, Hamming scans, LF inversion,
 * a hand-worked example, D-safety); none is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OCK 64            /* Occ checkpoint spacing (rows) */
#define SYM_DOLLAR 4
#define READ_MAX 255      /* longest read searched; longer reads are flagged */
#define Z_MAX 7           /* largest per-read difference limit accepted */

/* result flags (same meaning as the product's, defined independently) */
#define F_HIT_OVERFLOW 0x01
#define F_READ_TOO_LONG 0x08
#define F_BAD_LIMIT 0x10
#define F_MANY_BEST 0x80
#define STRATA_SCORE 2    /* score-ordered mode: see align_one */

typedef struct {
    uint64_t n;        /* text length without $ */
    uint8_t *text;     /* codes 0..3, length n */
    uint32_t *sa;      /* n+1 suffix starts in sorted order */
    uint8_t *bwt;      /* n+1 symbols, SYM_DOLLAR at the primary row */
    uint32_t *ck;      /* ck[4*b + c] = count of c in bwt[0 .. b*OCK-1] */
    uint64_t C[4];
    uint64_t primary;
} otext;

typedef struct {
    otext t[2];        /* t[0] = X, t[1] = Xr */
} orc_index;

/* ------------------------------------------------------------ N replacement */

/* SplitMix64 output function (Steele, Lea, Flood 2014) on state x + golden. */
static uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The mix function itself (exported for its pin against published outputs). */
uint64_t orc_mix64(uint64_t x) { return mix64(x); }

/* ------------------------------------------------------------ suffix sort */

static const uint8_t *g_sort_text;
static uint64_t g_sort_n;

/* Compare suffixes i and j of text$: byte-wise, the shorter is smaller on a tie. */
static int suffix_cmp(uint32_t i, uint32_t j)
{
    uint64_t li = g_sort_n - i, lj = g_sort_n - j;
    uint64_t m = li < lj ? li : lj;
    int c = memcmp(g_sort_text + i, g_sort_text + j, m);
    if (c) return c;
    return li < lj ? -1 : (li > lj ? 1 : 0);
}

static int qsort_cmp(const void *a, const void *b)
{
    return suffix_cmp(*(const uint32_t *)a, *(const uint32_t *)b);
}

/* Bucket of suffix i: its first bk symbols as a base-4 number, a suffix shorter
 * than bk symbols padded with A (code 0).  Such a short suffix is smaller than
 * every other suffix of its bucket (they all continue it, and $ is the smallest
 * symbol), and the bucket order agrees with the suffix order otherwise, so
 * sorting every bucket with the comparator gives the order of one global sort. */
static uint64_t bucket_of(const uint8_t *text, uint64_t n, uint64_t i, int bk)
{
    uint64_t key = 0;
    for (int j = 0; j < bk; j++) key = 4 * key + (i + j < n ? text[i + j] : 0);
    return key;
}

typedef struct {
    const uint8_t *text;
    uint64_t n, lo, hi;     /* suffix starts [lo, hi) of this thread */
    int bk;
    uint32_t *count;        /* per-thread bucket counts, then write cursors */
    uint32_t *out;
} scatter_job;

static void *count_worker(void *p)
{
    scatter_job *j = (scatter_job *)p;
    for (uint64_t i = j->lo; i < j->hi; i++) j->count[bucket_of(j->text, j->n, i, j->bk)]++;
    return NULL;
}

static void *scatter_worker(void *p)
{
    scatter_job *j = (scatter_job *)p;
    for (uint64_t i = j->lo; i < j->hi; i++) {
        uint64_t b = bucket_of(j->text, j->n, i, j->bk);
        j->out[j->count[b]++] = (uint32_t)i;
    }
    return NULL;
}

typedef struct {
    uint32_t *a;            /* suffix starts, grouped by bucket */
    const uint64_t *start;  /* bucket b is a[start[b] .. start[b+1]-1] */
    uint64_t n_buckets, next;
    pthread_mutex_t *mu;
} bucket_job;

static void *bucket_sort_worker(void *p)
{
    bucket_job *j = (bucket_job *)p;
    for (;;) {
        pthread_mutex_lock(j->mu);
        uint64_t b0 = j->next, b1 = b0 + 1024 < j->n_buckets ? b0 + 1024 : j->n_buckets;
        j->next = b1;
        pthread_mutex_unlock(j->mu);
        if (b0 >= j->n_buckets) break;
        for (uint64_t b = b0; b < b1; b++) {
            uint64_t len = j->start[b + 1] - j->start[b];
            if (len > 1) qsort(j->a + j->start[b], len, sizeof(uint32_t), qsort_cmp);
        }
    }
    return NULL;
}

/* Naive suffix sort of text$ (text of length n): suffix starts grouped by their
 * first bk symbols (bk = 0: chosen from n), then every group sorted by qsort
 * with the byte-wise comparator, groups in parallel. */
static int naive_sa(const uint8_t *text, uint64_t n, uint32_t *sa, int nthreads, int bk)
{
    g_sort_text = text;
    g_sort_n = n;
    sa[0] = (uint32_t)n;                 /* the suffix "$" is the smallest */
    if (n == 0) return 0;
    if (bk <= 0) {                       /* about 64 suffixes per bucket, 1..12 symbols */
        bk = 1;
        while (bk < 12 && ((uint64_t)1 << (2 * bk)) * 64 < n) bk++;
    }
    if (bk > 12) bk = 12;
    uint64_t nb = (uint64_t)1 << (2 * bk);
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > n / 4096 + 1) nthreads = (int)(n / 4096 + 1);
    while (nthreads > 1 && (uint64_t)nthreads * nb * sizeof(uint32_t) > ((uint64_t)2 << 30)) nthreads--;
    uint32_t *count = (uint32_t *)calloc((uint64_t)nthreads * nb, sizeof(uint32_t));
    uint64_t *start = (uint64_t *)malloc((nb + 1) * sizeof(uint64_t));
    pthread_t *th = (pthread_t *)malloc(nthreads * sizeof(pthread_t));
    scatter_job *sj = (scatter_job *)malloc(nthreads * sizeof(scatter_job));
    if (!count || !start || !th || !sj) return -1;
    for (int t = 0; t < nthreads; t++) {
        sj[t].text = text; sj[t].n = n; sj[t].bk = bk; sj[t].out = sa + 1;
        sj[t].lo = n * (uint64_t)t / nthreads;
        sj[t].hi = n * (uint64_t)(t + 1) / nthreads;
        sj[t].count = count + (uint64_t)t * nb;
        pthread_create(&th[t], NULL, count_worker, &sj[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    /* bucket b starts after all smaller buckets; thread t writes after threads < t */
    uint64_t acc = 0;
    for (uint64_t b = 0; b < nb; b++) {
        start[b] = acc;
        for (int t = 0; t < nthreads; t++) {
            uint32_t c = count[(uint64_t)t * nb + b];
            count[(uint64_t)t * nb + b] = (uint32_t)acc;  /* cursor (acc < n < 2^32) */
            acc += c;
        }
    }
    start[nb] = acc;
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, scatter_worker, &sj[t]);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(count);
    pthread_mutex_t mu;
    pthread_mutex_init(&mu, NULL);
    bucket_job bj = {sa + 1, start, nb, 0, &mu};
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, bucket_sort_worker, &bj);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&mu);
    free(start); free(th); free(sj);
    return 0;
}

/* ------------------------------------------------------------ index */

typedef struct { const otext *t; uint64_t lo, hi; uint8_t *bwt; } bwt_job;

/* B[r] = Y[SA[r]-1], or $ where SA[r] = 0, for rows [lo, hi) */
static void *bwt_worker(void *p)
{
    bwt_job *j = (bwt_job *)p;
    for (uint64_t r = j->lo; r < j->hi; r++) {
        uint32_t s = j->t->sa[r];
        j->bwt[r] = s == 0 ? SYM_DOLLAR : j->t->text[s - 1];
    }
    return NULL;
}

static int build_text(otext *t, const uint8_t *codes, uint64_t n, int nthreads, int bk)
{
    t->n = n;
    t->text = (uint8_t *)malloc(n ? n : 1);
    t->sa = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    t->bwt = (uint8_t *)malloc(n + 1);
    uint64_t nck = (n + 1) / OCK + 2;
    t->ck = (uint32_t *)calloc(4 * nck, sizeof(uint32_t));
    if (!t->text || !t->sa || !t->bwt || !t->ck) return -1;
    memcpy(t->text, codes, n);
    if (naive_sa(t->text, n, t->sa, nthreads, bk)) return -1;
    int nt = nthreads < 1 ? 1 : nthreads;
    pthread_t th[256];
    bwt_job bj[256];
    if (nt > 256) nt = 256;
    for (int q = 0; q < nt; q++) {
        bj[q].t = t; bj[q].bwt = t->bwt;
        bj[q].lo = (n + 1) * (uint64_t)q / nt;
        bj[q].hi = (n + 1) * (uint64_t)(q + 1) / nt;
        pthread_create(&th[q], NULL, bwt_worker, &bj[q]);
    }
    for (int q = 0; q < nt; q++) pthread_join(th[q], NULL);
    for (uint64_t r = 0; r <= n; r++)
        if (t->bwt[r] == SYM_DOLLAR) t->primary = r;
    /* C[c] = number of symbols smaller than c in Y */
    uint64_t cnt[4] = {0, 0, 0, 0};
    for (uint64_t i = 0; i < n; i++) cnt[t->text[i]]++;
    t->C[0] = 0;
    for (int c = 1; c < 4; c++) t->C[c] = t->C[c - 1] + cnt[c - 1];
    /* checkpoints: plain running counts */
    uint32_t run[4] = {0, 0, 0, 0};
    for (uint64_t r = 0; r <= n + 1; r++) {
        if (r % OCK == 0) for (int c = 0; c < 4; c++) t->ck[4 * (r / OCK) + c] = run[c];
        if (r <= n && t->bwt[r] < 4) run[t->bwt[r]]++;
    }
    return 0;
}

/* Occ(c, r): number of c in B[0..r]; r = -1 gives 0. */
static uint64_t occ(const otext *t, int c, int64_t r)
{
    if (r < 0) return 0;
    uint64_t rows = (uint64_t)r + 1;
    uint64_t b = rows / OCK;
    uint64_t v = t->ck[4 * b + c];
    for (uint64_t i = b * OCK; i < rows; i++) v += (t->bwt[i] == c);
    return v;
}

/* Extend [k, l] by c (prepend c to the pattern).  Returns 1 if non-empty. */
static int lf_extend(const otext *t, int c, uint64_t k, uint64_t l, uint64_t *k2, uint64_t *l2)
{
    uint64_t a = t->C[c] + occ(t, c, (int64_t)k - 1) + 1;
    uint64_t b = t->C[c] + occ(t, c, (int64_t)l);
    *k2 = a;
    *l2 = b;
    return a <= b;
}

/* Index of X and of Xr.  bucket_k: leading symbols the suffix sort groups by
 * before sorting each group (0 = chosen from n); the suffix array does not
 * depend on it. */
orc_index *orc_build(const uint8_t *codes, uint64_t n, uint64_t n_seed, int nthreads, int bucket_k)
{
    if (n >= 0xFFFFFFFFULL) return NULL;
    orc_index *ix = (orc_index *)calloc(1, sizeof(orc_index));
    uint8_t *x = (uint8_t *)malloc(n ? n : 1);
    uint8_t *xr = (uint8_t *)malloc(n ? n : 1);
    if (!ix || !x || !xr) return NULL;
    /* every N (code 4, or anything above 3) becomes mix64(n_seed ^ pos) & 3 */
    for (uint64_t i = 0; i < n; i++)
        x[i] = codes[i] < 4 ? codes[i] : (uint8_t)(mix64(n_seed ^ i) & 3);
    for (uint64_t i = 0; i < n; i++) xr[i] = x[n - 1 - i];
    if (build_text(&ix->t[0], x, n, nthreads, bucket_k) || build_text(&ix->t[1], xr, n, nthreads, bucket_k))
        return NULL;
    free(x);
    free(xr);
    return ix;
}

void orc_free(orc_index *ix)
{
    if (!ix) return;
    for (int w = 0; w < 2; w++) {
        free(ix->t[w].text); free(ix->t[w].sa); free(ix->t[w].bwt); free(ix->t[w].ck);
    }
    free(ix);
}

uint64_t orc_n(const orc_index *ix) { return ix->t[0].n; }
void orc_get_text(const orc_index *ix, int w, uint8_t *out) { memcpy(out, ix->t[w].text, ix->t[w].n); }
void orc_get_sa(const orc_index *ix, int w, uint32_t *out) { memcpy(out, ix->t[w].sa, (ix->t[w].n + 1) * 4); }
void orc_get_bwt(const orc_index *ix, int w, uint8_t *out) { memcpy(out, ix->t[w].bwt, ix->t[w].n + 1); }
void orc_get_C(const orc_index *ix, int w, uint64_t *out) { memcpy(out, ix->t[w].C, 4 * sizeof(uint64_t)); }
uint64_t orc_primary(const orc_index *ix, int w) { return ix->t[w].primary; }
uint64_t orc_occ(const orc_index *ix, int w, int c, int64_t r) { return occ(&ix->t[w], c, r); }

/* Exact backward search of pattern p[0..len-1] in text w: the pattern is
 * extended from its last symbol to its first.  Returns 1 and [k, l] if present. */
int orc_exact(const orc_index *ix, int w, const uint8_t *p, int len, uint64_t *k, uint64_t *l)
{
    const otext *t = &ix->t[w];
    uint64_t a = 0, b = t->n;
    for (int i = len - 1; i >= 0; i--) {
        if (p[i] > 3) return 0;
        if (!lf_extend(t, p[i], a, b, &a, &b)) return 0;
    }
    *k = a;
    *l = b;
    return 1;
}

/* ------------------------------------------------------------ search */

typedef struct {
    int z;               /* default difference limit (used when no per-read z) */
    int max_gapo, max_gape;
    int seed_len, seed_z;
    int indel_end_skip;  /* e */
    int hit_cap;
    int strata;          /* 0 = BEST1, 1 = FULL */
    int use_d;           /* 1 = prune with D, 0 = D taken as all zero */
    int sc_mm, sc_gapo, sc_gape; /* score-ordered mode: penalty of a mismatch, gap open, gap extension */
    int max_best;        /* score-ordered mode: more best placements than this list the best only; 0 = no cap */
} orc_params;

typedef struct {         /* one reported hit */
    uint32_t k, l;
    uint16_t aligned_len;
    uint8_t strand, n_diff, n_mm, n_gapo, n_gape, pad;
} orc_hit;

typedef struct {
    uint32_t c0, c1;
    uint8_t n_hits, flags, d_best, pad;
} orc_res;

typedef struct {
    const orc_index *ix;
    const otext *I;        /* index searched for this strand */
    uint8_t q[READ_MAX];   /* processed symbols */
    int m;
    int D[READ_MAX + 1];
    int budget;
    int strand;
    const orc_params *p;
    orc_hit *cand;
    int n_cand, cap_cand;
    uint64_t lookups;
} ctx_t;

enum { OP_M = 0, OP_I = 1, OP_D = 2 };

/* witness order: (diffs, n_gapo, n_gape, n_mm, aligned_len) */
/* Penalty score of a witness (score-ordered mode): lower is better. */
static int score_of(const orc_params *p, const orc_hit *h)
{
    return p->sc_mm * h->n_mm + p->sc_gapo * h->n_gapo + p->sc_gape * h->n_gape;
}

/* witness order: (diffs, n_gapo, n_gape, n_mm, aligned_len), in the
 * score-ordered mode preceded by the score */
static int witness_less(const orc_hit *a, const orc_hit *b, const orc_params *p)
{
    if (p->strata == STRATA_SCORE) {
        int sa = score_of(p, a), sb = score_of(p, b);
        if (sa != sb) return sa < sb;
    }
    if (a->n_diff != b->n_diff) return a->n_diff < b->n_diff;
    if (a->n_gapo != b->n_gapo) return a->n_gapo < b->n_gapo;
    if (a->n_gape != b->n_gape) return a->n_gape < b->n_gape;
    if (a->n_mm != b->n_mm) return a->n_mm < b->n_mm;
    return a->aligned_len < b->aligned_len;
}

/* Record a candidate; equal (strand, k, l) merge keeping the minimal witness. */
static void record(ctx_t *c, uint64_t k, uint64_t l, int n_mm, int n_gapo, int n_gape, int alen)
{
    orc_hit h;
    memset(&h, 0, sizeof h);
    h.k = (uint32_t)k; h.l = (uint32_t)l; h.strand = (uint8_t)c->strand;
    h.n_mm = (uint8_t)n_mm; h.n_gapo = (uint8_t)n_gapo; h.n_gape = (uint8_t)n_gape;
    h.n_diff = (uint8_t)(n_mm + n_gapo + n_gape); h.aligned_len = (uint16_t)alen;
    for (int i = 0; i < c->n_cand; i++) {
        orc_hit *o = &c->cand[i];
        if (o->strand == h.strand && o->k == h.k && o->l == h.l) {
            if (witness_less(&h, o, c->p)) *o = h;
            return;
        }
    }
    if (c->n_cand == c->cap_cand) {
        c->cap_cand = c->cap_cand ? 2 * c->cap_cand : 64;
        c->cand = (orc_hit *)realloc(c->cand, c->cap_cand * sizeof(orc_hit));
    }
    c->cand[c->n_cand++] = h;
}

/*
 * Depth-first enumeration of all edit transcripts of the processed symbols
 * q[0..m-1] within the budget.  State: i symbols consumed, interval [k, l] of
 * the target built so far, the counts, and the last operation (for telling a
 * gap open from a gap extension).
 *  - match / mismatch: extend by each base b; b = q[i] is a match (an N never
 *    matches), any other b is a mismatch;
 *  - insertion: consume q[i] without extending, allowed for e <= i <= m-1-e;
 *  - deletion: extend by b without consuming, placed before read index i,
 *    allowed for max(e,1) <= i <= m-max(e,1);
 *  - a run of insertions (or of deletions) of length g costs one gap open and
 *    g-1 gap extensions, and g differences;
 *  - seed: an operation at read index i < seed_len (a deletion placed before
 *    index i) adds one seed difference, limited by seed_z when seed_len > 0;
 *  - pruning: stop when budget - diffs < D[i] (D is a lower bound on the
 *    differences needed by q[i..m-1]).
 * A node at i = m with a non-empty target is a candidate hit.
 */
static void dfs(ctx_t *c, int i, uint64_t k, uint64_t l, int n_mm, int n_gapo, int n_gape,
                int n_ins, int n_del, int seed, int last)
{
    const orc_params *p = c->p;
    int diffs = n_mm + n_gapo + n_gape;
    if (c->budget - diffs < c->D[i]) return;
    if (i == c->m) {
        int alen = i + n_del - n_ins;
        if (alen >= 1) record(c, k, l, n_mm, n_gapo, n_gape, alen);
        return;
    }
    int m = c->m, e = p->indel_end_skip;
    int in_seed = (p->seed_len > 0 && i < p->seed_len);
    int seed_ok = !in_seed || (seed + 1 <= p->seed_z);
    int seed2 = seed + in_seed;
    uint64_t kk[4], ll[4];
    int ne[4];
    c->lookups += 2; /* one 4-symbol Occ evaluation at rows k-1 and l */
    for (int b = 0; b < 4; b++) ne[b] = lf_extend(c->I, b, k, l, &kk[b], &ll[b]);
    /* match and mismatches */
    for (int b = 0; b < 4; b++) {
        if (!ne[b]) continue;
        if (c->q[i] == b)
            dfs(c, i + 1, kk[b], ll[b], n_mm, n_gapo, n_gape, n_ins, n_del, seed, OP_M);
        else if (seed_ok)
            dfs(c, i + 1, kk[b], ll[b], n_mm + 1, n_gapo, n_gape, n_ins, n_del, seed2, OP_M);
    }
    /* insertion of q[i] */
    if (seed_ok && i >= e && i <= m - 1 - e) {
        if (last == OP_I) {
            if (n_gape + 1 <= p->max_gape)
                dfs(c, i + 1, k, l, n_mm, n_gapo, n_gape + 1, n_ins + 1, n_del, seed2, OP_I);
        } else if (n_gapo + 1 <= p->max_gapo) {
            dfs(c, i + 1, k, l, n_mm, n_gapo + 1, n_gape, n_ins + 1, n_del, seed2, OP_I);
        }
    }
    /* deletion of a target base before read index i */
    int e1 = e < 1 ? 1 : e;
    if (seed_ok && i >= e1 && i <= m - e1) {
        for (int b = 0; b < 4; b++) {
            if (!ne[b]) continue;
            if (last == OP_D) {
                if (n_gape + 1 <= p->max_gape)
                    dfs(c, i, kk[b], ll[b], n_mm, n_gapo, n_gape + 1, n_ins, n_del + 1, seed2, OP_D);
            } else if (n_gapo + 1 <= p->max_gapo) {
                dfs(c, i, kk[b], ll[b], n_mm, n_gapo + 1, n_gape, n_ins, n_del + 1, seed2, OP_D);
            }
        }
    }
}

/*
 * D array for the processed symbols q[0..m-1] against the text of `other`:
 * scan from the far end, extending the segment q[j..] one symbol at a time
 * (a symbol is prepended, so the segment is matched in the same orientation as
 * the search target); when it no longer occurs (or the symbol is N) count one
 * difference and restart with an empty segment.  D[j] = count after symbol j,
 * D[m] = 0.  Each disjoint failed segment needs at least one difference.
 */
static uint64_t dscan(const otext *other, const uint8_t *q, int m, int *D)
{
    uint64_t look = 0;
    uint64_t k = 0, l = other->n;
    int cnt = 0;
    D[m] = 0;
    for (int j = m - 1; j >= 0; j--) {
        int ok = 0;
        if (q[j] < 4) {
            look += 2;
            ok = lf_extend(other, q[j], k, l, &k, &l);
        }
        if (!ok) {
            cnt++;
            k = 0;
            l = other->n;
        }
        D[j] = cnt;
    }
    return look;
}

/* Strand setup: strand 0 searches q = W on the index of Xr (D from X);
 * strand 1 searches q = complement(W) on the index of X (D from Xr).  Both
 * process the read from its 5' end. */
static void setup_strand(ctx_t *c, const orc_index *ix, const uint8_t *w, int m, int strand)
{
    c->strand = strand;
    c->m = m;
    for (int i = 0; i < m; i++) {
        uint8_t b = w[i];
        c->q[i] = (b > 3) ? 4 : (strand ? (uint8_t)(3 - b) : b);
    }
    c->I = &ix->t[strand ? 0 : 1];
}

static int cand_order(const void *a, const void *b)
{
    const orc_hit *x = (const orc_hit *)a, *y = (const orc_hit *)b;
    if (x->n_diff != y->n_diff) return x->n_diff < y->n_diff ? -1 : 1;
    if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    if (x->l != y->l) return x->l < y->l ? -1 : 1;
    return 0;
}

/* Run both strands at one budget; returns the number of candidates. */
static int search_pass(ctx_t c[2], int budget)
{
    for (int s = 0; s < 2; s++) {
        c[s].budget = budget;
        c[s].n_cand = 0;
        c[s].lookups = 0;
        dfs(&c[s], 0, 0, c[s].I->n, 0, 0, 0, 0, 0, 0, OP_M);
    }
    return c[0].n_cand + c[1].n_cand;
}

/*
 * Score-ordered mode (the variant BWA and BarraCUDA ship: hits ranked by a
 * mismatch / gap-open / gap-extension penalty rather than by difference count).
 * The hits are every hit within the difference limit z (as in FULL), each with
 * its least witness by (score, diffs, gap opens, gap extensions, mismatches,
 * length).  S1 = the least score, S2 = the least score above it; c0 / c1 = the
 * summed widths of the hits scoring S1 / S2; the hits scoring S1 or S2 are
 * listed in the order (score, strand, k, l), only those scoring S1 when more
 * than max_best places score S1 (> 0; flag F_MANY_BEST).  d_best = the fewest
 * differences among the S1 hits; the result's spare byte holds S1 (at most 254).
 */
static void score_strata(const orc_params *p, orc_hit *all, int nc, orc_res *res, orc_hit *hits)
{
    int s1 = -1, s2 = -1;
    for (int i = 0; i < nc; i++) {
        int sc = score_of(p, &all[i]);
        if (s1 < 0 || sc < s1) s1 = sc;
    }
    for (int i = 0; i < nc; i++) {
        int sc = score_of(p, &all[i]);
        if (sc > s1 && (s2 < 0 || sc < s2)) s2 = sc;
    }
    uint64_t c0 = 0, c1 = 0;
    int d_best = 255;
    for (int i = 0; i < nc; i++) {
        int sc = score_of(p, &all[i]);
        uint64_t wdt = (uint64_t)all[i].l - all[i].k + 1;
        if (sc == s1) {
            c0 += wdt;
            if (all[i].n_diff < d_best) d_best = all[i].n_diff;
        } else if (sc == s2) {
            c1 += wdt;
        }
    }
    int many = p->max_best > 0 && c0 > (uint64_t)p->max_best;
    int nk = 0;
    for (int i = 0; i < nc; i++) {
        int sc = score_of(p, &all[i]);
        if (sc == s1 || (!many && sc == s2)) all[nk++] = all[i];
    }
    /* order (score, strand, k, l): insertion sort */
    for (int i = 1; i < nk; i++) {
        orc_hit h = all[i];
        int sh = score_of(p, &h), j = i;
        while (j > 0) {
            const orc_hit *o = &all[j - 1];
            int so = score_of(p, o);
            int after = so > sh || (so == sh && (o->strand > h.strand || (o->strand == h.strand &&
                        (o->k > h.k || (o->k == h.k && o->l > h.l)))));
            if (!after) break;
            all[j] = all[j - 1];
            j--;
        }
        all[j] = h;
    }
    int out = nk < p->hit_cap ? nk : p->hit_cap;
    if (nk > p->hit_cap) res->flags |= F_HIT_OVERFLOW;
    if (many) res->flags |= F_MANY_BEST;
    memcpy(hits, all, out * sizeof(orc_hit));
    res->n_hits = (uint8_t)out;
    res->d_best = (uint8_t)d_best;
    res->pad = (uint8_t)(s1 > 254 ? 254 : s1);
    res->c0 = c0 > 0xFFFFFFFFULL ? 0xFFFFFFFFu : (uint32_t)c0;
    res->c1 = c1 > 0xFFFFFFFFULL ? 0xFFFFFFFFu : (uint32_t)c1;
}

/* Align one read; writes res and up to hit_cap hits; returns canonical lookups. */
static uint64_t align_one(const orc_index *ix, const uint8_t *w, int m, int z, const orc_params *p,
                          orc_res *res, orc_hit *hits, ctx_t c[2])
{
    memset(res, 0, sizeof *res);
    res->d_best = 255;
    if (p->strata == STRATA_SCORE) res->pad = 255; /* the best score, 255 while there is no hit */
    if (m > READ_MAX) { res->flags |= F_READ_TOO_LONG; return 0; }
    if (z > Z_MAX) { res->flags |= F_BAD_LIMIT; return 0; }
    uint64_t look = 0;
    for (int s = 0; s < 2; s++) {
        c[s].p = p;
        c[s].ix = ix;
        setup_strand(&c[s], ix, w, m, s);
        const otext *other = &ix->t[s ? 1 : 0];
        look += dscan(other, c[s].q, m, c[s].D);
        if (!p->use_d) for (int i = 0; i <= m; i++) c[s].D[i] = 0;
    }
    int final_budget = -1;
    if (p->strata == 1 || p->strata == STRATA_SCORE) {
        final_budget = z;
        search_pass(c, z);
    } else {
        /* BEST1: iterative deepening 0, 1, ... to the first budget with a hit
         * (= d_best), then one pass at min(z, d_best + 1). */
        for (int b = 0; b <= z; b++) {
            if (search_pass(c, b) > 0) {
                final_budget = b + 1 <= z ? b + 1 : z;
                if (final_budget != b) search_pass(c, final_budget);
                break;
            }
        }
        if (final_budget < 0) final_budget = z; /* no hit: the tree at budget z was the last */
    }
    look += c[0].lookups + c[1].lookups;
    int nc = c[0].n_cand + c[1].n_cand;
    if (nc == 0) return look;
    orc_hit *all = (orc_hit *)malloc(nc * sizeof(orc_hit));
    memcpy(all, c[0].cand, c[0].n_cand * sizeof(orc_hit));
    memcpy(all + c[0].n_cand, c[1].cand, c[1].n_cand * sizeof(orc_hit));
    if (p->strata == STRATA_SCORE) {
        score_strata(p, all, nc, res, hits);
        free(all);
        return look;
    }
    int d_best = 255;
    for (int i = 0; i < nc; i++) if (all[i].n_diff < d_best) d_best = all[i].n_diff;
    int keep_max = (p->strata == 1) ? z : (d_best + 1 <= z ? d_best + 1 : z);
    int nk = 0;
    uint64_t c0 = 0, c1 = 0;
    for (int i = 0; i < nc; i++) {
        if (all[i].n_diff > keep_max) continue;
        uint64_t wdt = (uint64_t)all[i].l - all[i].k + 1;
        if (all[i].n_diff == d_best) c0 += wdt;
        else if (all[i].n_diff == d_best + 1) c1 += wdt;
        all[nk++] = all[i];
    }
    qsort(all, nk, sizeof(orc_hit), cand_order);
    int out = nk < p->hit_cap ? nk : p->hit_cap;
    if (nk > p->hit_cap) res->flags |= F_HIT_OVERFLOW;
    memcpy(hits, all, out * sizeof(orc_hit));
    res->n_hits = (uint8_t)out;
    res->d_best = (uint8_t)d_best;
    res->c0 = c0 > 0xFFFFFFFFULL ? 0xFFFFFFFFu : (uint32_t)c0;
    res->c1 = c1 > 0xFFFFFFFFULL ? 0xFFFFFFFFu : (uint32_t)c1;
    free(all);
    return look;
}

typedef struct {
    const orc_index *ix;
    const uint8_t *codes;
    const uint64_t *off;
    const uint16_t *len;
    const uint8_t *z;
    const orc_params *p;
    orc_res *res;
    orc_hit *hits;
    uint64_t *lookups;
    uint64_t next, n;
    pthread_mutex_t *mu;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *b = (batch_job *)arg;
    ctx_t c[2];
    memset(c, 0, sizeof c);
    for (;;) {
        pthread_mutex_lock(b->mu);
        uint64_t r = b->next;
        uint64_t hi = r + 16 < b->n ? r + 16 : b->n;
        b->next = hi;
        pthread_mutex_unlock(b->mu);
        if (r >= b->n) break;
        for (; r < hi; r++) {
            int z = b->z ? b->z[r] : b->p->z;
            uint64_t lk = align_one(b->ix, b->codes + b->off[r], b->len[r], z, b->p,
                                    &b->res[r], b->hits + r * (uint64_t)b->p->hit_cap, c);
            if (b->lookups) b->lookups[r] = lk;
        }
    }
    free(c[0].cand);
    free(c[1].cand);
    return NULL;
}

/* Align a batch of reads with nthreads host threads.  Reads are codes 0..4,
 * read r at codes[off[r] .. off[r]+len[r]-1]; z may be NULL (p->z for all).
 * hits has room for n * hit_cap records; lookups (may be NULL) gets the
 * canonical Occ-lookup count per read. */
int orc_align(const orc_index *ix, const uint8_t *codes, const uint64_t *off, const uint16_t *len,
              const uint8_t *z, uint64_t n, const orc_params *p, int nthreads,
              orc_res *res, orc_hit *hits, uint64_t *lookups)
{
    if (!ix || !p || p->hit_cap < 0 || p->hit_cap > 255) return -1;
    pthread_mutex_t mu;
    pthread_mutex_init(&mu, NULL);
    batch_job job = {ix, codes, off, len, z, p, res, hits, lookups, 0, n, &mu};
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(nthreads * sizeof(pthread_t));
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, batch_worker, &job);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&mu);
    return 0;
}

/* D array of one read on one strand (for tests). */
int orc_dscan(const orc_index *ix, int strand, const uint8_t *w, int m, int *D)
{
    ctx_t c;
    memset(&c, 0, sizeof c);
    if (m > READ_MAX) return -1;
    setup_strand(&c, ix, w, m, strand);
    dscan(&ix->t[strand ? 1 : 0], c.q, m, D);
    return 0;
}

static int u64_cmp(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y);
}

/* Forward-strand 0-based start of the target for every row of a hit of width
 * <= max_width, from the full suffix arrays: strand 0 -> n - SA_Xr[j] - len,
 * strand 1 -> SA_X[j].  Positions of one hit are sorted ascending and written
 * at pos[hit_i * max_width ...]; npos[hit_i] = count (0 if the hit is wider). */
int orc_positions(const orc_index *ix, const orc_hit *h, uint64_t nh, uint32_t max_width,
                  uint64_t *pos, uint32_t *npos)
{
    uint64_t n = ix->t[0].n;
    for (uint64_t i = 0; i < nh; i++) {
        uint64_t w = (uint64_t)h[i].l - h[i].k + 1;
        npos[i] = 0;
        if (h[i].l < h[i].k || w > max_width) continue;
        uint64_t *o = pos + i * max_width;
        for (uint64_t j = 0; j < w; j++) {
            uint64_t row = h[i].k + j;
            o[j] = h[i].strand ? ix->t[0].sa[row] : n - ix->t[1].sa[row] - h[i].aligned_len;
        }
        qsort(o, w, sizeof(uint64_t), u64_cmp);
        npos[i] = (uint32_t)w;
    }
    return 0;
}

/* ------------------------------------------------------------ pairing
 *
 * Paired reads after the search (the pipeline's pairing stage, Sec. 2 and the
 * pipeline of Sec. 3: mate hits are combined using the fragment length).  Read
 * 2p is mate 1 and read 2p+1 mate 2 of pair p.  The paper gives no rule; the
 * one restated here (the project's reading, written out in the design notes):
 *  - placements of a mate: every position of every hit in its best stratum
 *    (n_diff == d_best), each with the hit's strand, target length and n_diff.
 *    A mate is placed iff 1 <= c0 <= max_place (c0 = its number of best
 *    placements) and all of its best hits were written;
 *  - a combination (one placement of each mate) is FR if the strands differ;
 *    with f the forward and v the reverse placement, its insert is
 *    v.pos + v.len - f.pos (may be <= 0);
 *  - insert-size window: over the pairs whose mates both have c0 == 1 and whose
 *    single combination is FR with 1 <= insert <= 65535 (the unique pairs), the
 *    sorted inserts s[0..u-1] give q1 = s[u/4], q2 = s[u/2], q3 = s[3u/4]
 *    (integer division) and the window [max(1, q1 - 2 (q3 - q1)),
 *    min(65535, q3 + 2 (q3 - q1))]; with fewer than 8 unique pairs the window is
 *    [1, 65535] and q1 = q2 = q3 = 0;
 *  - a combination is proper if FR with its insert inside the window; the pair's
 *    choice is the proper combination smallest by (n_diff1 + n_diff2,
 *    |insert - q2|, insert, pos1, pos2, strand1, len1, len2);
 *  - flags: 1, 2 mate 1 / 2 has a hit; 4, 8 mate 1 / 2 is placed; 16 unique
 *    pair; 32 proper (a choice exists); 64 discordant (both placed, no proper
 *    combination).
 */
#define OP_MAPPED1 0x01
#define OP_MAPPED2 0x02
#define OP_PLACED1 0x04
#define OP_PLACED2 0x08
#define OP_UNIQUE 0x10
#define OP_PROPER 0x20
#define OP_DISCORDANT 0x40
#define ISIZE_MAX 65535

typedef struct {
    uint64_t pos[2];
    uint32_t insert;
    uint16_t n_proper;
    uint8_t strand[2];
    uint8_t flags;
    uint8_t pad[3];
    uint32_t pad2;
} orc_pair;

typedef struct {
    uint32_t n_unique, q1, q2, q3, lo, hi, pad[2];
} orc_pair_stats;

typedef struct { uint64_t pos; uint32_t len; uint8_t strand, n_diff; } placement;

/* Placements of one read (its best stratum), from the full suffix arrays. */
static int placements_of(const orc_index *ix, const orc_res *r, const orc_hit *h, int max_place, placement *out)
{
    if (r->n_hits == 0 || r->c0 < 1 || r->c0 > (uint32_t)max_place) return -1;
    uint64_t n = ix->t[0].n;
    int k = 0;
    for (int j = 0; j < r->n_hits; j++) {
        if (h[j].n_diff != r->d_best) continue;
        for (uint64_t row = h[j].k; row <= h[j].l; row++) {
            if (k == max_place) return -1;
            out[k].pos = h[j].strand ? ix->t[0].sa[row] : n - ix->t[1].sa[row] - h[j].aligned_len;
            out[k].len = h[j].aligned_len;
            out[k].strand = h[j].strand;
            out[k].n_diff = h[j].n_diff;
            k++;
        }
    }
    return (uint32_t)k == r->c0 ? k : -1;  /* every best placement was written */
}

/* Insert of a combination (0 and FR flag clear if the strands are equal). */
static int64_t insert_of(const placement *a, const placement *b, int *fr)
{
    *fr = a->strand != b->strand;
    if (!*fr) return 0;
    const placement *f = a->strand == 0 ? a : b, *v = a->strand == 0 ? b : a;
    return (int64_t)v->pos + (int64_t)v->len - (int64_t)f->pos;
}

static int u32_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y);
}

int orc_pair_resolve(const orc_index *ix, const orc_res *res, const orc_hit *hits, uint32_t hit_cap,
                     uint64_t n_pairs, int max_place, orc_pair *out, orc_pair_stats *st)
{
    if (!ix || max_place < 1 || max_place > 64) return -1;
    placement *pa = (placement *)malloc(max_place * sizeof(placement));
    placement *pb = (placement *)malloc(max_place * sizeof(placement));
    uint32_t *ins = (uint32_t *)malloc((n_pairs ? n_pairs : 1) * sizeof(uint32_t));
    if (!pa || !pb || !ins) return -1;
    /* unique pairs -> insert-size window */
    uint64_t u = 0;
    for (uint64_t p = 0; p < n_pairs; p++) {
        const orc_res *r1 = &res[2 * p], *r2 = &res[2 * p + 1];
        if (r1->c0 != 1 || r2->c0 != 1) continue;
        int na = placements_of(ix, r1, hits + 2 * p * hit_cap, max_place, pa);
        int nb = placements_of(ix, r2, hits + (2 * p + 1) * hit_cap, max_place, pb);
        if (na != 1 || nb != 1) continue;
        int fr;
        int64_t x = insert_of(&pa[0], &pb[0], &fr);
        if (fr && x >= 1 && x <= ISIZE_MAX) ins[u++] = (uint32_t)x;
    }
    memset(st, 0, sizeof *st);
    st->n_unique = (uint32_t)u;
    st->lo = 1;
    st->hi = ISIZE_MAX;
    if (u >= 8) {
        qsort(ins, u, sizeof(uint32_t), u32_cmp);
        st->q1 = ins[u / 4];
        st->q2 = ins[u / 2];
        st->q3 = ins[(3 * u) / 4];
        int64_t iqr = (int64_t)st->q3 - st->q1;
        int64_t lo = (int64_t)st->q1 - 2 * iqr, hi = (int64_t)st->q3 + 2 * iqr;
        st->lo = (uint32_t)(lo < 1 ? 1 : lo);
        st->hi = (uint32_t)(hi > ISIZE_MAX ? ISIZE_MAX : hi);
    }
    /* each pair: proper combinations and the choice */
    for (uint64_t p = 0; p < n_pairs; p++) {
        const orc_res *r1 = &res[2 * p], *r2 = &res[2 * p + 1];
        orc_pair *o = &out[p];
        memset(o, 0, sizeof *o);
        o->pos[0] = o->pos[1] = UINT64_MAX;
        o->strand[0] = o->strand[1] = 255;
        if (r1->n_hits) o->flags |= OP_MAPPED1;
        if (r2->n_hits) o->flags |= OP_MAPPED2;
        int na = placements_of(ix, r1, hits + 2 * p * hit_cap, max_place, pa);
        int nb = placements_of(ix, r2, hits + (2 * p + 1) * hit_cap, max_place, pb);
        if (na > 0) o->flags |= OP_PLACED1;
        if (nb > 0) o->flags |= OP_PLACED2;
        if (na <= 0 || nb <= 0) continue;
        if (na == 1 && nb == 1) {
            int fr;
            int64_t x = insert_of(&pa[0], &pb[0], &fr);
            if (fr && x >= 1 && x <= ISIZE_MAX) o->flags |= OP_UNIQUE;
        }
        uint32_t nproper = 0;
        int best_i = -1, best_j = -1;
        int64_t best_x = 0;
        for (int i = 0; i < na; i++) {
            for (int j = 0; j < nb; j++) {
                int fr;
                int64_t x = insert_of(&pa[i], &pb[j], &fr);
                if (!fr || x < (int64_t)st->lo || x > (int64_t)st->hi) continue;
                nproper++;
                int better = best_i < 0;
                if (!better) {
                    int d = pa[i].n_diff + pb[j].n_diff, db = pa[best_i].n_diff + pb[best_j].n_diff;
                    int64_t e = x > st->q2 ? x - st->q2 : st->q2 - x;
                    int64_t eb = best_x > st->q2 ? best_x - st->q2 : st->q2 - best_x;
                    if (d != db) better = d < db;
                    else if (e != eb) better = e < eb;
                    else if (x != best_x) better = x < best_x;
                    else if (pa[i].pos != pa[best_i].pos) better = pa[i].pos < pa[best_i].pos;
                    else if (pb[j].pos != pb[best_j].pos) better = pb[j].pos < pb[best_j].pos;
                    else if (pa[i].strand != pa[best_i].strand) better = pa[i].strand < pa[best_i].strand;
                    else if (pa[i].len != pa[best_i].len) better = pa[i].len < pa[best_i].len;
                    else better = pb[j].len < pb[best_j].len;
                }
                if (better) {
                    best_i = i;
                    best_j = j;
                    best_x = x;
                }
            }
        }
        o->n_proper = (uint16_t)(nproper > 65535 ? 65535 : nproper);
        if (best_i >= 0) {
            o->flags |= OP_PROPER;
            o->pos[0] = pa[best_i].pos;
            o->pos[1] = pb[best_j].pos;
            o->strand[0] = pa[best_i].strand;
            o->strand[1] = pb[best_j].strand;
            o->insert = (uint32_t)best_x;
        } else {
            o->flags |= OP_DISCORDANT;
        }
    }
    free(pa);
    free(pb);
    free(ins);
    return 0;
}
