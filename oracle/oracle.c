/*
 * Plain, slow, obviously-correct CPU oracle for the relational operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path.
 *
 * The paper expresses every relational operator as a tensor program and
 * defers the operator algorithms to its predecessor (Sec. 2, "Query
 * Processor"); the results it relies on are plain SQL results, so each
 * function below is the SQL definition written out:
 *
 *   filter   -- WHERE with a conjunction of comparisons (Sec. 5.2 query):
 *               scan the rows in order, keep those where every predicate holds.
 *   group-by -- GROUP BY ... COUNT(*) (Sec. 2 example, Sec. 4 trainable query)
 *               with SUM / AVG aggregates (Sec. 5.2): order the selected rows
 *               by (key tuple, row id) with a library sort, then walk the runs.
 *               Groups come out in ascending key order.  AVG is rounded half
 *               away from zero in the column's own fixed-point scale.
 *   join     -- inner equi-join: for every probe row in probe order, every
 *               build row with an equal key in build-row order (sort the build
 *               side, binary-search each probe key).
 *   top-k    -- order all groups by (value descending, key ascending) with a
 *               library sort and keep the first k.
 *   sort     -- stable ordering of (key, value) pairs by key (library sort on
 *               (key, original position)).
 *
 * All arithmetic is exact int64.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_I8 = 0, ORC_I32 = 1, ORC_I64 = 2, ORC_U8 = 3 };
enum { ORC_LT = 0, ORC_LE, ORC_GT, ORC_GE, ORC_EQ, ORC_NE };
enum { ORC_COUNT = 0, ORC_SUM, ORC_SUM_MUL_KMINUS, ORC_AVG, ORC_MIN, ORC_MAX };

static int64_t get(const void *p, int dt, int64_t i)
{
    switch (dt) {
    case ORC_I8: return ((const int8_t *)p)[i];
    case ORC_U8: return ((const uint8_t *)p)[i];
    case ORC_I32: return ((const int32_t *)p)[i];
    default: return ((const int64_t *)p)[i];
    }
}

static int holds(int64_t v, int cmp, int64_t lit)
{
    switch (cmp) {
    case ORC_LT: return v < lit;
    case ORC_LE: return v <= lit;
    case ORC_GT: return v > lit;
    case ORC_GE: return v >= lit;
    case ORC_EQ: return v == lit;
    default: return v != lit;
    }
}

/* WHERE p_0 AND p_1 AND ...: row ids of qualifying rows, ascending. */
int64_t orc_filter(int64_t n, int npred, const void **cols, const int *dts,
                   const int *cmps, const int64_t *lits, int32_t *out_rowid)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        int ok = 1;
        for (int p = 0; p < npred && ok; p++)
            ok = holds(get(cols[p], dts[p], i), cmps[p], lits[p]);
        if (ok)
            out_rowid[m++] = (int32_t)i;
    }
    return m;
}

/* ---------------------------------------------------------------- group-by */

struct key_ctx {
    int nkeys;
    const void **cols;
    const int *dts;
};

static int cmp_rows_by_key(const void *pa, const void *pb, void *vctx)
{
    const struct key_ctx *c = (const struct key_ctx *)vctx;
    int64_t ra = *(const int64_t *)pa, rb = *(const int64_t *)pb;
    for (int k = 0; k < c->nkeys; k++) {
        int64_t a = get(c->cols[k], c->dts[k], ra), b = get(c->cols[k], c->dts[k], rb);
        if (a != b)
            return a < b ? -1 : 1;
    }
    return ra < rb ? -1 : (ra > rb ? 1 : 0);
}

/* Round-half-away-from-zero quotient s / c for c > 0. */
int64_t orc_avg_round(int64_t s, int64_t c)
{
    int64_t sg = s > 0 ? 1 : (s < 0 ? -1 : 0);
    return (2 * s + sg * c) / (2 * c);
}

/*
 * GROUP BY key columns over the selected rows (sel == NULL: all n rows).
 * Aggregate j: ops[j] over column a[j] (and b[j], k[j] for SUM(a*(k-b))).
 * Writes up to cap groups: out_keys[g*nkeys + k], out_aggs[g*naggs + j].
 * Returns the number of groups.
 */
int64_t orc_groupby(int64_t n, const int32_t *sel, int64_t nsel,
                    int nkeys, const void **keycols, const int *keydts,
                    int naggs, const int *ops, const void **acols, const int *adts,
                    const void **bcols, const int *bdts, const int64_t *ks,
                    int64_t *out_keys, int64_t *out_aggs, int64_t cap)
{
    int64_t m = sel ? nsel : n;
    int64_t *rows = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < m; i++)
        rows[i] = sel ? sel[i] : i;
    struct key_ctx ctx = { nkeys, keycols, keydts };
    qsort_r(rows, (size_t)m, sizeof(int64_t), cmp_rows_by_key, &ctx);

    int64_t ng = 0;
    int64_t i = 0;
    while (i < m) {
        int64_t j = i;
        while (j < m) {
            int same = 1;
            for (int k = 0; k < nkeys && same; k++)
                same = get(keycols[k], keydts[k], rows[j]) == get(keycols[k], keydts[k], rows[i]);
            if (!same)
                break;
            j++;
        }
        /* rows[i..j) is one group */
        if (ng < cap) {
            for (int k = 0; k < nkeys; k++)
                out_keys[ng * nkeys + k] = get(keycols[k], keydts[k], rows[i]);
            for (int a = 0; a < naggs; a++) {
                int64_t acc = 0, cnt = j - i;
                for (int64_t r = i; r < j; r++) {
                    int64_t x = ops[a] == ORC_COUNT ? 1 : get(acols[a], adts[a], rows[r]);
                    if (ops[a] == ORC_SUM_MUL_KMINUS)
                        x = x * (ks[a] - get(bcols[a], bdts[a], rows[r]));
                    if (ops[a] == ORC_MIN)
                        acc = (r == i || x < acc) ? x : acc;
                    else if (ops[a] == ORC_MAX)
                        acc = (r == i || x > acc) ? x : acc;
                    else
                        acc += x;
                }
                if (ops[a] == ORC_AVG)
                    acc = orc_avg_round(acc, cnt);
                out_aggs[ng * naggs + a] = acc;
            }
        }
        ng++;
        i = j;
    }
    free(rows);
    return ng;
}

/* -------------------------------------------------------------------- join */

static int cmp_build(const void *pa, const void *pb, void *vkeys)
{
    const int32_t *keys = (const int32_t *)vkeys;
    int64_t ra = *(const int64_t *)pa, rb = *(const int64_t *)pb;
    if (keys[ra] != keys[rb])
        return keys[ra] < keys[rb] ? -1 : 1;
    return ra < rb ? -1 : (ra > rb ? 1 : 0);
}

/*
 * Inner equi-join.  Build rows: bsel (NULL: all nb rows); probe rows: psel
 * (NULL: all np rows), visited in that order.  For each match writes the
 * probe row id and the build row id.  *dup is set when two selected build
 * rows share a key.  Returns the number of matches (writes at most cap).
 */
int64_t orc_join(int64_t nb, const int32_t *bkey, const int32_t *bsel, int64_t nbsel,
                 int64_t np, const int32_t *pkey, const int32_t *psel, int64_t npsel,
                 int32_t *out_probe, int32_t *out_build, int64_t cap, int *dup)
{
    int64_t mb = bsel ? nbsel : nb;
    int64_t *b = (int64_t *)malloc((size_t)(mb > 0 ? mb : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < mb; i++)
        b[i] = bsel ? bsel[i] : i;
    qsort_r(b, (size_t)mb, sizeof(int64_t), cmp_build, (void *)bkey);
    *dup = 0;
    for (int64_t i = 1; i < mb; i++)
        if (bkey[b[i]] == bkey[b[i - 1]])
            *dup = 1;

    int64_t mp = psel ? npsel : np;
    int64_t out = 0;
    for (int64_t q = 0; q < mp; q++) {
        int64_t pr = psel ? psel[q] : q;
        int32_t k = pkey[pr];
        int64_t lo = 0, hi = mb; /* first index with bkey >= k */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (bkey[b[mid]] < k)
                lo = mid + 1;
            else
                hi = mid;
        }
        for (int64_t t = lo; t < mb && bkey[b[t]] == k; t++) {
            if (out < cap) {
                out_probe[out] = (int32_t)pr;
                out_build[out] = (int32_t)b[t];
            }
            out++;
        }
    }
    free(b);
    return out;
}

/* ------------------------------------------------------------------- top-k */

struct topk_ctx {
    const int64_t *vals;
    const int64_t *keys;
};

static int cmp_topk(const void *pa, const void *pb, void *vctx)
{
    const struct topk_ctx *c = (const struct topk_ctx *)vctx;
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (c->vals[a] != c->vals[b])
        return c->vals[a] > c->vals[b] ? -1 : 1;
    if (c->keys[a] != c->keys[b])
        return c->keys[a] < c->keys[b] ? -1 : 1;
    return 0;
}

/* The first k of all n (value, key) rows ordered by value desc, key asc. */
int64_t orc_topk(int64_t n, const int64_t *vals, const int64_t *keys, int64_t k,
                 int64_t *out_vals, int64_t *out_keys)
{
    int64_t *idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++)
        idx[i] = i;
    struct topk_ctx ctx = { vals, keys };
    qsort_r(idx, (size_t)n, sizeof(int64_t), cmp_topk, &ctx);
    int64_t m = n < k ? n : k;
    for (int64_t i = 0; i < m; i++) {
        out_vals[i] = vals[idx[i]];
        out_keys[i] = keys[idx[i]];
    }
    free(idx);
    return m;
}

/* -------------------------------------------------------------------- sort */

static int cmp_pairs(const void *pa, const void *pb, void *vkeys)
{
    const uint64_t *keys = (const uint64_t *)vkeys;
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (keys[a] != keys[b])
        return keys[a] < keys[b] ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Stable sort of (key, value) pairs by unsigned key. */
void orc_sort_pairs(int64_t n, const uint64_t *keys, const uint32_t *vals,
                    uint64_t *out_keys, uint32_t *out_vals)
{
    int64_t *idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++)
        idx[i] = i;
    qsort_r(idx, (size_t)n, sizeof(int64_t), cmp_pairs, (void *)keys);
    for (int64_t i = 0; i < n; i++) {
        out_keys[i] = keys[idx[i]];
        out_vals[i] = vals[idx[i]];
    }
    free(idx);
}

/* ------------------------------------------------- OpenMP variants (timing) */
/*
 * Row-partitioned versions of filter, join and group-by for the timed CPU
 * baseline on all host cores.  Each gives exactly the result of its
 * single-threaded counterpart above (pinned by the tests):
 *   filter   -- every thread scans a contiguous block of rows; the blocks'
 *               counts give each block its output offset, so the row ids
 *               stay in ascending order.
 *   join     -- the build side is sorted once (single thread); probe rows
 *               are split into contiguous blocks, each counted, then written
 *               at its offset: probe order, build-row order within a key.
 *   group-by -- every thread sorts its block of selected rows by key and
 *               reduces the runs to partial groups; the sorted partial lists
 *               are merged by key (sums and counts added, minima / maxima
 *               combined, AVG rounded from the merged sum and count).
 */
#include <omp.h>

int orc_omp_threads(void) { return omp_get_max_threads(); }

int64_t orc_filter_omp(int64_t n, int npred, const void **cols, const int *dts,
                       const int *cmps, const int64_t *lits, int32_t *out_rowid)
{
    int T = omp_get_max_threads();
    int64_t *cnt = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
#pragma omp parallel num_threads(T)
    {
        int t = omp_get_thread_num();
        int64_t lo = n * t / T, hi = n * (t + 1) / T, c = 0;
        for (int64_t i = lo; i < hi; i++) {
            int ok = 1;
            for (int p = 0; p < npred && ok; p++)
                ok = holds(get(cols[p], dts[p], i), cmps[p], lits[p]);
            c += ok;
        }
        cnt[t + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int k = 0; k < T; k++)
            cnt[k + 1] += cnt[k];
        int64_t o = cnt[t];
        for (int64_t i = lo; i < hi; i++) {
            int ok = 1;
            for (int p = 0; p < npred && ok; p++)
                ok = holds(get(cols[p], dts[p], i), cmps[p], lits[p]);
            if (ok)
                out_rowid[o++] = (int32_t)i;
        }
    }
    int64_t m = cnt[T];
    free(cnt);
    return m;
}

static int64_t first_ge(const int32_t *bkey, const int64_t *b, int64_t mb, int32_t k)
{
    int64_t lo = 0, hi = mb;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (bkey[b[mid]] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

int64_t orc_join_omp(int64_t nb, const int32_t *bkey, const int32_t *bsel, int64_t nbsel,
                     int64_t np, const int32_t *pkey, const int32_t *psel, int64_t npsel,
                     int32_t *out_probe, int32_t *out_build, int64_t cap, int *dup)
{
    int64_t mb = bsel ? nbsel : nb;
    int64_t *b = (int64_t *)malloc((size_t)(mb > 0 ? mb : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < mb; i++)
        b[i] = bsel ? bsel[i] : i;
    qsort_r(b, (size_t)mb, sizeof(int64_t), cmp_build, (void *)bkey);
    *dup = 0;
    for (int64_t i = 1; i < mb; i++)
        if (bkey[b[i]] == bkey[b[i - 1]])
            *dup = 1;
    int64_t mp = psel ? npsel : np;
    int T = omp_get_max_threads();
    int64_t *cnt = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
#pragma omp parallel num_threads(T)
    {
        int t = omp_get_thread_num();
        int64_t lo = mp * t / T, hi = mp * (t + 1) / T, c = 0;
        for (int64_t q = lo; q < hi; q++) {
            int32_t k = pkey[psel ? psel[q] : q];
            for (int64_t u = first_ge(bkey, b, mb, k); u < mb && bkey[b[u]] == k; u++)
                c++;
        }
        cnt[t + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int k = 0; k < T; k++)
            cnt[k + 1] += cnt[k];
        int64_t o = cnt[t];
        for (int64_t q = lo; q < hi; q++) {
            int64_t pr = psel ? psel[q] : q;
            int32_t k = pkey[pr];
            for (int64_t u = first_ge(bkey, b, mb, k); u < mb && bkey[b[u]] == k; u++, o++)
                if (o < cap) {
                    out_probe[o] = (int32_t)pr;
                    out_build[o] = (int32_t)b[u];
                }
        }
    }
    int64_t m = cnt[T];
    free(cnt);
    free(b);
    return m;
}

/* One partial group: its key tuple (row of the first member), and for every
 * aggregate the running value and the member count. */
struct part {
    int64_t row;
    int64_t cnt;
    int64_t acc[16];
};

static int same_key(const struct key_ctx *c, int64_t ra, int64_t rb)
{
    for (int k = 0; k < c->nkeys; k++)
        if (get(c->cols[k], c->dts[k], ra) != get(c->cols[k], c->dts[k], rb))
            return 0;
    return 1;
}

static int key_cmp(const struct key_ctx *c, int64_t ra, int64_t rb)
{
    for (int k = 0; k < c->nkeys; k++) {
        int64_t a = get(c->cols[k], c->dts[k], ra), b = get(c->cols[k], c->dts[k], rb);
        if (a != b)
            return a < b ? -1 : 1;
    }
    return 0;
}

int64_t orc_groupby_omp(int64_t n, const int32_t *sel, int64_t nsel,
                        int nkeys, const void **keycols, const int *keydts,
                        int naggs, const int *ops, const void **acols, const int *adts,
                        const void **bcols, const int *bdts, const int64_t *ks,
                        int64_t *out_keys, int64_t *out_aggs, int64_t cap)
{
    if (naggs > 16)
        return -1;
    int64_t m = sel ? nsel : n;
    struct key_ctx ctx = { nkeys, keycols, keydts };
    int T = omp_get_max_threads();
    struct part **parts = (struct part **)calloc((size_t)T, sizeof(struct part *));
    int64_t *np = (int64_t *)calloc((size_t)T, sizeof(int64_t));
#pragma omp parallel num_threads(T)
    {
        int t = omp_get_thread_num();
        int64_t lo = m * t / T, hi = m * (t + 1) / T, len = hi - lo;
        int64_t *rows = (int64_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int64_t));
        for (int64_t i = 0; i < len; i++)
            rows[i] = sel ? sel[lo + i] : lo + i;
        qsort_r(rows, (size_t)len, sizeof(int64_t), cmp_rows_by_key, &ctx);
        struct part *p = (struct part *)malloc((size_t)(len > 0 ? len : 1) * sizeof(struct part));
        int64_t g = -1;
        for (int64_t i = 0; i < len; i++) {
            int64_t r = rows[i];
            if (g < 0 || !same_key(&ctx, p[g].row, r)) {
                g++;
                p[g].row = r;
                p[g].cnt = 0;
            }
            for (int a = 0; a < naggs; a++) {
                int64_t x = ops[a] == ORC_COUNT ? 1 : get(acols[a], adts[a], r);
                if (ops[a] == ORC_SUM_MUL_KMINUS)
                    x = x * (ks[a] - get(bcols[a], bdts[a], r));
                if (p[g].cnt == 0)
                    p[g].acc[a] = x;
                else if (ops[a] == ORC_MIN)
                    p[g].acc[a] = x < p[g].acc[a] ? x : p[g].acc[a];
                else if (ops[a] == ORC_MAX)
                    p[g].acc[a] = x > p[g].acc[a] ? x : p[g].acc[a];
                else
                    p[g].acc[a] += x;
            }
            p[g].cnt++;
        }
        parts[t] = p;
        np[t] = g + 1;
        free(rows);
    }
    /* merge the sorted partial lists by key */
    int64_t *pos = (int64_t *)calloc((size_t)T, sizeof(int64_t));
    int64_t ng = 0;
    for (;;) {
        int best = -1;
        for (int t = 0; t < T; t++)
            if (pos[t] < np[t] && (best < 0 || key_cmp(&ctx, parts[t][pos[t]].row, parts[best][pos[best]].row) < 0))
                best = t;
        if (best < 0)
            break;
        struct part acc = parts[best][pos[best]];
        pos[best]++;
        for (int t = 0; t < T; t++)
            while (pos[t] < np[t] && same_key(&ctx, parts[t][pos[t]].row, acc.row)) {
                const struct part *q = &parts[t][pos[t]];
                for (int a = 0; a < naggs; a++) {
                    if (ops[a] == ORC_MIN)
                        acc.acc[a] = q->acc[a] < acc.acc[a] ? q->acc[a] : acc.acc[a];
                    else if (ops[a] == ORC_MAX)
                        acc.acc[a] = q->acc[a] > acc.acc[a] ? q->acc[a] : acc.acc[a];
                    else
                        acc.acc[a] += q->acc[a];
                }
                acc.cnt += q->cnt;
                pos[t]++;
            }
        if (ng < cap) {
            for (int k = 0; k < nkeys; k++)
                out_keys[ng * nkeys + k] = get(keycols[k], keydts[k], acc.row);
            for (int a = 0; a < naggs; a++)
                out_aggs[ng * naggs + a] = ops[a] == ORC_AVG ? orc_avg_round(acc.acc[a], acc.cnt) : acc.acc[a];
        }
        ng++;
    }
    for (int t = 0; t < T; t++)
        free(parts[t]);
    free(parts);
    free(np);
    free(pos);
    return ng;
}
