/*
 * CPU oracle for the sieved multi-way join -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  It shares no code, header or
 * constant table with the CUDA library and is deliberately plain and slow.
 *
 * What it computes is the plain definition of the join the method returns:
 * SieveJoin prunes with Bloom filters, which never drop a matching tuple
 * (Sec. 1, Sec. 2.1), and then runs an ordinary binary join plan over the pruned
 * relations (Sec. 2.2, enumeration phase), so the final COUNT / SUM / tuples are
 * those of the unpruned natural join.  This file holds
 *
 *   - a chained-bucket binary hash join level (pairs of matching rows, and the
 *     aggregate form used at the last level), whose probe can be split over
 *     threads (orc_set_threads) with the same results,
 *   - a nested-loop enumeration of a whole tree-shaped join (the brute force
 *     used on tiny inputs), and
 *   - the per-key (count, sum) message counting of chain queries over one
 *     relation pool, with dense messages (checks many served results).
 *
 * COUNT is kept in 128 bits so overflow of 2^63 can be reported (the chain
 * counting keeps it modulo 2^64); SUM is the
 * int64 sum taken modulo 2^64 (two's complement wrap), which is order-free.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Probe threads of the join levels (the build stays serial).  The probe rows
 * are split into equal contiguous slices, one per thread, and the slices'
 * results are put together in slice order, so every result is the same for
 * any thread count. */
static int g_threads = 1;
void orc_set_threads(int t) { g_threads = t < 1 ? 1 : (t > 256 ? 256 : t); }
int orc_get_threads(void) { return g_threads; }

typedef void (*slice_fn)(void *arg, int64_t lo, int64_t hi, int slice);
typedef struct { slice_fn fn; void *arg; int64_t lo, hi; int slice; } slice_job;
static void *slice_run(void *p) {
    slice_job *j = (slice_job *)p;
    j->fn(j->arg, j->lo, j->hi, j->slice);
    return NULL;
}
/* Run fn over [0, n) in `nt` slices; slice s covers [n s / nt, n (s+1) / nt). */
static void run_slices(slice_fn fn, void *arg, int64_t n, int nt) {
    if (nt <= 1) { fn(arg, 0, n, 0); return; }
    pthread_t th[256];
    slice_job jobs[256];
    int started[256];
    for (int s = 0; s < nt; ++s) {
        jobs[s].fn = fn; jobs[s].arg = arg; jobs[s].slice = s;
        jobs[s].lo = n * s / nt; jobs[s].hi = n * (s + 1) / nt;
        started[s] = pthread_create(&th[s], NULL, slice_run, &jobs[s]) == 0;
        if (!started[s]) slice_run(&jobs[s]);
    }
    for (int s = 0; s < nt; ++s)
        if (started[s]) pthread_join(th[s], NULL);
}

/* ---------------- chained hash table over an int32 key column ------------- */

typedef struct {
    int64_t *head;   /* bucket -> first row, -1 = none */
    int64_t *next;   /* row -> next row in the same bucket, -1 = end */
    uint64_t mask;
} chain_table;

static uint64_t bucket_of(int32_t key, uint64_t mask) {
    /* Knuth multiplicative hashing; any function works for a chained table. */
    uint64_t x = (uint64_t)(uint32_t)key * 11400714819323198485ull;
    return (x >> 29) & mask;
}

static int chain_build(chain_table *t, const int32_t *keys, int64_t n) {
    uint64_t nb = 1;
    while (nb < (uint64_t)(n > 0 ? n : 1)) nb <<= 1;
    t->mask = nb - 1;
    t->head = (int64_t *)malloc(nb * sizeof(int64_t));
    t->next = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!t->head || !t->next) { free(t->head); free(t->next); return -1; }
    for (uint64_t b = 0; b < nb; ++b) t->head[b] = -1;
    for (int64_t r = 0; r < n; ++r) {
        uint64_t b = bucket_of(keys[r], t->mask);
        t->next[r] = t->head[b];
        t->head[b] = r;
    }
    return 0;
}

static void chain_free(chain_table *t) { free(t->head); free(t->next); }

/* Number of (probe row, build row) pairs with equal keys in probe rows
 * [lo, hi). */
static int64_t count_range(const chain_table *t, const int32_t *pk, const int32_t *bk,
                           int64_t lo, int64_t hi) {
    int64_t total = 0;
    for (int64_t i = lo; i < hi; ++i)
        for (int64_t r = t->head[bucket_of(pk[i], t->mask)]; r >= 0; r = t->next[r])
            if (bk[r] == pk[i]) ++total;
    return total;
}

typedef struct {
    const chain_table *t;
    const int32_t *pk, *bk;
    const uint64_t *psum, *bval;
    int64_t *cnt;                 /* per slice */
    int64_t *out_probe, *out_build;
    const int64_t *off;           /* per slice: first output position */
    u128 *acnt;                   /* per slice */
    uint64_t *asum;               /* per slice */
} probe_job;

static void count_slice(void *p, int64_t lo, int64_t hi, int s) {
    probe_job *j = (probe_job *)p;
    j->cnt[s] = count_range(j->t, j->pk, j->bk, lo, hi);
}
static void fill_slice(void *p, int64_t lo, int64_t hi, int s) {
    probe_job *j = (probe_job *)p;
    int64_t o = j->off[s];
    for (int64_t i = lo; i < hi; ++i)
        for (int64_t r = j->t->head[bucket_of(j->pk[i], j->t->mask)]; r >= 0; r = j->t->next[r])
            if (j->bk[r] == j->pk[i]) { j->out_probe[o] = i; j->out_build[o] = r; ++o; }
}
static void agg_slice(void *p, int64_t lo, int64_t hi, int s) {
    probe_job *j = (probe_job *)p;
    u128 count = 0;
    uint64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i)
        for (int64_t r = j->t->head[bucket_of(j->pk[i], j->t->mask)]; r >= 0; r = j->t->next[r])
            if (j->bk[r] == j->pk[i]) {
                count += 1;
                sum += (j->psum ? j->psum[i] : 0) + (j->bval ? j->bval[r] : 0);
            }
    j->acnt[s] = count;
    j->asum[s] = sum;
}

/* Number of (probe row, build row) pairs with equal keys; -1 if out of memory. */
int64_t orc_join_pairs_count(const int32_t *pk, int64_t np, const int32_t *bk, int64_t nb) {
    chain_table t;
    if (chain_build(&t, bk, nb)) return -1;
    int64_t cnt[256];
    probe_job j = {&t, pk, bk, NULL, NULL, cnt, NULL, NULL, NULL, NULL, NULL};
    run_slices(count_slice, &j, np, g_threads);
    int64_t total = 0;
    for (int s = 0; s < g_threads; ++s) total += cnt[s];
    chain_free(&t);
    return total;
}

/* Fill the matching pairs, probe-row order; returns 0, or -1 if out of memory. */
int orc_join_pairs_fill(const int32_t *pk, int64_t np, const int32_t *bk, int64_t nb,
                        int64_t *out_probe, int64_t *out_build) {
    chain_table t;
    if (chain_build(&t, bk, nb)) return -1;
    int64_t cnt[256], off[256];
    probe_job j = {&t, pk, bk, NULL, NULL, cnt, out_probe, out_build, off, NULL, NULL};
    run_slices(count_slice, &j, np, g_threads);
    int64_t o = 0;
    for (int s = 0; s < g_threads; ++s) { off[s] = o; o += cnt[s]; }
    run_slices(fill_slice, &j, np, g_threads);
    chain_free(&t);
    return 0;
}

/*
 * Last join level folded into the aggregate: for every matching pair (i, r)
 * COUNT += 1 and SUM += psum[i] + bval[r] (mod 2^64).  psum / bval may be NULL
 * (treated as 0).  out[0..1] = COUNT as a 128-bit value (lo, hi), out[2] = SUM.
 */
int orc_join_agg(const int32_t *pk, int64_t np, const uint64_t *psum,
                 const int32_t *bk, int64_t nb, const uint64_t *bval, uint64_t *out) {
    chain_table t;
    if (chain_build(&t, bk, nb)) return -1;
    u128 acnt[256];
    uint64_t asum[256];
    probe_job j = {&t, pk, bk, psum, bval, NULL, NULL, NULL, NULL, acnt, asum};
    run_slices(agg_slice, &j, np, g_threads);
    u128 count = 0;
    uint64_t sum = 0;
    for (int s = 0; s < g_threads; ++s) { count += acnt[s]; sum += asum[s]; }
    chain_free(&t);
    out[0] = (uint64_t)count;
    out[1] = (uint64_t)(count >> 64);
    out[2] = sum;
    return 0;
}

/* ---------------- nested-loop brute force over a whole join tree ---------- */

typedef struct {
    int nrel;
    const int64_t *nrows;
    const int32_t *const *cols;   /* relation r, column c at cols[coloff[r] + c] */
    const int *coloff;
    int nedge;
    const int *edges;             /* 4 ints per edge: rel_a, col_a, rel_b, col_b */
    const int32_t *preds;         /* 3 per relation: col (<0 none), lo, hi */
    int nagg;
    const int *agg;               /* 3 per term: rel, col, wide */
    int64_t *cur;                 /* chosen row per relation */
    u128 count;
    uint64_t sum;
} nl_state;

static int32_t nl_val(const nl_state *s, int rel, int col, int64_t row) {
    return s->cols[s->coloff[rel] + col][row];
}

static void nl_rec(nl_state *s, int depth) {
    if (depth == s->nrel) {
        uint64_t v = 0;
        for (int a = 0; a < s->nagg; ++a) {
            int rel = s->agg[3 * a], col = s->agg[3 * a + 1], wide = s->agg[3 * a + 2];
            int64_t row = s->cur[rel];
            int64_t x;
            if (wide) {
                uint64_t lo = (uint32_t)nl_val(s, rel, col, row);
                uint64_t hi = (uint32_t)nl_val(s, rel, col + 1, row);
                x = (int64_t)(lo | (hi << 32));
            } else {
                x = (int64_t)nl_val(s, rel, col, row);
            }
            v += (uint64_t)x;
        }
        s->count += 1;
        s->sum += v;
        return;
    }
    for (int64_t row = 0; row < s->nrows[depth]; ++row) {
        const int32_t *p = s->preds + 3 * depth;
        if (p[0] >= 0) {
            int32_t v = nl_val(s, depth, p[0], row);
            if (v < p[1] || v >= p[2]) continue;
        }
        int ok = 1;
        s->cur[depth] = row;
        for (int e = 0; e < s->nedge && ok; ++e) {
            int ra = s->edges[4 * e], ca = s->edges[4 * e + 1];
            int rb = s->edges[4 * e + 2], cb = s->edges[4 * e + 3];
            /* check each edge once, when its later relation is chosen */
            int later = ra > rb ? ra : rb;
            if (later != depth) continue;
            if (nl_val(s, ra, ca, s->cur[ra]) != nl_val(s, rb, cb, s->cur[rb])) ok = 0;
        }
        if (ok) nl_rec(s, depth + 1);
    }
}

/* out[0..1] = COUNT (lo, hi), out[2] = SUM mod 2^64. */
int orc_nested_loop(int nrel, const int64_t *nrows, const int32_t *const *cols,
                    const int *coloff, int nedge, const int *edges, const int32_t *preds,
                    int nagg, const int *agg, uint64_t *out) {
    nl_state s;
    s.nrel = nrel; s.nrows = nrows; s.cols = cols; s.coloff = coloff;
    s.nedge = nedge; s.edges = edges; s.preds = preds; s.nagg = nagg; s.agg = agg;
    s.cur = (int64_t *)calloc((size_t)nrel, sizeof(int64_t));
    if (!s.cur) return -1;
    s.count = 0; s.sum = 0;
    nl_rec(&s, 0);
    free(s.cur);
    out[0] = (uint64_t)s.count;
    out[1] = (uint64_t)(s.count >> 64);
    out[2] = s.sum;
    return 0;
}

/* ---------------- chain aggregate of many queries over one pool ------------
 *
 * The counting of agg_propagation (per-key (count, sum) messages pushed toward
 * relation 0 of the join tree; (c, s) (x) (c', s') = (c c', s c' + s' c))
 * restricted to one query family and with the messages held densely over the
 * key domain: query q joins pool relations r_0 .. r_k (two columns, x = 0 and
 * y = 1) on r_i.y = r_{i+1}.x, keeps the rows of r_0 with lo <= x < hi and
 * returns COUNT(*) and SUM(r_0.x + r_k.y), both modulo 2^64.  Every key must
 * lie in [0, domain).  The queries are taken one at a time by the oracle's
 * threads (orc_set_threads); each query is computed the same way by any
 * thread, so the results do not depend on the thread count.
 */
typedef struct { uint64_t c, s; } cs_pair;

typedef struct {
    int nq;
    const int32_t *qoff, *qrel, *qlo, *qhi;
    const int64_t *pool_n;
    const int32_t *const *pool_x, *const *pool_y;
    int64_t domain;
    uint64_t *out_count, *out_sum;
    int64_t next;   /* next query to take (atomic) */
    int failed;
} chain_job;

/* Zero a message written by relation r: its x positions, or the whole
 * buffer when that is cheaper. */
static void chain_clear(const chain_job *J, int r, cs_pair *m) {
    const int64_t n = J->pool_n[r];
    if (n > J->domain / 4) { memset(m, 0, sizeof(cs_pair) * (size_t)J->domain); return; }
    const int32_t *x = J->pool_x[r];
    for (int64_t i = 0; i < n; ++i) { m[x[i]].c = 0; m[x[i]].s = 0; }
}

/* One query; both buffers are all zero on entry and on return. */
static void chain_one(const chain_job *J, int q, cs_pair *cur, cs_pair *nxt) {
    const int32_t *rel = J->qrel + J->qoff[q];
    const int k = J->qoff[q + 1] - J->qoff[q] - 1;
    const int32_t lo = J->qlo[q], hi = J->qhi[q];
    uint64_t count = 0, sum = 0;
    if (k == 0) {
        const int32_t *x = J->pool_x[rel[0]], *y = J->pool_y[rel[0]];
        for (int64_t i = 0; i < J->pool_n[rel[0]]; ++i)
            if (x[i] >= lo && x[i] < hi) { count += 1; sum += (uint64_t)(int64_t)x[i] + (uint64_t)(int64_t)y[i]; }
        J->out_count[q] = count;
        J->out_sum[q] = sum;
        return;
    }
    /* the message of r_k to r_{k-1}: per x, (rows, SUM of y) */
    {
        const int32_t *x = J->pool_x[rel[k]], *y = J->pool_y[rel[k]];
        for (int64_t i = 0; i < J->pool_n[rel[k]]; ++i) {
            cur[x[i]].c += 1;
            cur[x[i]].s += (uint64_t)(int64_t)y[i];
        }
    }
    /* middle relations: a row's pair is its child's message at y (no term of
     * its own); the message to the parent adds the rows' pairs per x */
    for (int j = k - 1; j >= 1; --j) {
        const int32_t *x = J->pool_x[rel[j]], *y = J->pool_y[rel[j]];
        for (int64_t i = 0; i < J->pool_n[rel[j]]; ++i) {
            const cs_pair m = cur[y[i]];
            nxt[x[i]].c += m.c;
            nxt[x[i]].s += m.s;
        }
        chain_clear(J, rel[j + 1], cur);
        cs_pair *t = cur; cur = nxt; nxt = t;
    }
    /* r_0: the predicate, then (1, x) (x) message at y */
    {
        const int32_t *x = J->pool_x[rel[0]], *y = J->pool_y[rel[0]];
        for (int64_t i = 0; i < J->pool_n[rel[0]]; ++i) {
            if (x[i] < lo || x[i] >= hi) continue;
            const cs_pair m = cur[y[i]];
            count += m.c;
            sum += m.s + (uint64_t)(int64_t)x[i] * m.c;
        }
    }
    chain_clear(J, rel[1], cur);
    J->out_count[q] = count;
    J->out_sum[q] = sum;
}

static void chain_slice(void *p, int64_t lo, int64_t hi, int s) {
    (void)lo; (void)hi; (void)s;
    chain_job *J = (chain_job *)p;
    cs_pair *a = (cs_pair *)calloc((size_t)J->domain, sizeof(cs_pair));
    cs_pair *b = (cs_pair *)calloc((size_t)J->domain, sizeof(cs_pair));
    if (!a || !b) {
        __atomic_store_n(&J->failed, 1, __ATOMIC_RELAXED);
        free(a); free(b);
        return;
    }
    for (;;) {
        const int64_t q = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (q >= J->nq) break;
        chain_one(J, (int)q, a, b);
    }
    free(a); free(b);
}

int orc_chain_agg(int nq, const int32_t *qoff, const int32_t *qrel, const int32_t *qlo,
                  const int32_t *qhi, const int64_t *pool_n, const int32_t *const *pool_x,
                  const int32_t *const *pool_y, int64_t domain, uint64_t *out_count,
                  uint64_t *out_sum) {
    chain_job J;
    J.nq = nq; J.qoff = qoff; J.qrel = qrel; J.qlo = qlo; J.qhi = qhi;
    J.pool_n = pool_n; J.pool_x = pool_x; J.pool_y = pool_y; J.domain = domain;
    J.out_count = out_count; J.out_sum = out_sum; J.next = 0; J.failed = 0;
    int nt = g_threads < nq ? g_threads : nq;
    if (nt < 1) nt = 1;
    run_slices(chain_slice, &J, nt, nt);
    return J.failed ? -1 : 0;
}
