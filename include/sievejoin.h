/*
 * sievejoin.h -- C ABI of the B300 (sm_103a) sieved multi-way join library.
 *
 * SieveJoin (Sec. 2.2) answers a multi-way equi-join in two phases:
 *   1. pruning: Bloom filters are built on join keys and propagated along the
 *      join path; every relation keeps only the tuples whose join keys pass
 *      the filters arriving from its neighbours (Bloomjoin, Sec. 2.1, extended
 *      to n relations), so tuples that cannot reach the result die early;
 *   2. enumeration: an ordinary binary join plan (here a hash join) runs over
 *      the pruned relations.
 * Bloom filters have no false negatives (Sec. 1), so the result is exactly the
 * natural join of the unpruned relations.
 *
 * Conventions shared by every entry point
 *   - A context owns one CUDA device and one stream.  Every call enqueues its
 *     work on that stream in call order.  Calls on one context must not run
 *     concurrently from several host threads.
 *   - Columns are int32, column-major (one contiguous array per column),
 *     16-byte aligned device memory.  Relations have at most SJ_MAX_COLS
 *     columns and fewer than 2^31 rows.  Any int32 value is a valid key.
 *   - Return value: SJ_OK (0) or an error code.  sj_last_error() gives a
 *     one-line description of the last failure on a context.  A failed call
 *     leaves its output arguments untouched and frees what it allocated.
 *   - Device memory is taken from the allocator given to sj_create (or, when
 *     none is given, from the device's stream-ordered pool via
 *     cudaMallocAsync on the context stream).
 *   - Device-side waits (the compaction scans' waits on the counts of earlier
 *     chunks and tiles, and the probe chains of the hash tables) are
 *     bounded: when a bound is hit the kernel
 *     records the error in a device status word and returns; the next call
 *     that synchronises reports SJ_ETIMEOUT or SJ_ETABLEFULL.
 */
#ifndef SIEVEJOIN_H
#define SIEVEJOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SJ_API __attribute__((visibility("default")))
#else
#define SJ_API
#endif

#define SJ_MAX_COLS 8    /* columns per relation */
#define SJ_MAX_REL 8     /* relations per join path */
#define SJ_MAX_PROBES 4  /* filters probed by one sieve step */
#define SJ_MAX_TERMS 8   /* SUM terms / projected output columns */

typedef int sj_status;
enum {
    SJ_OK = 0,
    SJ_EINVAL = 1,      /* bad argument: null pointer, column out of range, not a tree, ... */
    SJ_ENOMEM = 2,      /* the allocator returned NULL */
    SJ_ETABLEFULL = 3,  /* a hash-table probe chain exceeded its bound */
    SJ_ETIMEOUT = 4,    /* a bounded device wait gave up */
    SJ_EOVERFLOW = 5,   /* COUNT(*) reached 2^63 */
    SJ_ECUDA = 6        /* a CUDA runtime call failed; see sj_last_error */
};

typedef struct sj_ctx sj_ctx;
typedef struct sj_rel_s *sj_rel;
typedef struct sj_filter_s *sj_filter;

/* Allocator callbacks: return 256-byte aligned device memory, or NULL. */
typedef void *(*sj_alloc_fn)(size_t bytes, void *user);
typedef void (*sj_free_fn)(void *ptr, size_t bytes, void *user);

/* ------------------------------------------------------------------ context */

/*
 * Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  `alloc`/`free_` may both be NULL (use
 * cudaMallocAsync / cudaFreeAsync on the stream) or both be set; `user` is
 * passed back to them.  The context owns a small device status word and a
 * scratch area for the compaction scans.
 */
SJ_API sj_status sj_create(sj_ctx **out, int device, void *cuda_stream, sj_alloc_fn alloc,
                    sj_free_fn free_, void *user);
/* Synchronise the stream and release everything the context still owns. */
SJ_API sj_status sj_destroy(sj_ctx *ctx);
/* Wait for all work enqueued on the context; report device-side errors. */
SJ_API sj_status sj_sync(sj_ctx *ctx);
SJ_API const char *sj_last_error(const sj_ctx *ctx);
SJ_API const char *sj_status_str(sj_status s);
/* Library version as "major.minor.patch". */
SJ_API const char *sj_version(void);

/* ---------------------------------------------------------------- relations */

enum {
    SJ_DEVICE_BORROW = 0, /* keep the caller's device pointers; they must outlive the handle */
    SJ_DEVICE_COPY = 1,   /* copy device columns into library memory */
    SJ_HOST_COPY = 2,     /* copy host columns (pinned memory is fastest) to the device */
    SJ_HOST_MAPPED = 3    /* keep page-locked host columns where they are; kernels read them
                             over the host link each time they touch them */
};

/*
 * Load a columnar relation (the paper's storage is column-oriented, Sec. 3.1).
 * `cols` is an array of `ncols` column pointers with `nrows` int32 values
 * each.  With SJ_HOST_COPY the copies are enqueued on the context stream and
 * the host buffers must stay valid until the next sj_sync (or any call that
 * synchronises).  With SJ_HOST_MAPPED nothing is copied: every column must be
 * page-locked host memory the device can address (cudaHostAlloc or
 * cudaHostRegister with the mapped flag, or any pinned allocation on a system
 * with unified addressing), 16-byte aligned, and it must outlive the handle.
 * Kernels read such columns from host memory, so only what they touch
 * crosses the link: sj_sieve_join copies the columns it reads in full (a
 * relation's first tested key column, the column a filter is built from
 * before that, the join columns of a relation it never sieves) to the device
 * in bulk on a copy stream, in the order the pruning needs them, and the
 * pruning of each relation waits only for its own columns; the surviving rows
 * of the other columns and the SUM terms of matching rows are read in place
 * (the paper's point: tuples that cannot reach the result are dropped before
 * they are moved).  Other calls read mapped columns in place.  Errors:
 * SJ_EINVAL (ncols outside 1..SJ_MAX_COLS, nrows < 0 or >= 2^31, a null or
 * misaligned pointer, host memory the device cannot address), SJ_ENOMEM.
 */
SJ_API sj_status sj_load_relation(sj_ctx *ctx, int ncols, const int32_t *const *cols, int64_t nrows,
                           int where, sj_rel *out);
/* Row count (host-known for every handle this library returns), column count and
 * device column pointers (array of SJ_MAX_COLS entries; may be NULL). */
SJ_API sj_status sj_rel_info(sj_rel rel, int64_t *nrows, int *ncols, const int32_t **cols);
SJ_API sj_status sj_free_rel(sj_ctx *ctx, sj_rel rel);

/* ------------------------------------------------------------ Bloom filters */

enum { SJ_REGBLOCKED32 = 0, SJ_BLOCKED256 = 1, SJ_CLASSIC = 2 };

/*
 * Filter parameters.  The paper sizes Bloomjoin's filter at one bit per tuple
 * (Sec. 2.1 step 2) and leaves the hash family and layout open (Sec. 1 cites
 * Kirsch and Mitzenmacher).  Here: h = fmix64(uint32(key) xor seed)
 * (MurmurHash3's finaliser); m = 256 * max(1, ceil(bits_per_key * n / 256))
 * bits for n inserted rows, stored as m / 32 uint32 words; word w holds bits
 * 32w..32w+31, least significant bit first.
 *   SJ_REGBLOCKED32 (default): all k bits of a key in one 32-bit word,
 *                  word = ((h >> 32) * (m / 32)) >> 32, bit i = (h >> 5i) & 31,
 *                  k <= 6.  One load per probe, one atomicOr per insert.
 *   SJ_BLOCKED256: block b = ((h >> 32) * (m / 256)) >> 32; bits (h >> 8i) & 255,
 *                  i < k, inside that 256-bit block (eight words); k <= 4.
 *   SJ_CLASSIC:    bits (h1 + i*h2) mod m, h1 = h & 0xffffffff,
 *                  h2 = (h >> 32) | 1; k <= 8.
 * A zeroed struct reads as: bits_per_key 8, k 3, SJ_REGBLOCKED32, seed 0.
 */
typedef struct {
    uint32_t bits_per_key;
    uint32_t k;
    uint32_t layout;
    uint32_t reserved;
    uint64_t seed;
} sj_filter_params;

/* Range predicate lo <= rel[col] < hi on one relation; col < 0 means none. */
typedef struct {
    int32_t col;
    int32_t lo;
    int32_t hi;
} sj_pred;

/*
 * Build a Bloom filter over column `key_col` of `rel` (Sec. 2.1 step 1), from
 * the rows passing `pred` (NULL = all rows).  The handle is reusable across
 * queries (Sec. 2.3): pass it to sj_sieve any number of times.  Errors:
 * SJ_EINVAL, SJ_ENOMEM, SJ_ECUDA.
 */
SJ_API sj_status sj_build_filter(sj_ctx *ctx, sj_rel rel, int key_col, const sj_pred *pred,
                          const sj_filter_params *params, sj_filter *out);
/* Synchronise, then report the block count, inserted rows and the device word
 * array (nblocks * 8 uint32 words). */
SJ_API sj_status sj_filter_info(sj_ctx *ctx, sj_filter f, uint64_t *nblocks, uint64_t *n_inserted,
                         const uint32_t **words);
/* Membership test of n device keys (Sec. 2.1 step 3): out[i] = 1 if keys[i]
 * may be in the filter, 0 if it certainly is not.  out is n device bytes. */
SJ_API sj_status sj_filter_probe(sj_ctx *ctx, sj_filter f, const int32_t *keys, int64_t n,
                          uint8_t *out);
SJ_API sj_status sj_free_filter(sj_ctx *ctx, sj_filter f);

/*
 * Insert maintenance of a built filter (Sec. 2.4).  The `nrows` rows of
 * `rel` are new tuples of the relation whose column the filter `f` was built
 * over; `key_col` is that column in `rel`.  A row first meets the filters the
 * relation receives from its other neighbours (ngate of them, 0 <= ngate <=
 * SJ_MAX_PROBES: gates[j] tested on column gate_cols[j]): a row that fails any
 * cannot reach the join result and is dropped (SJ_INSERT_GATED).  A row whose
 * key the filter already contains needs no update (SJ_INSERT_CONTAINED).  The
 * key bits of every other row are set (SJ_INSERT_NEW): the filter changed, and
 * those rows are the ones whose effect must be followed to the adjacent
 * relations -- their neighbours' tuples that join with them may now survive a
 * sieve by this filter (the paper's search from the relation to its adjacent
 * relations).  Containment is judged against the filter as it was before the
 * call, so the outcome does not depend on row order; the filter keeps its size
 * (its false-positive rate grows as keys are added) and its inserted-row count
 * grows by the SJ_INSERT_NEW rows.  status_out is NULL or nrows device bytes
 * receiving each row's outcome; counts is NULL or host int64[3] receiving the
 * number of rows of each outcome (the call then synchronises).  Errors:
 * SJ_EINVAL (null filter or relation, column out of range, ngate out of
 * range), SJ_ENOMEM, SJ_ECUDA.
 */
enum { SJ_INSERT_GATED = 0, SJ_INSERT_CONTAINED = 1, SJ_INSERT_NEW = 2 };
SJ_API sj_status sj_filter_insert(sj_ctx *ctx, sj_filter f, sj_rel rel, int key_col, int ngate,
                                  const int *gate_cols, const sj_filter *gates, uint8_t *status_out,
                                  int64_t *counts);

/*
 * One sieve step (Sec. 2.2, pruning phase): keep, in input order, the rows of
 * `rel` that pass `pred` (NULL = none) and whose column key_cols[j] passes
 * filters[j] for every j < nprobe (0 <= nprobe <= SJ_MAX_PROBES).  The kept
 * rows (all columns) go to a new relation handle.  Synchronises to learn the
 * row count, which it also writes to *nrows_out when that is not NULL.
 */
SJ_API sj_status sj_sieve(sj_ctx *ctx, sj_rel rel, int nprobe, const int *key_cols,
                   const sj_filter *filters, const sj_pred *pred, sj_rel *out,
                   int64_t *nrows_out);

/*
 * Allocation-free sieve step.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory where they sieve --
 * code running inside a custom allocator or memory manager, or a runtime that
 * only hands out buffers it reserved up front and forbids cudaMalloc on its
 * hot path.  It needs no context, calls no cudaMalloc, cudaFree or other
 * allocating routine, and does the same work as sj_sieve with one filter and
 * no predicate: the rows of the relation (ncols device columns in_cols, nrows
 * rows) whose column key_col passes the filter are written, in input order,
 * to out_cols (ncols device columns with room for nrows rows each), and the
 * kept-row count to the device uint64 *out_count.  The filter is given by its
 * word array (nblocks * 8 uint32, the layout sj_filter_params describes; the
 * words of a filter built by sj_build_filter are reported by sj_filter_info)
 * and its params (k, layout and seed; bits_per_key is not used).  All
 * pointers are device pointers, 16-byte aligned.  `status` is NULL or a
 * device uint32 that receives SJ_ETIMEOUT-style bits (1 = a bounded wait gave
 * up) and is not cleared by the call.  With status NULL the bits go to a word
 * inside the library that no caller can read, so a wait that gave up cannot
 * be reported: pass a status word to learn that out_cols and *out_count are
 * not valid.  The work is enqueued on cuda_stream (NULL = legacy default
 * stream) of the current device; nothing is synchronised.
 *
 * Its scratch is one fixed device array of about 66 KiB inside this library
 * (held by every GPU that loads the library until the process exits), sized
 * for SJ_NOALLOC_MAX_ROWS rows; larger relations are rejected with SJ_EINVAL.
 * Every call shares that array and clears what must start at zero, so calls
 * that overlap on the GPU (other streams, other host threads) race: serialise
 * them.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  On failure *err (when err is not NULL) points to a
 * static message.  Errors: SJ_EINVAL, SJ_ECUDA.
 */
#define SJ_NOALLOC_MAX_ROWS (1ll << 27)
SJ_API sj_status sj_sieve_noalloc(void *cuda_stream, int ncols, const int32_t *const *in_cols,
                                  int64_t nrows, int key_col, const uint32_t *filter_words,
                                  uint64_t nblocks, const sj_filter_params *params,
                                  int32_t *const *out_cols, uint64_t *out_count, uint32_t *status,
                                  const char **err);

/* ---------------------------------------------------------------- join path */

/* Equality rel_a.col_a = rel_b.col_b. */
typedef struct {
    int32_t rel_a, col_a, rel_b, col_b;
} sj_edge;

/*
 * A tree-shaped equi-join over nrel relations (a chain R1 - R2 - ... - Rn is
 * the paper's running case, Sec. 2.2; a star is the bitvector-filtering case
 * of Sec. 1).  nrel - 1 edges must connect all relations without a cycle.
 * `root` is where pass 1 of the sieve ends (-1 = the last relation, so that a
 * chain is pruned R1 -> Rn and then Rn -> R1).  `preds` is NULL or holds
 * one predicate per relation (col < 0 for none).
 */
typedef struct {
    int32_t nrel;
    int32_t root;
    const sj_rel *rels;
    const sj_edge *edges;
    const sj_pred *preds;
} sj_path;

enum {
    SJ_FWD_BWD = 0,  /* pass 1 toward the root, then pass 2 back to the leaves (Sec. 2.2) */
    SJ_BWD_ONLY = 1, /* the paper's one-pass backward pruning: pass 2 only */
    SJ_NO_SIEVE = 2  /* apply the predicates only */
};

/*
 * leaf_filters (NULL, or one entry per relation) hands in reusable filters
 * (Sec. 2.3): for a leaf v of the join tree, a non-NULL leaf_filters[v] is
 * used in pass 1 instead of building the filter v sends to its parent.  It
 * must have been built (sj_build_filter) over the column of v on that edge,
 * from v's rows passing v's predicate, with the same filter parameters;
 * entries of non-leaves are ignored.  Handed-in filters are not freed.
 */
typedef struct {
    int32_t passes;
    int32_t reserved;
    sj_filter_params filter;
    const sj_filter *leaf_filters;
} sj_sieve_opts;

#define SJ_MAX_STEPS 32
typedef struct {
    int32_t nsteps;
    int32_t reserved;
    struct {
        int32_t kind; /* 0 = predicate select, 1 = pass-1 sieve, 2 = pass-2 sieve */
        int32_t rel;
        int64_t rows_in;
        int64_t rows_out;
    } step[SJ_MAX_STEPS];
    int64_t rows_final[SJ_MAX_REL];
    uint64_t filter_bytes; /* device bytes of all filters built */
} sj_sieve_stats;

/*
 * The whole pruning phase (Sec. 2.2).  Predicates are applied first.  Pass 1
 * visits the join tree from the leaves to the root: a relation is sieved by
 * the filters of its children, then builds -- from its surviving rows only
 * -- the filter it sends to its parent.  Pass 2 walks from the root back to
 * the leaves: each relation is sieved by the filter its parent built from the
 * parent's surviving rows.  On return out_sieved[i] is a new handle holding
 * relation i's surviving rows in input order (free with sj_free_rel).  The
 * join over them equals the join over the inputs.  Synchronises once at the
 * end.  `opts` NULL = SJ_FWD_BWD with default filter parameters; `stats` may
 * be NULL.
 */
SJ_API sj_status sj_sieve_path(sj_ctx *ctx, const sj_path *path, const sj_sieve_opts *opts,
                        sj_rel *out_sieved, sj_sieve_stats *stats);

/*
 * The pruning phases (Sec. 2.2) of `nq` queries in one call, for a serving
 * runtime that has several queries in hand at once.  paths[q] and, unless
 * `opts` is NULL, opts[q] describe query q exactly as for sj_sieve_path
 * (opts[q].leaf_filters hands in query q's reusable leaf filters, Sec. 2.3).
 * The queries' sieve steps and filter builds run in lock step: an operation
 * runs at one more than the level of everything it reads (the step that
 * produced its input relation, the builds of the filters it probes), and all
 * steps of one level, over all queries, are one kernel launch, as are all
 * builds of one level.  A batch therefore takes two launches per level of its
 * longest schedule instead of a launch per step and build of every query.
 * On return out_sieved[q * SJ_MAX_REL + i] is query q's relation i after
 * pruning (a new handle; free with sj_free_rel), identical, rows and order,
 * to what sj_sieve_path returns for that query alone; stats (NULL, or nq
 * entries) as for sj_sieve_path.  Every intermediate relation of the batch
 * stays allocated until the call ends.  Synchronises once.  SJ_EINVAL if any
 * query is invalid (nothing is then enqueued).  nq = 0 does nothing.
 */
SJ_API sj_status sj_sieve_path_batch(sj_ctx *ctx, int nq, const sj_path *paths,
                                     const sj_sieve_opts *opts, sj_rel *out_sieved,
                                     sj_sieve_stats *stats);

enum { SJ_COUNT_SUM = 0, SJ_MATERIALIZE = 1 };

/* A column reference: SUM term or projected output column.  wide = 1 reads an
 * int64 stored as two int32 columns col (low word) and col + 1 (high word). */
typedef struct {
    int32_t rel, col, wide, reserved;
} sj_colref;

typedef struct {
    uint64_t count;          /* COUNT(*), exact */
    uint64_t sum;            /* SUM of the terms as int64, two's complement mod 2^64 */
    uint64_t intermediate;   /* tuples materialised by the non-final join levels */
    sj_rel rows;             /* SJ_MATERIALIZE: one column per ref, caller frees */
} sj_result;

/*
 * The enumeration phase (Sec. 2.2): a left-deep binary hash join over the
 * path.  It starts at relation 0 and repeatedly adds the lowest-index
 * relation adjacent to those already joined.  Every non-final level builds an
 * open-addressing hash table on the new relation and materialises the
 * intermediate tuples (only the columns later levels need).
 *   SJ_COUNT_SUM: the last level probes a per-key (count, sum) table and
 *     accumulates COUNT(*) and SUM over `refs` (int64 per result tuple,
 *     wrapped mod 2^64); result->rows is NULL.
 *   SJ_MATERIALIZE: result->rows holds one int32 column per ref (wide must be
 *     0), rows in unspecified order.
 * `inputs` NULL joins the path's own relations after applying its predicates;
 * otherwise inputs[i] replaces relation i and is taken as already filtered by
 * predicate i (the output of sj_sieve_path).  Synchronises at every level.
 * A hash table's build side holds at most 2^30 rows (SJ_EINVAL beyond: slot
 * counts and row ids are 32-bit on the device); sj_sieve_join has the same
 * limit.  Errors: SJ_EINVAL, SJ_ENOMEM, SJ_EOVERFLOW (COUNT >= 2^63),
 * SJ_ETABLEFULL, SJ_ETIMEOUT, SJ_ECUDA.
 */
SJ_API sj_status sj_join(sj_ctx *ctx, const sj_path *path, const sj_rel *inputs, int mode, int nrefs,
                  const sj_colref *refs, sj_result *result);

/* ------------------------------------------------------------ cyclic query */

typedef struct {
    int64_t edges_in;        /* rows of the edge relation */
    int64_t edges_sieved;    /* edges left after the pruning rounds */
    uint64_t candidates;     /* closing pairs looked up */
    uint64_t filter_passed;  /* of those, passed by the closing-pair filter */
    uint64_t triangles;      /* sum of counts */
} sj_tri_stats;

/*
 * Cyclic triangle query E(a,b) |x| E(b,c) |x| E(c,a) over a directed edge
 * relation (columns 0 = source, 1 = target; distinct edges, no self-loops),
 * answered as nsub subqueries in one launch: counts[i] = number of ordered
 * (a, b, c) with a->b, b->c, c->a and cuts[i] <= a < cuts[i+1] (a below
 * cuts[0] counts in subquery 0, at or above cuts[nsub] in subquery nsub-1).
 * Pruning (Sec. 2.2) runs `sieve_rounds` rounds (default 2 when < 0): filters
 * over the sources and targets keep the edges whose target has an out-edge
 * and whose source has an in-edge.  Enumeration follows Sec. 2.3's cyclic
 * case: the filter of the closing condition -- here over the packed pair
 * (c, a) -- is rebuilt on the fly from the pruned edges and screens every
 * wedge before an exact pair-set lookup.  Each directed 3-cycle is walked
 * once, from its smallest vertex a (an edge a -> b with a < b, then c > a
 * from the shorter of out(b) and in(a)), and its three ordered answers are
 * added to the subqueries of a, b and c.  The pair filter uses the register-blocked
 * layout with `params`' bits_per_key, k (<= 6) and seed (NULL = defaults).
 * 1 <= nsub <= 256; `cuts` (nsub + 1 increasing values) and `counts` are host
 * arrays.  Synchronises.  Errors: SJ_EINVAL, SJ_ENOMEM, SJ_ETABLEFULL, SJ_ECUDA.
 */
SJ_API sj_status sj_triangles(sj_ctx *ctx, sj_rel edges, int nsub, const int32_t *cuts,
                              int sieve_rounds, const sj_filter_params *params, uint64_t *counts,
                              sj_tri_stats *stats);

/* ---------------------------------------------------------------- serving */

/*
 * A query server over resident relations.  Queries (tree-shaped equi-joins
 * over registered relations, returning COUNT(*) and SUM) are queued and run
 * by `nslots` workers, each with its own context and CUDA stream, so queries
 * that arrive while others run are admitted as soon as a slot and enough of
 * the device-memory budget are free, and their kernels overlap on the GPU
 * (continuous batching).  With cache_filters the server keeps the reusable
 * leaf filters of pass 1 (Sec. 2.3: filters pre-built for one query serve
 * later queries that contain the same relation, column and predicate), keyed
 * by (relation, column, predicate), on the device until it is destroyed.
 * Results are identical to running each query alone.
 */
typedef struct sj_server sj_server;

typedef struct {
    int32_t device;
    int32_t nslots;          /* concurrent queries (workers); default 4 */
    uint64_t hbm_budget;     /* bytes in-flight queries may use; 0 = half the free memory */
    int32_t passes;          /* sieve schedule (SJ_FWD_BWD, ...) */
    int32_t cache_filters;   /* 1 = reuse leaf filters across queries */
    sj_filter_params filter; /* parameters of every filter the server builds */
    int32_t batch;           /* > 1: a worker takes up to `batch` queued queries at once and runs
                                their pruning phases as one sj_sieve_path_batch call, then
                                each query's join; 0 or 1 = one query at a time */
    int32_t reserved;
    uint64_t batch_max_rows; /* batch mode: a query whose relations hold more rows than this
                                in all runs alone, so it does not hold back a batch of small
                                ones (0 = no limit) */
} sj_server_opts;

typedef struct {
    int32_t nrel;
    int32_t root;                      /* as in sj_path; -1 = last relation */
    int32_t rel[SJ_MAX_REL];           /* registered relation ids */
    sj_edge edges[SJ_MAX_REL - 1];     /* rel_a / rel_b are positions 0..nrel-1 */
    sj_pred preds[SJ_MAX_REL];         /* col < 0 for none */
    int32_t nterms;
    sj_colref terms[SJ_MAX_TERMS];     /* SUM terms; rel is a position */
} sj_query;

typedef struct {
    uint64_t ticket;
    sj_status status;
    int32_t cache_hits;      /* leaf filters taken from the cache */
    uint64_t count;
    uint64_t sum;
    double submit_ms;        /* host clock, ms since server creation */
    double start_ms;         /* admitted to a slot */
    double done_ms;          /* result on the host */
} sj_completion;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t cache_hits, cache_misses, cached_filters;
    uint64_t peak_inflight_bytes;
    int32_t peak_concurrency;
    int32_t peak_batch;      /* most queries pruned by one sj_sieve_path_batch call */
    uint64_t batches;        /* sj_sieve_path_batch calls (batch mode) */
} sj_server_stats;

/* Create a server (starts its workers).  Errors: SJ_EINVAL, SJ_ECUDA, SJ_ENOMEM. */
SJ_API sj_status sj_server_create(sj_server **out, const sj_server_opts *opts);
/* Register a resident relation: `ncols` device columns of `nrows` rows,
 * 16-byte aligned, borrowed (they must outlive the server).  Returns its id.
 * Register relations before submitting the queries that use them; this call
 * must not run concurrently with sj_server_submit. */
SJ_API sj_status sj_server_add_relation(sj_server *srv, int ncols, const int32_t *const *dev_cols,
                                        int64_t nrows, int32_t *rel_id);
/* Queue a query (copied); returns at once with its ticket.  SJ_EINVAL if the
 * query names an unknown relation or column or is not a tree. */
SJ_API sj_status sj_server_submit(sj_server *srv, const sj_query *q, uint64_t *ticket);
/* Take up to `max` finished queries; wait up to `wait_ms` for the first one. */
SJ_API sj_status sj_server_poll(sj_server *srv, sj_completion *out, int max, int *n, int wait_ms);
SJ_API sj_status sj_server_stats_get(sj_server *srv, sj_server_stats *stats);
/* Finish queued queries, stop the workers and free cached filters. */
SJ_API sj_status sj_server_destroy(sj_server *srv);

/*
 * The whole method in one call: sj_sieve_path, then sj_join over the sieved
 * relations, which are freed before returning (Sec. 2.2: pruning phase, then
 * enumeration phase).  `opts` and `stats` as for sj_sieve_path, the rest as
 * for sj_join.  Errors: those of the two calls.
 *
 * Repeated COUNT_SUM queries of one shape (same relation handles and device
 * buffers, edges, predicates, options and SUM columns; `stats` NULL) run
 * faster: the first call is exact and synchronises per join level; later
 * calls keep every size on the device, with intermediate buffers of twice the
 * previous run's size, and synchronise once (an intermediate that outgrows its
 * buffer is detected and the call reruns exactly, so the result never
 * depends on this); from the third call the query is captured once as a CUDA
 * graph and replayed (see sj_graph_stats, sj_graphs_enable).  The contents of
 * the relations may change between calls.  Temporaries come from a
 * per-context arena that grows to the largest call.
 */
SJ_API sj_status sj_sieve_join(sj_ctx *ctx, const sj_path *path, const sj_sieve_opts *opts,
                               int mode, int nrefs, const sj_colref *refs, sj_result *result,
                               sj_sieve_stats *stats);

/*
 * Self-test of the bounded device waits (no counterpart in the paper): one
 * warp polls a device flag that nothing sets, with the bound and backoff of
 * the compaction scans' waits.  The wait gives up after about a second, records
 * SJ_ETIMEOUT in the status word and the kernel finishes; this call then
 * synchronises and returns SJ_ETIMEOUT, and the context stays usable.  It
 * faults or traps nothing.
 */
SJ_API sj_status sj_selftest_wait_timeout(sj_ctx *ctx);

/* ---------------------------------------------------------------- profiling */

enum {
    SJ_K_BLOOM_BUILD = 0,   /* Bloom filter build */
    SJ_K_SIEVE = 1,         /* probe + stream compaction (also predicate selects) */
    SJ_K_HT_BUILD = 2,      /* hash-table inserts, offsets scan and row scatter */
    SJ_K_HT_PROBE = 3,      /* probe + match compaction of a join level */
    SJ_K_HT_EXPAND = 4,     /* intermediate-tuple output of a join level */
    SJ_K_AGG = 5,           /* per-key aggregate table build and final probe */
    SJ_K_OTHER = 6,
    SJ_K_COUNT = 7
};

/*
 * Per-kernel-class timing with CUDA events recorded on the context stream
 * around every launch while enabled.  sj_prof_read synchronises and returns,
 * for class `kind`: launches, summed device milliseconds and the summed
 * algorithmic bytes (the bytes the operation must move, counted from its
 * inputs and outputs).  sj_counters reports, since the last sj_prof_reset,
 * every kernel this library launched on the context (profiled or not) and
 * the bytes it copied host-to-device and device-to-host.
 */
SJ_API sj_status sj_prof_enable(sj_ctx *ctx, int on);
/* Restrict profiling to the kernel classes whose bit (1 << SJ_K_*) is set in
 * `mask` (default: all).  Each profiled launch costs two event records, which
 * inside a CUDA graph are nodes of their own: profiling one class keeps the
 * timing of the others undisturbed. */
SJ_API sj_status sj_prof_kinds(sj_ctx *ctx, uint32_t mask);
SJ_API sj_status sj_prof_reset(sj_ctx *ctx);
SJ_API sj_status sj_prof_read(sj_ctx *ctx, int kind, int64_t *launches, double *ms, double *bytes);
SJ_API sj_status sj_counters(sj_ctx *ctx, int64_t *launches, int64_t *h2d_bytes, int64_t *d2h_bytes);
/* CUDA-graph use of sj_sieve_join since the context was created.  A query
 * shape (relations, their device buffers, edges, predicates, options) runs
 * exactly on its first call; later calls keep every size on the device, with
 * intermediate buffers sized from the previous run; the third call captures a
 * CUDA graph and the fourth and later calls replay it.  `replays`, successful
 * `captures` and failed `failures` (any may be null); `why` (optional, `len`
 * bytes, NUL-terminated) receives the reason of the last failed capture. */
SJ_API sj_status sj_graph_stats(sj_ctx *ctx, int64_t *replays, int64_t *captures, int64_t *failures,
                                char *why, int len);
/* Turn the capture of CUDA graphs by sj_sieve_join on (default) or off for
 * this context; off also drops the graphs held.  A capture costs the calling
 * thread about as much host time as the query it captures, which pays off
 * for query shapes that repeat many times and not for a stream of mostly
 * distinct shapes (the serving runtime's workers turn it off). */
SJ_API sj_status sj_graphs_enable(sj_ctx *ctx, int on);
/* Device idle time (ms) between the end of a profiled launch of each class and
 * the start of the next profiled launch (host work, syncs, memsets), summed
 * per class into gap_ms[SJ_K_COUNT]. */
SJ_API sj_status sj_prof_gaps(sj_ctx *ctx, double *gap_ms);

#ifdef __cplusplus
}
#endif
#endif /* SIEVEJOIN_H */
